"""Multi-rank path on CPU: 2 gloo ranks split photon ranges of a batch, walk them with
the oracle (the same walk as the GPU, bit for bit) and sum the int64 counts with
all_reduce; the result equals the single-rank run exactly.  A rank that fails before
the reduction is reported on the other rank by the process-group timeout (host-made
failure; no device involved)."""
import datetime
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2409_00165_gb300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _batch():
    rng = np.random.default_rng(21)
    n_st, L = 5, 2
    return dict(n_stacks=n_st, n_wl=1, max_layers=L, n_layers=np.array([1, 2, 2, 1, 2], np.int32),
                mu_s=rng.uniform(1, 10, n_st * L), mu_a=rng.uniform(0.05, 1, n_st * L),
                g=rng.uniform(0, 0.9, n_st * L), n_layer=rng.uniform(1.2, 1.7, n_st * L),
                thickness=rng.uniform(0.1, 0.5, n_st * L),
                n_photons=np.array([3001, 17, 2500, 0, 999], np.int64), seed=77)


def _paint_batch():
    """The strong-scaling split of the benchmark: one paint-layer spectrum (here 12
    wavelengths x 3000 photons) whose photon ids are split across the ranks."""
    import oracle
    from paper_2409_00165_gb300 import workloads as W
    m = W.paint_layer(n_wl=12, photons=3000, seed=5)
    p = oracle.mie_properties(m["wl"], m["nm"], m["species_group"], m["n_p"], m["radius"],
                              m["vol_frac"])
    return dict(n_stacks=1, n_wl=12, max_layers=1, mu_s=p["mu_s"].reshape(-1),
                mu_a=p["mu_a"].reshape(-1), g=p["g"].reshape(-1),
                n_layer=m["nm"].real.reshape(-1), thickness=m["thickness"],
                n_photons=np.full(12, 3000, np.int64), seed=m["seed"])


def _worker(rank, world, port, fail_rank, q, which="stacks"):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=10))
    try:
        b = _batch() if which == "stacks" else _paint_batch()
        first, count = shard.photon_ranges(b["n_photons"], rank, world)
        bb = dict(b, photon_first=first, n_photons=count)
        c = torch.as_tensor(oracle.mc_run(bb, fp32=True))
        if rank == fail_rank:
            raise RuntimeError("rank failed before the reduction")
        shard.allreduce_counts(c)
        q.put((rank, "ok", c.numpy()))
    except Exception as exc:  # report, do not hang
        q.put((rank, "error", type(exc).__name__))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def _run(world, fail_rank=-1, which="stacks"):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, fail_rank, q, which))
          for r in range(world)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in ps:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    return sorted(out, key=lambda t: t[0])


def test_photon_ranges_partition():
    for n in (0, 1, 7, 1000, 12345):
        for w in (1, 2, 3, 8):
            parts = [shard.photon_range(n, r, w) for r in range(w)]
            assert sum(c for _, c in parts) == n
            assert all(parts[i][0] + parts[i][1] == parts[i + 1][0] for i in range(w - 1))
            f, c = shard.photon_ranges([n, n + 1], 0, w)
            assert f[0] == 0


def test_two_gloo_ranks_sum_to_the_single_run(orc):
    single = orc.mc_run(_batch(), fp32=True)
    res = _run(2)
    assert [r[1] for r in res] == ["ok", "ok"]
    for _, _, c in res:
        assert np.array_equal(c, single)


def test_two_gloo_ranks_split_one_paint_layer_spectrum(orc):
    """bench.py --scaling strong: the ranks' photon ranges of one spectrum, summed by
    all_reduce, equal the single-rank spectrum bit for bit."""
    single = orc.mc_run(_paint_batch(), fp32=True)
    res = _run(2, which="paint")
    assert [r[1] for r in res] == ["ok", "ok"]
    for _, _, c in res:
        assert np.array_equal(c, single)
    assert np.all(single[:, :4].sum(axis=1) == 3000)


def test_failed_rank_is_reported_not_hung():
    res = _run(2, fail_rank=1)
    assert res[1][1] == "error"
    assert res[0][1] == "error"   # rank 0's all_reduce ends with an error (peer gone)
