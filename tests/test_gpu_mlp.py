"""Parity of the tcgen05 surrogate kernels (GEMM, forward, backward, Adam) with the
FP64 NumPy oracle (oracle/mlp.py), through the C-ABI."""
import math

import numpy as np
import pytest

from oracle import mlp as M
from paper_2409_00165_gb300 import fos

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

REAL = [(256, 9), (256, 256), (256, 256), (256, 256), (3, 256)]


def _bf16(rng, shape, scale=1.0):
    return torch.as_tensor(rng.normal(0, scale, size=shape), dtype=torch.float32).to(
        torch.bfloat16).cuda()


@pytest.mark.parametrize("Mr,N,K,splits", [(128, 256, 64, 1), (256, 256, 256, 1),
                                          (300, 64, 512, 1), (64, 256, 8192, 32),
                                          (1000, 256, 256, 4), (128, 64, 64, 1),
                                          (8192, 256, 256, 1)])
def test_gemm_matches_fp64(Mr, N, K, splits):
    rng = np.random.default_rng(Mr * 7 + N + K)
    A = _bf16(rng, (Mr, K))
    B = _bf16(rng, (N, K))
    C = torch.zeros((splits, Mr, N), dtype=torch.float32, device="cuda")
    fos.check(fos.fos_gemm_bf16(A, B, C, splits), "fos_gemm_bf16")
    a = A.float().double().cpu().numpy()
    b = B.float().double().cpu().numpy()
    ref = a @ b.T
    bound = np.abs(a) @ np.abs(b).T
    got = C.sum(dim=0).double().cpu().numpy()
    assert np.all(np.abs(got - ref) <= 1e-5 * bound + 1e-6)


def _stats(x):
    mean, std = x.mean(axis=0), x.std(axis=0) + 1e-3
    lo, hi = x.min(axis=0), x.max(axis=0)
    st = np.zeros(64, np.float32)
    st[0:9], st[16:25], st[32:41], st[48:57] = mean, std, lo, hi
    st[16 + 9:32] = 1.0
    return st, mean, std


def _params(model, member=0):
    P = fos.fos_surrogate_param_count()
    w_off, b_off = fos.fos_surrogate_param_offsets()
    mb = fos.fos_surrogate_model_bytes()
    theta = model[member * mb: member * mb + 4 * P].view(torch.float32).double().cpu().numpy()
    out = []
    shapes = [(256, 64), (256, 256), (256, 256), (256, 256), (64, 256)]
    for l, ((o, i), (ro, ri)) in enumerate(zip(shapes, REAL)):
        W = theta[w_off[l]: w_off[l] + o * i].reshape(o, i)
        b = theta[b_off[l]: b_off[l] + o]
        out.append((W, b, W[:ro, :ri].copy(), b[:ro].copy()))
    return out, theta


def _model(n_members, stats, seed=1):
    mb = fos.fos_surrogate_model_bytes()
    model = torch.zeros(n_members * mb, dtype=torch.uint8, device="cuda")
    fos.check(fos.fos_surrogate_init(model, n_members, seed, stats), "init")
    return model


def _host_theta(seed):
    """He-uniform weights and small biases drawn on the host in the padded layout."""
    rng = np.random.default_rng(seed)
    P = fos.fos_surrogate_param_count()
    w_off, b_off = fos.fos_surrogate_param_offsets()
    theta = np.zeros(P, np.float32)
    shapes = [(256, 64), (256, 256), (256, 256), (256, 256), (64, 256)]
    params = []
    for l, ((o, i), (ro, ri)) in enumerate(zip(shapes, REAL)):
        lim = math.sqrt(6.0 / ri)
        W = np.zeros((o, i), np.float32)
        W[:ro, :ri] = rng.uniform(-lim, lim, (ro, ri))
        b = np.zeros(o, np.float32)
        b[:ro] = rng.uniform(-0.05, 0.05, ro)
        theta[w_off[l]: w_off[l] + o * i] = W.reshape(-1)
        theta[b_off[l]: b_off[l] + o] = b
        params.append((W[:ro, :ri].astype(np.float64), b[:ro].astype(np.float64)))
    return theta, params


def _loaded_model(stats, seed):
    """A one-member model holding host-drawn parameters (the oracle gets the same ones)."""
    theta, params = _host_theta(seed)
    mb = fos.fos_surrogate_model_bytes()
    model = torch.zeros(mb, dtype=torch.uint8, device="cuda")
    fos.check(fos.fos_surrogate_load(model, 0, torch.as_tensor(theta).cuda(), stats), "load")
    return model, theta, params


def _data(n, seed=0):
    rng = np.random.default_rng(seed)
    x = np.column_stack([rng.uniform(0.3, 2.5, n), rng.uniform(2.5, 3.1, n),
                         rng.uniform(-4, -0.3, n), rng.uniform(0.05, 1, n),
                         rng.uniform(0.01, 0.3, n), rng.uniform(1, 2.7, n),
                         rng.uniform(0, 0.9, n), rng.uniform(-1, 3, n), rng.uniform(-4, 2, n)])
    y = rng.dirichlet(np.ones(3), size=n)
    return x, y


def test_init_layout_and_padding():
    x, _ = _data(100)
    st, _, _ = _stats(x)
    model = _model(2, st)
    p0, th0 = _params(model, 0)
    p1, th1 = _params(model, 1)
    for l, (W, b, Wr, br) in enumerate(p0):
        ro, ri = REAL[l]
        lim = math.sqrt(6.0 / ri)
        assert np.all(np.abs(Wr) <= lim) and np.all(b == 0)
        assert np.all(W[ro:, :] == 0) and np.all(W[:, ri:] == 0)
        assert np.std(Wr) > 0.3 * lim
    assert not np.array_equal(th0, th1)


def test_load_stores_the_given_parameters():
    x, _ = _data(100)
    st, _, _ = _stats(x)
    model, theta, _ = _loaded_model(st, 12)
    _, th = _params(model)
    assert np.array_equal(th.astype(np.float32), theta)


def test_forward_matches_oracle():
    x, _ = _data(1000, 1)
    st, mean, std = _stats(x)
    model, _, ps = _loaded_model(st, 1)
    feats = torch.as_tensor(x, dtype=torch.float32).cuda().contiguous()
    rat = torch.zeros((1000, 3), dtype=torch.float32, device="cuda")
    fos.check(fos.fos_surrogate_predict(model, 1, feats, rat), "predict")
    got = rat.double().cpu().numpy()
    assert np.allclose(got.sum(axis=1), 1.0, atol=1e-5)
    xs = np.asarray(x, np.float32).astype(np.float64)
    ref = M.forward(ps, xs, mean.astype(np.float32), std.astype(np.float32))
    mirror = M.forward(ps, xs, mean.astype(np.float32), std.astype(np.float32),
                       round_fn=M.bf16_round)
    # The mirror rounds to bf16 where the kernel does; an activation that sits near a
    # bf16 rounding boundary can still round one ulp (2^-8 relative) apart, because the
    # kernel accumulates in FP32 on the tensor cores and the mirror in FP64.  Such rare
    # flips bound the worst row; the typical row agrees far closer.
    assert np.max(np.abs(got - mirror)) < 6e-3
    assert np.mean(np.abs(got - mirror)) < 5e-4
    assert np.max(np.abs(got - ref)) < 2e-2


def test_gradients_match_oracle():
    n, B = 2000, 512
    x, y = _data(n, 2)
    st, mean, std = _stats(x)
    model, _, ps = _loaded_model(st, 5)
    feats = torch.as_tensor(x, dtype=torch.float32).cuda().contiguous()
    targ = torch.as_tensor(y, dtype=torch.float32).cuda().contiguous()
    rows = np.random.default_rng(9).integers(0, n, size=B).astype(np.int32)
    P = fos.fos_surrogate_param_count()
    grad = torch.zeros(P, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    fos.check(fos.fos_surrogate_train_step(model, 0, feats, targ, B, 1, 0, 1e-3,
                                           batch_rows=torch.as_tensor(rows).cuda(),
                                           loss_out=loss, grad_out=grad), "grad")
    xs = np.asarray(x, np.float32).astype(np.float64)[rows]
    ys = np.asarray(y, np.float32).astype(np.float64)[rows]
    L, gref = M.loss_and_grads(ps, xs, ys, mean.astype(np.float32), std.astype(np.float32))
    assert abs(loss.item() - L) < 2e-3 * abs(L)
    g = grad.double().cpu().numpy()
    w_off, b_off = fos.fos_surrogate_param_offsets()
    shapes = [(256, 64), (256, 256), (256, 256), (256, 256), (64, 256)]
    for l, ((o, i), (ro, ri)) in enumerate(zip(shapes, REAL)):
        gw = g[w_off[l]: w_off[l] + o * i].reshape(o, i)
        gb = g[b_off[l]: b_off[l] + o]
        assert np.all(gw[ro:, :] == 0) and np.all(gw[:, ri:] == 0) and np.all(gb[ro:] == 0)
        for got, want in ((gw[:ro, :ri], gref[l][0]), (gb[:ro], gref[l][1])):
            rel = np.linalg.norm(got - want) / np.linalg.norm(want)
            cos = np.sum(got * want) / (np.linalg.norm(got) * np.linalg.norm(want))
            assert rel < 2e-2 and cos > 0.9995, (l, rel, cos)


def test_adam_update_arithmetic():
    """Adam's first step (Kingma & Ba): m_hat = g, v_hat = g^2, so every parameter moves
    by -lr g / (|g| + eps), i.e. by lr against the sign of its gradient.  The gradient's
    sign comes from the FP64 oracle where it is large enough to be certain."""
    n, B = 1024, 256
    x, y = _data(n, 3)
    st, mean, std = _stats(x)
    model, th0, ps = _loaded_model(st, 8)
    feats = torch.as_tensor(x, dtype=torch.float32).cuda().contiguous()
    targ = torch.as_tensor(y, dtype=torch.float32).cuda().contiguous()
    rows = torch.arange(B, dtype=torch.int32, device="cuda")
    fos.check(fos.fos_surrogate_train_step(model, 0, feats, targ, B, 1, 0, 1e-3, batch_rows=rows),
              "step")
    _, th1 = _params(model)
    xs = np.asarray(x, np.float32).astype(np.float64)[:B]
    ys = np.asarray(y, np.float32).astype(np.float64)[:B]
    _, gref = M.loss_and_grads(ps, xs, ys, mean.astype(np.float32), std.astype(np.float32))
    w_off, b_off = fos.fos_surrogate_param_offsets()
    shapes = [(256, 64), (256, 256), (256, 256), (256, 256), (64, 256)]
    d = th1 - th0.astype(np.float64)
    for l, ((o, i), (ro, ri)) in enumerate(zip(shapes, REAL)):
        dw = d[w_off[l]: w_off[l] + o * i].reshape(o, i)
        db = d[b_off[l]: b_off[l] + o]
        assert np.all(dw[ro:, :] == 0) and np.all(dw[:, ri:] == 0) and np.all(db[ro:] == 0)
        for got, g in ((dw[:ro, :ri], gref[l][0]), (db[:ro], gref[l][1])):
            sure = np.abs(g) > 0.3 * np.sqrt(np.mean(g * g))   # sign beyond bf16 noise
            assert np.all(np.abs(np.abs(got[sure]) - 1e-3) < 2e-6), l
            assert np.all(np.sign(got[sure]) == -np.sign(g[sure])), l


def test_training_reduces_loss_and_fits():
    n = 40000
    rng = np.random.default_rng(4)
    x, _ = _data(n, 4)
    st, mean, std = _stats(x)
    Wt = rng.normal(size=(3, 9)) * 0.8
    z = ((x - mean) / std) @ Wt.T
    y = np.exp(z) / np.exp(z).sum(axis=1, keepdims=True)
    model = _model(1, st, seed=2)
    feats = torch.as_tensor(x, dtype=torch.float32).cuda().contiguous()
    targ = torch.as_tensor(y, dtype=torch.float32).cuda().contiguous()
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    losses = []
    for step in range(400):
        fos.check(fos.fos_surrogate_train_step(model, 0, feats, targ, 1024, 11, step, 1e-3,
                                               loss_out=loss), "train")
        losses.append(loss.item())
    H = -np.mean(np.sum(y * np.log(y), axis=1))
    assert losses[-1] - H < 0.1 * (losses[0] - H)
    rat = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    fos.check(fos.fos_surrogate_predict(model, 1, feats, rat), "predict")
    assert np.mean(np.abs(rat.cpu().numpy() - y)) < 0.03


def test_ensemble_spread_and_fallback_flags():
    x, _ = _data(3000, 5)
    st, _, _ = _stats(x)
    model = _model(2, st, seed=3)
    mb = fos.fos_surrogate_model_bytes()
    model[mb:2 * mb].copy_(model[:mb])          # two identical members
    xx = x.copy()
    xx[10, 0] = 9.0                              # wavelength outside the training range
    xx[11, 5] = -1.0                             # thickness outside the training range
    feats = torch.as_tensor(xx, dtype=torch.float32).cuda().contiguous()
    rat = torch.zeros((3000, 3), dtype=torch.float32, device="cuda")
    spread = torch.full((3000,), -1.0, dtype=torch.float32, device="cuda")
    needs = torch.full((3000,), 7, dtype=torch.uint8, device="cuda")
    fos.check(fos.fos_surrogate_predict(model, 2, feats, rat, spread, needs, 0.01), "predict")
    assert torch.all(spread == 0)
    nz = set(torch.nonzero(needs).flatten().tolist())
    assert nz == {10, 11}
    one = torch.zeros_like(rat)
    fos.check(fos.fos_surrogate_predict(model, 1, feats, one), "predict1")
    assert torch.allclose(one, rat, atol=1e-6)
    # two different members: spread > 0 and flags follow the threshold
    model2 = _model(2, st, seed=4)
    fos.check(fos.fos_surrogate_predict(model2, 2, feats, rat, spread, needs, 0.0), "predict2")
    assert torch.all(spread > 0) and torch.all(needs == 1)


def test_features_and_fractions():
    rng = np.random.default_rng(6)
    nd, nw = 7, 5
    f64 = torch.float64
    wl = rng.uniform(0.3, 2.5, nw)
    arr = {k: rng.uniform(0.1, 3.0, nd * nw) for k in ("np_re", "np_im", "g", "mu_s", "mu_a")}
    arr["np_im"] = 10 ** rng.uniform(-4, -0.3, nd * nw)
    arr["g"] = rng.uniform(0, 0.9, nd * nw)
    des = {k: rng.uniform(0.05, 1.0, nd) for k in ("radius", "vol_frac")}
    thick = rng.uniform(10, 500, nd)
    t = lambda a: torch.as_tensor(a, dtype=f64).cuda()
    feats = torch.zeros((nd * nw, 9), dtype=torch.float32, device="cuda")
    fos.check(fos.fos_surrogate_features(t(wl), t(arr["np_re"]), t(arr["np_im"]), t(des["radius"]),
                                         t(des["vol_frac"]), t(thick), t(arr["g"]), t(arr["mu_s"]),
                                         t(arr["mu_a"]), feats), "features")
    d = np.repeat(np.arange(nd), nw)
    w = np.tile(np.arange(nw), nd)
    want = np.column_stack([wl[w], arr["np_re"], np.log10(arr["np_im"]), des["radius"][d],
                            des["vol_frac"][d], np.log10(thick[d]), arr["g"],
                            np.log10(arr["mu_s"] * thick[d] + 1e-6),
                            np.log10(arr["mu_a"] * thick[d] + 1e-6)]).astype(np.float32)
    assert np.allclose(feats.cpu().numpy(), want, rtol=1e-6, atol=1e-6)
    counts = torch.as_tensor([[3, 5, 2, 0, 77, 1], [0, 0, 0, 0, 0, 0]], dtype=torch.int64).cuda()
    fr = torch.zeros((2, 3), dtype=torch.float32, device="cuda")
    fos.check(fos.fos_counts_to_fractions(counts, fr), "fractions")
    torch.cuda.synchronize()
    assert np.allclose(fr.cpu().numpy(), [[0.3, 0.5, 0.2], [0, 0, 0]])
    # scatter into given rows
    big = torch.full((5, 3), -1.0, dtype=torch.float32, device="cuda")
    fos.check(fos.fos_counts_to_fractions(counts, big, torch.tensor([4, 1], dtype=torch.int32,
                                                                    device="cuda")), "scatter")
    torch.cuda.synchronize()
    b = big.cpu().numpy()
    assert np.allclose(b[4], [0.3, 0.5, 0.2]) and np.allclose(b[1], 0) and np.all(b[0] == -1)


def test_mask_to_rows():
    rng = np.random.default_rng(8)
    for n in (0, 1, 1023, 1024, 1025, 300000):
        m = (rng.random(n) < 0.01).astype(np.uint8)
        if n:
            m[-1] = 1
        mask = torch.as_tensor(m, device="cuda")
        rows = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        fos.check(fos.fos_mask_to_rows(mask, rows, cnt), "mask_to_rows")
        k = int(cnt.item())
        got = np.sort(rows[:k].cpu().numpy())
        assert np.array_equal(got, np.nonzero(m)[0])


def test_in_kernel_wait_gives_up_and_reports_timeout():
    """A pipeline stage that never fills (test flag): the bounded mbarrier wait runs
    out, the kernel drains its other copies, frees its tensor memory and returns; the
    host reads FOS_ERR_TIMEOUT and the context stays usable."""
    rng = np.random.default_rng(1)
    A = _bf16(rng, (256, 512))
    B = _bf16(rng, (256, 512))
    C = torch.zeros((1, 256, 256), dtype=torch.float32, device="cuda")
    st = fos.fos_gemm_bf16(A, B, C, 1, flags=fos.FOS_TEST_STALL)
    assert st == fos.FOS_ERR_TIMEOUT
    st = fos.fos_gemm_bf16(A, B, C, 1)
    assert st == fos.FOS_OK
    ref = A.float().double().cpu().numpy() @ B.float().double().cpu().numpy().T
    assert np.allclose(C[0].double().cpu().numpy(), ref, rtol=1e-4, atol=1e-3)


def test_fused_ensemble_matches_oracle_on_a_ragged_batch():
    """Three members with host-drawn parameters over 50,001 rows (390 full tiles and a
    ragged one, more tiles than CTAs): mean, spread and fallback flags on sampled rows
    against the bf16-mirrored oracle forward of each member."""
    n = 50001
    x, _ = _data(n, 6)
    st, mean, std = _stats(x)
    mb = fos.fos_surrogate_model_bytes()
    model = torch.zeros(3 * mb, dtype=torch.uint8, device="cuda")
    params = []
    for k in range(3):
        theta, ps = _host_theta(100 + k)
        fos.check(fos.fos_surrogate_load(model[k * mb:(k + 1) * mb], 0,
                                         torch.as_tensor(theta).cuda(), st), "load")
        params.append(ps)
    xx = x.copy()
    xx[17, 2] = 5.0          # outside the training range of feature 2
    feats = torch.as_tensor(xx, dtype=torch.float32).cuda().contiguous()
    rat = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    spread = torch.zeros(n, dtype=torch.float32, device="cuda")
    needs = torch.zeros(n, dtype=torch.uint8, device="cuda")
    thr = 0.05
    fos.check(fos.fos_surrogate_predict(model, 3, feats, rat, spread, needs, thr), "predict")
    rng = np.random.default_rng(3)
    rows = np.unique(np.concatenate([rng.integers(0, n, 1500), [0, 17, n - 1, n - 2]]))
    xs = np.asarray(xx, np.float32).astype(np.float64)[rows]
    outs = np.stack([M.forward(ps, xs, mean.astype(np.float32), std.astype(np.float32),
                               round_fn=M.bf16_round) for ps in params])
    got_rat = rat.double().cpu().numpy()[rows]
    got_spr = spread.double().cpu().numpy()[rows]
    assert np.max(np.abs(got_rat - outs.mean(axis=0))) < 6e-3
    want_spr = (outs.max(axis=0) - outs.min(axis=0)).max(axis=1)
    assert np.max(np.abs(got_spr - want_spr)) < 1.2e-2
    got_need = needs.cpu().numpy()[rows]
    clear = np.abs(want_spr - thr) > 1.2e-2          # away from the threshold
    lo, hi = st[32:41], st[48:57]
    out_rng = np.any((xs < lo) | (xs > hi), axis=1)
    want_need = (want_spr > thr) | out_rng
    assert np.array_equal(got_need[clear], want_need[clear])
    assert got_need[list(rows).index(17)] == 1


def test_fused_ensemble_small_and_empty_batches():
    """Batches of 0, 1, 127, 128 and 129 rows (fewer tiles than CTAs, one full tile, a
    full tile plus one row): an empty call succeeds and writes nothing; every row of the
    others matches the bf16-mirrored oracle forward, and a row's result does not depend on
    the batch it comes in (bit for bit)."""
    x, _ = _data(129, 11)
    st, mean, std = _stats(x)
    mb = fos.fos_surrogate_model_bytes()
    model = torch.zeros(2 * mb, dtype=torch.uint8, device="cuda")
    params = []
    for k in range(2):
        theta, ps = _host_theta(200 + k)
        fos.check(fos.fos_surrogate_load(model[k * mb:(k + 1) * mb], 0,
                                         torch.as_tensor(theta).cuda(), st), "load")
        params.append(ps)
    feats = torch.as_tensor(x, dtype=torch.float32).cuda().contiguous()
    rat0 = torch.full((1, 3), -1.0, dtype=torch.float32, device="cuda")
    assert fos.fos_surrogate_predict(model, 2, feats[:0], rat0[:0]) == fos.FOS_OK
    assert torch.all(rat0 == -1.0)
    xs = np.asarray(x, np.float32).astype(np.float64)
    outs = np.stack([M.forward(ps, xs, mean.astype(np.float32), std.astype(np.float32),
                               round_fn=M.bf16_round) for ps in params])
    want = outs.mean(axis=0)
    results = {}
    for n in (1, 127, 128, 129):
        rat = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
        spread = torch.zeros(n, dtype=torch.float32, device="cuda")
        fos.check(fos.fos_surrogate_predict(model, 2, feats[:n].contiguous(), rat, spread),
                  f"predict {n}")
        got = rat.double().cpu().numpy()
        assert np.max(np.abs(got - want[:n])) < 6e-3, n
        assert np.allclose(got.sum(axis=1), 1.0, atol=1e-5)
        results[n] = (rat.cpu(), spread.cpu())
    for n in (1, 127, 128):
        assert torch.equal(results[n][0], results[129][0][:n])
        assert torch.equal(results[n][1], results[129][1][:n])


def test_fused_inference_wait_gives_up_and_reports_timeout():
    """The fused inference kernel with its first weight copy withheld (test flag): the
    bounded waits run out, the kernel drains and returns FOS_ERR_TIMEOUT, and the next
    call succeeds with the same results as before."""
    x, _ = _data(3000, 7)
    st, _, _ = _stats(x)
    model, _, _ = _loaded_model(st, 21)
    feats = torch.as_tensor(x, dtype=torch.float32).cuda().contiguous()
    r1 = torch.zeros((3000, 3), dtype=torch.float32, device="cuda")
    fos.check(fos.fos_surrogate_predict(model, 1, feats, r1), "predict")
    r2 = torch.zeros((3000, 3), dtype=torch.float32, device="cuda")
    assert fos.fos_surrogate_predict(model, 1, feats, r2, flags=fos.FOS_TEST_STALL) == \
        fos.FOS_ERR_TIMEOUT
    fos.check(fos.fos_surrogate_predict(model, 1, feats, r2), "predict again")
    assert torch.equal(r1, r2)


def test_fused_ensemble_with_more_members_than_parameter_slots():
    """Six members: more than the kernel's four shared-memory parameter slots, so the
    biases and statistics are staged member by member.  Mean and spread against the
    bf16-mirrored oracle forward of each member."""
    n = 3000
    x, _ = _data(n, 9)
    st, mean, std = _stats(x)
    mb = fos.fos_surrogate_model_bytes()
    model = torch.zeros(6 * mb, dtype=torch.uint8, device="cuda")
    params = []
    for k in range(6):
        theta, ps = _host_theta(200 + k)
        fos.check(fos.fos_surrogate_load(model[k * mb:(k + 1) * mb], 0,
                                         torch.as_tensor(theta).cuda(), st), "load")
        params.append(ps)
    feats = torch.as_tensor(x, dtype=torch.float32).cuda().contiguous()
    rat = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    spread = torch.zeros(n, dtype=torch.float32, device="cuda")
    fos.check(fos.fos_surrogate_predict(model, 6, feats, rat, spread), "predict")
    xs = np.asarray(x, np.float32).astype(np.float64)
    outs = np.stack([M.forward(ps, xs, mean.astype(np.float32), std.astype(np.float32),
                               round_fn=M.bf16_round) for ps in params])
    assert np.max(np.abs(rat.double().cpu().numpy() - outs.mean(axis=0))) < 6e-3
    want_spr = (outs.max(axis=0) - outs.min(axis=0)).max(axis=1)
    assert np.max(np.abs(spread.double().cpu().numpy() - want_spr)) < 1.2e-2
