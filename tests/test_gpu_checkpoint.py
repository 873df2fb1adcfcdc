"""Checkpoint and resume of surrogate training: a run split by save/restore ends in the
same model, byte for byte, as the uninterrupted run (training is deterministic: hashed
batch rows, fixed-order reductions)."""
import numpy as np
import pytest

from paper_2409_00165_gb300 import surrogate as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _data(n, seed):
    rng = np.random.default_rng(seed)
    x = np.column_stack([rng.uniform(0.3, 2.5, n), rng.uniform(2.5, 3.1, n),
                         rng.uniform(-4, -0.3, n), rng.uniform(0.05, 1, n),
                         rng.uniform(0.01, 0.3, n), rng.uniform(1, 2.7, n),
                         rng.uniform(0, 0.9, n), rng.uniform(-1, 3, n), rng.uniform(-4, 2, n)])
    y = rng.dirichlet(np.ones(3), size=n)
    f = torch.as_tensor(x, dtype=torch.float32).cuda().contiguous()
    t = torch.as_tensor(y, dtype=torch.float32).cuda().contiguous()
    return f, t


def test_resume_matches_uninterrupted_training(tmp_path):
    f, y = _data(20000, 1)
    stats = S.Surrogate.stats_of(f)
    whole = S.Surrogate(2, stats, seed=3)
    whole.fit(f, y, steps=40, batch=1024, lr=2e-3, schedule_steps=40)
    first = S.Surrogate(2, stats, seed=3)
    first.fit(f, y, steps=25, batch=1024, lr=2e-3, schedule_steps=40)
    path = str(tmp_path / "ckpt.npz")
    first.save(path)
    resumed = S.Surrogate.restore(path)
    assert resumed.steps_done == [25, 25]
    resumed.fit(f, y, steps=15, batch=1024, lr=2e-3, schedule_steps=40)
    assert torch.equal(resumed.model, whole.model)
    # and the restored model predicts like the original
    a = whole.predict(f[:5000])[0]
    b = resumed.predict(f[:5000])[0]
    assert torch.equal(a, b)
