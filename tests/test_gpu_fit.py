"""Graph-captured training (fos_surrogate_fit): every member's Adam steps with the step
count, learning rate and bias corrections on the device, one graph launch per ensemble
step.  It must do what the per-step entry point does: same batches, same updates (the
learning rate is computed on the device instead of the host, so parameters agree to
float rounding rather than bit for bit), and the step counts advance."""
import math

import numpy as np
import pytest

from paper_2409_00165_gb300 import fos
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
    return (torch.as_tensor(x, dtype=torch.float32).cuda().contiguous(),
            torch.as_tensor(y, dtype=torch.float32).cuda().contiguous())


def _theta(sur, k):
    P = fos.fos_surrogate_param_count()
    mb = fos.fos_surrogate_model_bytes()
    return sur.model[k * mb: k * mb + 4 * P].view(torch.float32)


def _per_step(sur, f, y, steps, batch, lr, lr_min, total, first=0):
    for t in range(first, first + steps):
        cur = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * min(t, total) / total))
        for k in range(sur.n_members):
            fos.check(fos.fos_surrogate_train_step(sur.model, k, f, y, batch, sur.seed, t, cur),
                      "train_step")
    torch.cuda.synchronize()


def test_fit_graph_matches_per_step_training():
    """Constant learning rate: every value of the step is the same on both paths (the
    bias corrections 1 - 0.9^t, 1 - 0.999^t rounded to float), so the models agree bit for
    bit; 5 members exercise slots 0-3 and a second member in slot 0."""
    f, y = _data(30000, 5)
    stats = S.Surrogate.stats_of(f)
    a = S.Surrogate(5, stats, seed=11)
    b = S.Surrogate(5, stats, seed=11)
    assert torch.equal(a.model, b.model)
    steps, lr = 30, 1e-3
    ha = a.fit(f, y, steps=steps, batch=2048, lr=lr, lr_min=lr, log_every=10)
    _per_step(b, f, y, steps, 2048, lr, lr, steps)
    for k in range(5):
        assert torch.equal(_theta(a, k), _theta(b, k)), k
    assert a.steps_done == [steps] * 5
    assert [h[-1][0] for h in ha.values()] == [steps - 1] * 5
    assert all(0 < h[-1][1] < 5 for h in ha.values())


def test_fit_graph_cosine_schedule_and_step_counts():
    """Cosine schedule (the learning rate computed on the device in place of the host:
    float roundings may differ, so the models agree closely rather than bit for bit), and
    the device step counts that both paths leave behind: one more graph step on each
    model continues alike."""
    f, y = _data(30000, 7)
    stats = S.Surrogate.stats_of(f)
    a = S.Surrogate(2, stats, seed=12)
    b = S.Surrogate(2, stats, seed=12)
    steps, lr, lr_min, total = 20, 2e-3, 2e-5, 21
    a.fit(f, y, steps=steps, batch=2048, lr=lr, lr_min=lr_min, schedule_steps=total)
    _per_step(b, f, y, steps, 2048, lr, lr_min, total)
    for sur in (a, b):
        sur.fit(f, y, steps=1, batch=2048, lr=lr, lr_min=lr_min, schedule_steps=total)
    for k in range(2):
        ta, tb = _theta(a, k), _theta(b, k)
        assert torch.max(torch.abs(ta - tb)).item() < 1e-3 * torch.max(torch.abs(tb)).item()


def test_fit_rejects_bad_arguments():
    f, y = _data(1000, 6)
    sur = S.Surrogate(1, S.Surrogate.stats_of(f), seed=1)
    bad = dict(batch=1000)
    assert fos.fos_surrogate_fit(sur.model, 1, f, y, 1000, 1, 1, 1e-3, 0.0, 0, 10) == \
        fos.FOS_ERR_INVALID_ARG
    assert fos.fos_surrogate_fit(sur.model, 1, f, y, 1024, 1, 1, 1e-3, 0.0, 0, 0) == \
        fos.FOS_ERR_INVALID_ARG
    assert fos.fos_surrogate_fit(sur.model, 0, f, y, 1024, 1, 1, 1e-3, 0.0, 0, 10) == \
        fos.FOS_ERR_INVALID_ARG
    del bad
