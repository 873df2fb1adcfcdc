"""Pins of the FP64 surrogate-MLP oracle (oracle/mlp.py)."""
import math

import numpy as np
import pytest

from oracle import mlp as M


def _small(seed=0):
    rng = np.random.default_rng(seed)
    params = M.init_params(rng, M.layer_shapes(9, 8, 2, 3))
    params = [(W, rng.normal(0, 0.1, size=b.shape)) for W, b in params]
    x = rng.normal(size=(13, 9))
    y = rng.dirichlet(np.ones(3), size=13)
    return params, x, y


def test_gradients_match_central_differences():
    params, x, y = _small()
    L, grads = M.loss_and_grads(params, x, y)
    h = 1e-6
    for li, (W, b) in enumerate(params):
        for arr, g in ((W, grads[li][0]), (b, grads[li][1])):
            for idx in list(np.ndindex(arr.shape))[:: max(1, arr.size // 12)]:
                old = arr[idx]
                arr[idx] = old + h
                lp = M.loss(params, x, y)
                arr[idx] = old - h
                lm = M.loss(params, x, y)
                arr[idx] = old
                fd = (lp - lm) / (2 * h)
                assert abs(fd - g[idx]) <= 1e-7 + 1e-6 * abs(fd)


def test_gradients_match_torch_autograd_full_size():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    params = M.init_params(rng)
    params = [(W, rng.normal(0, 0.05, size=b.shape)) for W, b in params]
    x = rng.normal(size=(32, 9))
    y = rng.dirichlet(np.ones(3), size=32)
    mean, std = rng.normal(size=9), rng.uniform(0.5, 2, size=9)
    L, grads = M.loss_and_grads(params, x, y, mean, std)
    tp = [(torch.tensor(W, requires_grad=True), torch.tensor(b, requires_grad=True))
          for W, b in params]
    h = (torch.tensor(x) - torch.tensor(mean)) / torch.tensor(std)
    for i, (W, b) in enumerate(tp):
        z = h @ W.T + b
        h = torch.nn.functional.gelu(z, approximate="tanh") if i < len(tp) - 1 else z
    lt = -(torch.tensor(y) * torch.log_softmax(h, dim=1)).sum(dim=1).mean()
    lt.backward()
    assert abs(lt.item() - L) < 1e-12
    for (W, b), (gW, gb) in zip(tp, grads):
        assert np.allclose(W.grad.numpy(), gW, rtol=1e-10, atol=1e-14)
        assert np.allclose(b.grad.numpy(), gb, rtol=1e-10, atol=1e-14)


def test_softmax_and_cross_entropy_identities():
    params, x, y = _small(5)
    p = M.forward(params, x)
    assert np.allclose(p.sum(axis=1), 1.0, atol=1e-15)
    assert np.all(p > 0)
    # gradient wrt logits is (p - y)/B: the last-layer bias gradient equals its mean
    L, grads = M.loss_and_grads(params, x, y)
    assert np.allclose(grads[-1][1], (p - y).mean(axis=0), atol=1e-15)
    # cross-entropy >= entropy of the labels, with equality iff p = y
    H = -np.mean(np.sum(y * np.log(y), axis=1))
    assert L >= H


def test_gelu_special_values():
    z = np.array([-3.0, -1.0, 0.0, 1.0, 3.0])
    g = M.gelu(z)
    assert g[2] == 0.0
    assert abs(g[3] - g[1] - 1.0) < 1e-15              # gelu(x) - gelu(-x) = x
    # the tanh form stays within 2e-3 of the exact x Phi(x)
    from scipy.special import erf
    exact = 0.5 * z * (1 + erf(z / math.sqrt(2)))
    assert np.max(np.abs(g - exact)) < 2e-3
    torch = pytest.importorskip("torch")
    tt = torch.nn.functional.gelu(torch.tensor(z), approximate="tanh").numpy()
    assert np.allclose(g, tt, rtol=1e-14, atol=1e-15)
    # derivative by finite differences
    h = 1e-6
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    assert np.allclose(fd, M.gelu_grad(z), atol=1e-8)


def test_adam_first_step_is_signed_lr():
    params, x, y = _small(7)
    _, grads = M.loss_and_grads(params, x, y)
    zeros = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    new, m, v = M.adam_step(params, grads, zeros, zeros, 1, lr=1e-3, eps=0.0)
    for (W, b), (W1, b1), (gW, gb) in zip(params, new, grads):
        nz = gW != 0
        assert np.allclose((W1 - W)[nz], -1e-3 * np.sign(gW[nz]), rtol=1e-12)


def test_bf16_rounding():
    a = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9, -2.5, 1e-3])
    r = M.bf16_round(a)
    assert r[0] == 1.0 and r[1] == 1.0     # halfway: ties to the even mantissa
    assert r[2] == 1.0                      # below half ulp
    assert r[3] == 1.0 + 2 ** -7            # above half ulp
    assert r[4] == -2.5
    assert abs(r[5] - 1e-3) <= 2 ** -9 * 1e-3
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(0).normal(size=1000)
    t = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(t, M.bf16_round(x))
