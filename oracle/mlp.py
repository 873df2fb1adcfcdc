"""FP64 NumPy reference of the surrogate MLP (test infrastructure only).

The paper replaces the Monte Carlo walk by a network trained on Monte Carlo spectra
(section "Photon transport", inputs in the ranges of Table 1).  The surrogate here maps 9
features to (R, A, T):

    x (9) -> standardise -> [Linear 256, GELU] x 4 -> Linear 3 -> softmax

GELU is its tanh form x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))) (Hendrycks &
Gimpel 2016), evaluated here with exact tanh.  The loss is the
softmax cross-entropy against the Monte Carlo fractions (soft labels), averaged over the
batch.  Adam (Kingma & Ba 2015) updates FP32 master weights.  Everything here is plain
float64 NumPy, written from those definitions, with no blocking or fusion.

Parity status: pinned (tests/test_oracle_mlp.py: central finite differences of the loss,
torch float64 autograd on the same network, softmax/cross-entropy identities, Adam's
first step equal to -lr * sign(g)).
"""
from __future__ import annotations

import math

import numpy as np

N_IN = 9
HIDDEN = 256
N_HIDDEN_LAYERS = 4
N_OUT = 3


def layer_shapes(n_in=N_IN, hidden=HIDDEN, n_hidden=N_HIDDEN_LAYERS, n_out=N_OUT):
    dims = [n_in] + [hidden] * n_hidden + [n_out]
    return [(dims[i + 1], dims[i]) for i in range(len(dims) - 1)]   # (out, in)


GELU_C = math.sqrt(2.0 / math.pi)
GELU_A = 0.044715


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(GELU_C * (z + GELU_A * z ** 3)))


def gelu_grad(z):
    t = np.tanh(GELU_C * (z + GELU_A * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * GELU_C * (1.0 + 3.0 * GELU_A * z * z)


def softmax(z):
    z = z - np.max(z, axis=1, keepdims=True)
    e = np.exp(z)
    return e / np.sum(e, axis=1, keepdims=True)


def standardise(x, mean, std):
    return (np.asarray(x, np.float64) - mean) / std


def forward(params, x, mean=None, std=None, keep=False, round_fn=None):
    """params: list of (W [out,in], b [out]).  Returns probabilities [B, 3]
    (and the pre-activations / activations when keep=True).

    round_fn, if given, is applied to the layer inputs and weights before each product
    and to the hidden activations after GELU (a mirror of reduced-precision storage)."""
    r = round_fn if round_fn is not None else (lambda a: a)
    h = np.asarray(x, np.float64)
    if mean is not None:
        h = standardise(h, mean, std)
    hs, zs = [h], []
    for i, (W, b) in enumerate(params):
        z = r(h) @ r(W).T + b
        zs.append(z)
        if i < len(params) - 1:
            h = gelu(z)
            hs.append(h)
    p = softmax(zs[-1])
    return (p, zs, hs) if keep else p


def loss(params, x, y, mean=None, std=None):
    p = forward(params, x, mean, std)
    return -np.mean(np.sum(np.asarray(y) * np.log(p), axis=1))


def loss_and_grads(params, x, y, mean=None, std=None):
    """Cross-entropy with soft labels y (rows sum to 1) and its gradients."""
    y = np.asarray(y, np.float64)
    B = y.shape[0]
    p, zs, hs = forward(params, x, mean, std, keep=True)
    L = -np.mean(np.sum(y * np.log(p), axis=1))
    dz = (p - y) / B                      # d loss / d logits
    grads = [None] * len(params)
    for i in range(len(params) - 1, -1, -1):
        W, _ = params[i]
        grads[i] = (dz.T @ hs[i], dz.sum(axis=0))
        if i > 0:
            dh = dz @ W
            dz = dh * gelu_grad(zs[i - 1])
    return L, grads


def init_params(rng, shapes=None):
    """He-uniform weights, zero biases (any reasonable initialisation; the tests do not
    depend on it)."""
    shapes = shapes or layer_shapes()
    out = []
    for (o, i) in shapes:
        lim = math.sqrt(6.0 / i)
        out.append((rng.uniform(-lim, lim, size=(o, i)), np.zeros(o)))
    return out


def adam_step(params, grads, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (bias-corrected); t counts from 1.  Returns new params, m, v."""
    new_p, new_m, new_v = [], [], []
    for (W, b), (gW, gb), (mW, mb), (vW, vb) in zip(params, grads, m, v):
        outs = []
        for x, g, mm, vv in ((W, gW, mW, vW), (b, gb, mb, vb)):
            mm = b1 * mm + (1 - b1) * g
            vv = b2 * vv + (1 - b2) * g * g
            mh = mm / (1 - b1 ** t)
            vh = vv / (1 - b2 ** t)
            outs.append((x - lr * mh / (np.sqrt(vh) + eps), mm, vv))
        new_p.append((outs[0][0], outs[1][0]))
        new_m.append((outs[0][1], outs[1][1]))
        new_v.append((outs[0][2], outs[1][2]))
    return new_p, new_m, new_v


def bf16_round(a):
    """Round-to-nearest-even to bfloat16, returned as float64."""
    a32 = np.asarray(a, np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
