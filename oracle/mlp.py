"""Plain NumPy (FP64) forward and backward of the trimer-screen MLP.  TEST
INFRASTRUCTURE ONLY.

Network and parameter layout as in include/rimp2_mlp.h: 9 -> 64 -> 64 -> 64 -> 1, SiLU
after the hidden layers, parameters [W1 (64x9), b1, W2 (64x64), b2, W3, b3, W4 (1x64),
b4] flattened in that order.  Inputs are standardised with (x - mean) / std.  Loss is
the mean squared error over the batch.  The backward pass is derived by hand (chain
rule through SiLU(z) = z sigmoid(z), whose derivative is s (1 + z (1 - s))); its
finite-difference pin lives in tests/test_mlp_oracle.py.
"""
from __future__ import annotations

import numpy as np

SHAPES = [(64, 9), (64,), (64, 64), (64,), (64, 64), (64,), (1, 64), (1,)]
NPARAMS = int(sum(np.prod(s) for s in SHAPES))


def unpack(theta):
    out, off = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(np.asarray(theta[off:off + n], dtype=np.float64).reshape(s))
        off += n
    return out


def bf16_round(x):
    """Round-to-nearest-even to bfloat16, returned as float64."""
    a = np.asarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _sig(z):
    return 1.0 / (1.0 + np.exp(-z))


def forward(theta, x, mean, std):
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(theta)
    xs = (np.asarray(x, dtype=np.float64) - mean) / std
    z1 = xs @ W1.T + b1
    h1 = z1 * _sig(z1)
    z2 = h1 @ W2.T + b2
    h2 = z2 * _sig(z2)
    z3 = h2 @ W3.T + b3
    h3 = z3 * _sig(z3)
    y = (h3 @ W4.T + b4)[:, 0]
    return y, (xs, z1, h1, z2, h2, z3, h3)


def loss(theta, x, t, mean, std):
    y, _ = forward(theta, x, mean, std)
    return float(np.mean((y - t) ** 2))


def grad(theta, x, t, mean, std):
    """Gradient of the mean squared error with respect to theta (float64)."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(theta)
    y, (xs, z1, h1, z2, h2, z3, h3) = forward(theta, x, mean, std)
    n = len(t)
    dy = 2.0 * (y - t) / n                       # [n]

    def dsilu(z):
        s = _sig(z)
        return s * (1.0 + z * (1.0 - s))

    gW4 = dy[None, :] @ h3                       # [1, 64]
    gb4 = np.array([dy.sum()])
    dz3 = (dy[:, None] * W4) * dsilu(z3)         # [n, 64]
    gW3 = dz3.T @ h2
    gb3 = dz3.sum(0)
    dz2 = (dz3 @ W3) * dsilu(z2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * dsilu(z1)
    gW1 = dz1.T @ xs
    gb1 = dz1.sum(0)
    return np.concatenate([g.ravel() for g in (gW1, gb1, gW2, gb2, gW3, gb3, gW4, gb4)])


def init(seed=0):
    """He-style initial parameters (float64), the same draw on both sides of a test."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in SHAPES:
        if len(s) == 2:
            parts.append(rng.normal(0.0, np.sqrt(2.0 / s[1]), size=s).ravel())
        else:
            parts.append(np.zeros(s))
    return np.concatenate(parts)
