"""Pins of the MLP oracle (CPU): the hand-derived backward against central finite
differences of the loss, and the BF16 rounding helper against torch's bfloat16."""
import numpy as np
import pytest
import torch

from oracle import mlp


def _data(n=17, seed=3):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(n, 9)) * np.array([3, 3, 3, 4, 4, 4, 2, 2, 2]) + 5
    t = rng.normal(size=n)
    mean, std = x.mean(0), x.std(0) + 1e-3
    return x, t, mean, std


def test_layout_size():
    assert mlp.NPARAMS == 64 * 9 + 64 + 64 * 64 + 64 + 64 * 64 + 64 + 64 + 1


def test_backward_matches_finite_differences():
    x, t, mean, std = _data()
    theta = mlp.init(1)
    theta[576:640] = 0.1      # nonzero biases so every parameter block is exercised
    theta[-1] = 0.3
    g = mlp.grad(theta, x, t, mean, std)
    rng = np.random.default_rng(0)
    idx = np.concatenate([rng.choice(mlp.NPARAMS, 60, replace=False), [0, 575, 640, 9024]])
    h = 1e-6
    for k in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (mlp.loss(tp, x, t, mean, std) - mlp.loss(tm, x, t, mean, std)) / (2 * h)
        assert fd == pytest.approx(g[k], rel=1e-5, abs=1e-9), k


def test_bf16_round_matches_torch():
    v = np.random.default_rng(2).normal(size=1000) * 10 ** np.random.default_rng(3).uniform(-5, 5, 1000)
    ref = torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(v), ref)
