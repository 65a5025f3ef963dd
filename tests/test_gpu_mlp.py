"""GPU tests of the learned-screen kernels against the NumPy oracle (oracle/mlp.py).

The GPU forward uses BF16-rounded weights with FP32 accumulation; the oracle evaluates
the same network in FP64 with the same BF16-rounded weights, so gradients agree to FP32
accumulation error (tolerance 2e-4 relative in norm, 1e-3 per element above 1e-6).
"""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from paper_2410_21888_gb300 import rimp2, synth

pytestmark = pytest.mark.gpu


def _problem(n=300, seed=0):
    rng = np.random.default_rng(seed)
    x = np.abs(rng.normal(size=(n, 9))) * np.array([8, 10, 12, 4, 5, 6, 2, 2, 2]) + \
        np.array([2, 3, 4, 8, 9, 10, -12, -10, -8])
    y = -3 - 0.4 * x[:, 0] + 0.2 * x[:, 6] + 0.05 * rng.normal(size=n)
    theta = omlp.init(seed)
    theta[576:640] = 0.05 * rng.normal(size=64)
    theta[-1] = -2.0
    mean, std = x.mean(0), x.std(0) + 1e-3
    return x.astype(np.float32), y.astype(np.float32), theta.astype(np.float32), mean, std


def _dev(a, dt=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def test_grad_and_loss_match_oracle():
    x, y, theta, mean, std = _problem()
    idx = np.arange(0, 300, 2).astype(np.int32)
    g, loss = rimp2.mlp_grad(_dev(theta), _dev(x), _dev(y), _dev(idx, torch.int32), len(idx),
                             _dev(mean), _dev(std))
    tb = omlp.bf16_round(theta)
    xf, yf = x[idx].astype(np.float64), y[idx].astype(np.float64)
    mf, sf = mean.astype(np.float32).astype(np.float64), std.astype(np.float32).astype(np.float64)
    ref = omlp.grad(tb, xf, yf, mf, sf)
    got = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) <= 2e-4 * np.linalg.norm(ref)
    big = np.abs(ref) > 1e-6
    assert np.all(np.abs(got[big] - ref[big]) <= 1e-3 * np.abs(ref[big]) + 1e-6)
    assert float(loss.item()) == pytest.approx(omlp.loss(tb, xf, yf, mf, sf), rel=1e-4)


def test_predict_matches_oracle_forward():
    x, y, theta, mean, std = _problem(n=1000, seed=1)
    p = rimp2.mlp_predict(_dev(theta), _dev(x), _dev(mean), _dev(std)).cpu().numpy()
    ref, _ = omlp.forward(omlp.bf16_round(theta), x.astype(np.float64),
                          mean.astype(np.float32).astype(np.float64),
                          std.astype(np.float32).astype(np.float64))
    assert np.max(np.abs(p - ref)) <= 1e-4 * (1 + np.max(np.abs(ref)))


def test_adam_step_matches_formula():
    rng = np.random.default_rng(5)
    w = rng.normal(size=rimp2.MLP_PARAMS).astype(np.float32)
    g = rng.normal(size=rimp2.MLP_PARAMS).astype(np.float32)
    m = rng.normal(size=rimp2.MLP_PARAMS).astype(np.float32) * 0.1
    v = np.abs(rng.normal(size=rimp2.MLP_PARAMS)).astype(np.float32) * 0.1
    W, M, Vv = _dev(w), _dev(m), _dev(v)
    rimp2.mlp_adam(W, _dev(g), M, Vv, 3, 1e-3)
    m2 = 0.9 * m + 0.1 * g
    v2 = 0.999 * v + 0.001 * g * g
    w2 = w - 1e-3 * (m2 / (1 - 0.9 ** 3)) / (np.sqrt(v2 / (1 - 0.999 ** 3)) + 1e-8)
    assert np.allclose(W.cpu().numpy(), w2, rtol=1e-5, atol=1e-6)
    assert np.allclose(M.cpu().numpy(), m2, rtol=1e-6, atol=1e-7)


def test_training_reduces_loss():
    from paper_2410_21888_gb300.screen import TrimerScreen
    x, y, _, _, _ = _problem(n=2000, seed=2)
    sc = TrimerScreen(seed=0)
    fx, fy = _dev(x), _dev(y)
    sc.set_normalization(fx)
    l0 = sc.loss(fx, fy)
    hist = sc.fit(fx, fy, epochs=40, batch=256, lr=3e-3)
    assert hist[-1] < 0.05 * l0 and sc.loss(fx, fy) < 0.05 * l0


def test_features_and_corrections():
    s = synth.MonomerSystem(n_monomers=9, box=12.0, seed=3)
    tri = np.array([[0, 1, 2], [3, 5, 8], [1, 4, 7]], dtype=np.int32)
    rng = np.random.default_rng(0)
    table = rng.normal(size=(9, 9)) * 1e-4
    table = table + table.T
    f = rimp2.screen_features(_dev(s.centroids, torch.float64), _dev(s.nocc, torch.int32),
                              _dev(tri, torch.int32), _dev(table, torch.float64)).cpu().numpy()
    for k, (a, b, c) in enumerate(tri):
        d = sorted(np.linalg.norm(s.centroids[p] - s.centroids[q]) for p, q in ((a, b), (a, c), (b, c)))
        n = sorted(float(s.nocc[p]) for p in (a, b, c))
        e = sorted(np.log10(abs(table[p, q]) + 1e-16) for p, q in ((a, b), (a, c), (b, c)))
        assert np.allclose(f[k], np.array(d + n + e), rtol=1e-6, atol=1e-5)
    E = _dev(rng.normal(size=20), torch.float64)
    terms = torch.tensor([[3, 1, 2], [7, 0, 5]], dtype=torch.int32)
    out, lg = rimp2.mbe_corrections(E, terms, (1, -1, -1), want_log=True)
    e = E.cpu().numpy()
    ref = np.array([e[3] - e[1] - e[2], e[7] - e[0] - e[5]])
    assert np.allclose(out.cpu().numpy(), ref, rtol=0, atol=1e-15)
    assert np.allclose(lg.cpu().numpy(), np.log10(np.abs(ref) + 1e-16), rtol=1e-6)
