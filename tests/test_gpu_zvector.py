"""GPU tests of the gradient step after the densities (include/rimp2_grad.h) against the
oracle (oracle/zvector.py): Gamma^P, L', L'', D_ai element by element on fragments the
dense oracle solves, ragged across the 64 x 64 GEMM tiles; degenerate sizes; and, at the
nocc=100 nvir=500 naux=1500 fragment, sampled Lagrangian elements and the residual of the
Z-vector equation evaluated by the oracle's matrix-free operator.

Tolerances: Gamma^P, L', L'' are FP64 GEMMs (1e-12 relative Frobenius); D_ai comes from
conjugate gradients run to ||r|| <= 1e-12 ||rhs||, i.e. within the condition number
(below 10 for these inputs) times 1e-12 of the exact solution: 1e-10 relative."""
import numpy as np
import pytest
import torch

from oracle import oracle, zvector
from paper_2410_21888_gb300 import rimp2, synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


@pytest.mark.parametrize("dims,seed", [
    ((3, 5, 7), 0),
    ((1, 1, 1), 1),
    ((10, 40, 150), 2),
    ((20, 70, 130), 3),     # several N tiles over nvir, naux and n
    ((66, 30, 70), 4),      # nocc past one 64-row tile
])
def test_zvector_step_matches_oracle(dims, seed):
    o, v, X = dims
    f = synth.full_mo_inputs(o, v, X, seed=seed)
    ref = oracle.fragment(f.frag.B, f.frag.eo, f.frag.ev)
    want = zvector.gradient_chain(f.Bf, f.eps, ref["gamma"], ref["pij"], ref["pab"], f.jmh, o)
    got = rimp2.zvector(f.Bf, f.eps, ref["gamma"], ref["pij"], ref["pab"], jmh=f.jmh)
    info = got["info"].cpu().numpy()
    assert 1 <= info[0] <= 100 and info[1] <= 1e-12, info
    for k in ("gamma_p", "lp", "lpp"):
        assert rel(got[k].cpu().numpy(), want[k]) <= 1e-12, k
    assert rel(got["dai"].cpu().numpy(), want["dai"]) <= 1e-10


def test_zvector_without_jmh_and_zero_sizes():
    f = synth.full_mo_inputs(4, 6, 9, seed=5)
    ref = oracle.fragment(f.frag.B, f.frag.eo, f.frag.ev)
    got = rimp2.zvector(f.Bf, f.eps, ref["gamma"], ref["pij"], ref["pab"])
    assert "gamma_p" not in got
    want = zvector.solve_dai(f.Bf, f.eps, ref["gamma"], ref["pij"], ref["pab"], f.jmh, 4)
    assert rel(got["dai"].cpu().numpy(), want) <= 1e-10
    for o, v, X in [(0, 5, 4), (3, 0, 4), (3, 4, 0)]:
        n = o + v
        out = rimp2.zvector(np.zeros((n, n, X)), np.arange(n, dtype=float) - o + 0.5,
                            np.zeros((o, v, X)), np.zeros((o, o)), np.zeros((v, v)))
        for k in ("lp", "lpp", "dai"):
            assert torch.count_nonzero(out[k]).item() == 0
        assert out["info"][0].item() == 0.0


def test_zvector_not_converged_reports_it():
    """One iteration cannot reach 1e-12: iterations = max_iter + 1 flags it."""
    f = synth.full_mo_inputs(6, 20, 40, seed=6)
    ref = oracle.fragment(f.frag.B, f.frag.eo, f.frag.ev)
    got = rimp2.zvector(f.Bf, f.eps, ref["gamma"], ref["pij"], ref["pab"], max_iter=1)
    info = got["info"].cpu().numpy()
    assert info[0] == 2.0 and info[1] > 1e-12


def test_zvector_large_fragment_residual():
    """nocc=100 nvir=500 naux=1500: Gamma and the densities are seeded draws of the same
    magnitudes (the step is linear in them); the residual of the Z-vector equation is
    recomputed by the oracle's matrix-free operator and right-hand side."""
    o, v, X = 100, 500, 1500
    f = synth.full_mo_inputs(o, v, X, seed=0)
    rng = np.random.default_rng(123)
    gamma = rng.normal(0.0, 1e-3, size=(o, v, X))
    pij = rng.normal(0.0, 1e-3, size=(o, o)); pij = -(pij @ pij.T)
    pab = rng.normal(0.0, 1e-3, size=(v, v)); pab = pab @ pab.T
    got = rimp2.zvector(f.Bf, f.eps, gamma, pij, pab, jmh=f.jmh)
    info = got["info"].cpu().numpy()
    assert 1 <= info[0] <= 100 and info[1] <= 1e-12, info
    D = got["dai"].cpu().numpy()
    r = zvector.zvector_rhs(f.Bf, gamma, pij, pab, o)
    res = zvector.zvector_apply(f.Bf, f.eps, D, o) - r
    assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(r)
    lp, lpp = got["lp"].cpu().numpy(), got["lpp"].cpu().numpy()
    for (i, q) in [(0, 0), (57, 333), (99, 599)]:
        ref = zvector.lagrangian_elem(gamma, f.Bf, f.jmh, o, "lp", i, q)
        assert abs(lp[i, q] - ref) <= 1e-11 * np.abs(lp).max()
    for (a, q) in [(0, 7), (250, 99), (499, 512)]:
        ref = zvector.lagrangian_elem(gamma, f.Bf, f.jmh, o, "lpp", a, q)
        assert abs(lpp[a, q] - ref) <= 1e-11 * np.abs(lpp).max()
    gp = got["gamma_p"].cpu().numpy()
    for (i, a) in [(3, 17), (88, 401)]:
        assert np.abs(gp[i, a] - f.jmh @ gamma[i, a]).max() <= 1e-12 * np.abs(gp).max()
