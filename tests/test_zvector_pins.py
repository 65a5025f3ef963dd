"""Pins of the gradient-step oracle (oracle/zvector.py) to facts outside itself:
brute-force index loops for the RI integrals and G, the definition of B through the
three-centre integrals, the identity J^{-1/2} J^{1/2} = 1 behind the MO-B form of L'
and L'', the symmetry of the Z-vector operator, a closed form when the occupied-virtual
block of B vanishes, and the Z-vector equation evaluated by loops over every index."""
import itertools

import numpy as np
import pytest

from oracle import oracle, zvector
from paper_2410_21888_gb300 import synth


def _inputs(o, v, X, seed):
    f = synth.full_mo_inputs(o, v, X, seed=seed)
    ref = oracle.fragment(f.frag.B, f.frag.eo, f.frag.ev)
    return f, ref


def _loops_eri(Bf):
    n, _, X = Bf.shape
    I = np.zeros((n, n, n, n))
    for p, q, r, s in itertools.product(range(n), repeat=4):
        I[p, q, r, s] = sum(Bf[p, q, Q] * Bf[r, s, Q] for Q in range(X))
    return I


def test_eri_and_g_match_index_loops():
    f = synth.full_mo_inputs(2, 3, 4, seed=3)
    I = _loops_eri(f.Bf)
    assert np.allclose(zvector.eri(f.Bf), I, rtol=0, atol=1e-15)
    G = zvector.g_tensor(f.Bf)
    n = f.Bf.shape[0]
    for p, q, r, s in itertools.product(range(n), repeat=4):
        assert abs(G[p, q, r, s] - (2 * I[p, q, r, s] - I[p, s, r, q])) <= 1e-15


def test_three_centre_integrals_reproduce_b():
    """B^Q_pq = sum_P (pq|P) J^{-1/2}_PQ is how B is defined from the integrals."""
    f = synth.full_mo_inputs(3, 4, 6, seed=5)
    T3 = zvector.three_centre(f.Bf, f.jmh)
    back = np.einsum("pqP,PQ->pqQ", T3, f.jmh)
    assert np.allclose(back, f.Bf, rtol=0, atol=1e-14)


@pytest.mark.parametrize("dims,seed", [((3, 5, 7), 0), ((4, 6, 9), 1)])
def test_lagrangian_equals_mo_b_form(dims, seed):
    """sum_P Gamma^P (P|..) = sum_Q Gamma^Q B^Q because J^{-1/2} J^{1/2} = 1."""
    f, ref = _inputs(*dims, seed)
    o = dims[0]
    Lp, Lpp = zvector.lagrangian(ref["gamma"], f.Bf, f.jmh, o)
    g = ref["gamma"]
    Lp2 = np.einsum("iaQ,qaQ->iq", g, f.Bf[:, o:, :])
    Lpp2 = np.einsum("iaQ,iqQ->aq", g, f.Bf[:o, :, :])
    scale = np.abs(Lp2).max() + np.abs(Lpp2).max()
    assert np.abs(Lp - Lp2).max() <= 1e-12 * scale
    assert np.abs(Lpp - Lpp2).max() <= 1e-12 * scale
    # J^{-1/2} = 1: Gamma^P is Gamma^Q
    assert np.array_equal(zvector.gamma_aux(g, np.eye(dims[2])), g)


def test_zvector_operator_symmetric_positive_definite():
    f, ref = _inputs(4, 6, 9, 2)
    A, _ = zvector.zvector_system(f.Bf, f.eps, ref["gamma"], ref["pij"], ref["pab"], f.jmh, 4)
    assert np.abs(A - A.T).max() <= 1e-15 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0


def test_zvector_closed_form_without_ov_block():
    """With B^Q_ia = 0 every G term of the equation vanishes (each holds an ov element of
    B), so D_ai = 2 (L''_ai - L'_ia) / (e_a - e_i), L' and L'' from the oo and vv blocks."""
    o, v, X = 3, 4, 5
    f = synth.full_mo_inputs(o, v, X, seed=7)
    Bf = f.Bf.copy()
    Bf[:o, o:] = 0.0
    Bf[o:, :o] = 0.0
    rng = np.random.default_rng(1)
    gamma = rng.normal(size=(o, v, X))
    pij = rng.normal(size=(o, o)); pij = pij + pij.T
    pab = rng.normal(size=(v, v)); pab = pab + pab.T
    D = zvector.solve_dai(Bf, f.eps, gamma, pij, pab, f.jmh, o)
    Lp = np.einsum("ibQ,abQ->ia", gamma, Bf[o:, o:, :])        # L'_ia = sum_bQ G^Q_ib B^Q_ab
    Lpp = np.einsum("jaQ,jiQ->ia", gamma, Bf[:o, :o, :])       # L''_ai = sum_jQ G^Q_ja B^Q_ji
    gap = f.eps[None, o:] - f.eps[:o, None]
    assert np.allclose(D, 2.0 * (Lpp - Lp) / gap, rtol=1e-12, atol=1e-14)


def test_zvector_solution_satisfies_equation_by_loops():
    """Every term of the Appendix's Z-vector equation summed by explicit loops over the
    MO indices, at the oracle's solution."""
    o, v, X = 2, 3, 4
    f, ref = _inputs(o, v, X, 9)
    n = o + v
    D = zvector.solve_dai(f.Bf, f.eps, ref["gamma"], ref["pij"], ref["pab"], f.jmh, o)
    I = _loops_eri(f.Bf)
    Lp, Lpp = zvector.lagrangian(ref["gamma"], f.Bf, f.jmh, o)

    def G(p, q, r, s):
        return 2 * I[p, q, r, s] - I[p, s, r, q]

    Dbar = np.zeros((n, n))
    Dbar[:o, :o] = ref["pij"]
    Dbar[o:, o:] = ref["pab"]
    worst = 0.0
    for i in range(o):
        for a in range(v):
            A_ = o + a
            lhs = 0.5 * (f.eps[A_] - f.eps[i]) * D[i, a]
            lhs += sum(G(A_, i, o + b, j) * D[j, b] for b in range(v) for j in range(o))
            rhs = Lpp[a, i] - Lp[i, A_]
            rhs -= sum(G(A_, i, p, q) * Dbar[p, q] for p in range(n) for q in range(n))
            worst = max(worst, abs(lhs - rhs) / (abs(rhs) + 1e-300))
    assert worst <= 1e-10


@pytest.mark.parametrize("dims,seed", [((3, 5, 7), 4), ((5, 8, 11), 6)])
def test_matrix_free_forms_match_dense_system(dims, seed):
    """The matrix-free operator and right-hand side (used where the dense system does not
    fit) against the system built from G, and single Lagrangian elements against L', L''."""
    o, v, X = dims
    f, ref = _inputs(o, v, X, seed)
    A, r = zvector.zvector_system(f.Bf, f.eps, ref["gamma"], ref["pij"], ref["pab"], f.jmh, o)
    x = np.random.default_rng(seed).normal(size=(o, v))
    Ax = zvector.zvector_apply(f.Bf, f.eps, x, o)
    assert np.abs(Ax.reshape(-1) - A @ x.reshape(-1)).max() <= 1e-13 * np.abs(A @ x.reshape(-1)).max()
    rr = zvector.zvector_rhs(f.Bf, ref["gamma"], ref["pij"], ref["pab"], o)
    assert np.abs(rr.reshape(-1) - r).max() <= 1e-12 * np.abs(r).max()
    Lp, Lpp = zvector.lagrangian(ref["gamma"], f.Bf, f.jmh, o)
    for (i, q) in [(0, 0), (o - 1, o + v - 1), (1, 2)]:
        assert abs(zvector.lagrangian_elem(ref["gamma"], f.Bf, f.jmh, o, "lp", i, q) - Lp[i, q]) \
            <= 1e-13 * np.abs(Lp).max()
    for (a, q) in [(0, 0), (v - 1, 1), (2, o + 3)]:
        assert abs(zvector.lagrangian_elem(ref["gamma"], f.Bf, f.jmh, o, "lpp", a, q) - Lpp[a, q]) \
            <= 1e-13 * np.abs(Lpp).max()


@pytest.mark.parametrize("dims", [(10, 40, 150), (20, 70, 130), (30, 50, 400)])
def test_synthetic_full_mo_inputs_keep_operator_positive_definite(dims):
    """The size-scaled spread of synth.full_mo_inputs keeps the Z-vector operator's
    spectrum inside ~[0.25, 2.5] (the orbital-gap range), so conjugate gradients apply;
    the hot path's i.i.d. spread 0.05 makes it indefinite at the first of these sizes."""
    o, v, X = dims
    f = synth.full_mo_inputs(o, v, X, seed=1)
    z = np.zeros((o, v, X))
    A, _ = zvector.zvector_system(f.Bf, f.eps, z, np.zeros((o, o)), np.zeros((v, v)), f.jmh, o)
    ev = np.linalg.eigvalsh(A)
    assert ev.min() > 0.2 and ev.max() < 2.6, (ev.min(), ev.max())
    if dims == (10, 40, 150):
        g = synth.full_mo_inputs(o, v, X, seed=1, sigma=0.05)
        A2, _ = zvector.zvector_system(g.Bf, g.eps, z, np.zeros((o, o)), np.zeros((v, v)), g.jmh, o)
        assert np.linalg.eigvalsh(A2).min() < 0
