"""Reference for the step of the RI-MP2 gradient after the densities (Appendix): the
J^{-1/2} back-transform of Gamma, the Lagrangian pieces L' and L'', and the Z-vector
equation for the occupied-virtual block D_ai of the relaxed MP2 density.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU
baseline may import this module.  Plain NumPy in FP64, written from the Appendix's
definitions term by term; library primitives (einsum, inv, solve) serve as steps.

Inputs (MO basis, occupied orbitals first, n = nocc + nvir):
  Bf[p][q][Q]   B^Q_pq = sum_P (pq|P) J^{-1/2}_PQ, symmetric in (p, q)
  eps[n]        orbital energies
  jmh[Q][P]     J^{-1/2}, symmetric positive definite
  gamma[i][a][Q], pij[i][j], pab[a][b]: Gamma^Q_ia = sum_jb Tt_ij(a,b) B^Q_jb and the
                unrelaxed densities D^MP2_ij, D^MP2_ab of the hot path

Readings (the Appendix states these only through its index names):
  * L'_ia in the Z-vector equation is L'_iq at q = a, L''_ai is L''_aq at q = i.
  * (P|pq) = sum_Q B^Q_pq J^{1/2}_QP with J^{1/2} = (J^{-1/2})^{-1}: the three-centre
    integrals that B was formed from.
  * The unknown D_bj on the left is the block D_ai being solved for; D-bar holds the
    D_ij and D_ab blocks.  eps_ai = e_a - e_i (the paper's macro).
  * The solution is returned as dai[i][a] = D_ai (occupied index first, like B^Q_ia).

Parity of solve_dai is pinned by brute-force loops for the integrals and G, by the
symmetry of the Z-vector operator, and by closed forms for special inputs; see
tests/test_zvector_pins.py.
"""
from __future__ import annotations

import numpy as np


def eri(Bf):
    """(pq|rs)_RI = sum_Q B^Q_pq B^Q_rs (Eq. MP2_ints), all four indices over the MOs."""
    return np.einsum("pqQ,rsQ->pqrs", Bf, Bf, optimize=True)


def g_tensor(Bf):
    """G^{rs}_pq = 2 (pq|rs)_RI - (ps|rq)_RI (Appendix), returned as G[p, q, r, s]."""
    I = eri(Bf)
    return 2.0 * I - I.transpose(0, 3, 2, 1)


def gamma_aux(gamma, jmh):
    """Gamma^P_ia = sum_Q Gamma^Q_ia J^{-1/2}_PQ (Appendix, auxiliary quantities)."""
    return np.einsum("iaQ,PQ->iaP", gamma, jmh, optimize=True)


def three_centre(Bf, jmh):
    """(P|pq) = sum_Q B^Q_pq J^{1/2}_QP with J^{1/2} the inverse of J^{-1/2}; [p][q][P]."""
    jh = np.linalg.inv(jmh)
    return np.einsum("pqQ,QP->pqP", Bf, jh, optimize=True)


def lagrangian(gamma, Bf, jmh, nocc):
    """L'_iq = sum_aP Gamma^P_ia (P|qa) and L''_aq = sum_iP Gamma^P_ia (P|iq) (Appendix),
    from the back-transformed Gamma and the three-centre integrals.  Returns
    (Lp[nocc][n], Lpp[nvir][n])."""
    gP = gamma_aux(gamma, jmh)
    T3 = three_centre(Bf, jmh)
    o = nocc
    Lp = np.einsum("iaP,qaP->iq", gP, T3[:, o:, :], optimize=True)
    Lpp = np.einsum("iaP,iqP->aq", gP, T3[:o, :, :], optimize=True)
    return Lp, Lpp


def zvector_system(Bf, eps, gamma, pij, pab, jmh, nocc):
    """The Z-vector equation as a dense linear system A z = r over the (a, i) pairs
    (Appendix):
      (e_a - e_i)/2 D_ai + sum_bj G^{bj}_ai D_bj = L''_ai - L'_ia - sum_pq G^{pq}_ai Dbar_pq.
    Returns (A[(i,a),(j,b)], r[(i,a)]) with the pair index (i, a) -> i * nvir + a."""
    o = nocc
    n = Bf.shape[0]
    v = n - o
    G = g_tensor(Bf)
    occ, vir = slice(0, o), slice(o, n)
    # G^{bj}_ai = G[a, i, b, j]
    Gvo = G[vir, occ, vir, occ]                                   # [a][i][b][j]
    A = np.einsum("aibj->iajb", Gvo).reshape(o * v, o * v).copy()
    gap = (eps[None, o:] - eps[:o, None]).reshape(-1)             # e_a - e_i at (i, a)
    A[np.diag_indices(o * v)] += 0.5 * gap
    Lp, Lpp = lagrangian(gamma, Bf, jmh, o)
    rhs = Lpp[:, :o].T - Lp[:, o:]                                # [i][a]: L''_ai - L'_ia
    rhs = rhs - np.einsum("aikl,kl->ia", G[vir, occ, occ, occ], pij, optimize=True)
    rhs = rhs - np.einsum("aibc,bc->ia", G[vir, occ, vir, vir], pab, optimize=True)
    return A, rhs.reshape(-1)


def solve_dai(Bf, eps, gamma, pij, pab, jmh, nocc):
    """D_ai from the Z-vector equation by a dense direct solve; returned as [nocc][nvir]."""
    A, r = zvector_system(Bf, eps, gamma, pij, pab, jmh, nocc)
    v = Bf.shape[0] - nocc
    return np.linalg.solve(A, r).reshape(nocc, v)


def gradient_chain(Bf, eps, gamma, pij, pab, jmh, nocc):
    """All outputs of the step: Gamma^P, L', L'', D_ai."""
    Lp, Lpp = lagrangian(gamma, Bf, jmh, nocc)
    return {"gamma_p": gamma_aux(gamma, jmh), "lp": Lp, "lpp": Lpp,
            "dai": solve_dai(Bf, eps, gamma, pij, pab, jmh, nocc)}


# ------------------------------------------------------------------ matrix-free forms
# For fragments too large for the dense system: the same operator and right-hand side
# contracted term by term (pinned against zvector_system in tests/test_zvector_pins.py).

def zvector_apply(Bf, eps, x, nocc):
    """(A x)_ia = (e_a - e_i)/2 x_ia + sum_bj [2 (ai|bj) - (aj|bi)] x_jb for x[i][a]."""
    o = nocc
    Bov = Bf[:o, o:, :]                                            # B^Q_ia
    coul = np.einsum("iaQ,Q->ia", Bov, np.einsum("jbQ,jb->Q", Bov, x, optimize=True),
                     optimize=True)
    W = np.einsum("ibQ,jb->ijQ", Bov, x, optimize=True)            # sum_b B^Q_ib x_jb
    exch = np.einsum("jaQ,ijQ->ia", Bov, W, optimize=True)         # sum_jQ B^Q_ja W^Q_ij
    gap = eps[None, o:] - eps[:o, None]
    return 0.5 * gap * x + 2.0 * coul - exch


def zvector_rhs(Bf, gamma, pij, pab, nocc):
    """L''_ai - L'_ia - sum_pq G^{pq}_ai Dbar_pq at [i][a], with L', L'' in their MO-B form
    (sum_Q Gamma^Q B^Q, equal to the three-centre form since J^{-1/2} J^{1/2} = 1)."""
    o = nocc
    Bov, Boo, Bvv = Bf[:o, o:, :], Bf[:o, :o, :], Bf[o:, o:, :]
    Lp_ia = np.einsum("icQ,acQ->ia", gamma, Bvv, optimize=True)    # L'_ia = sum_cQ G^Q_ic B^Q_ac
    Lpp_ai = np.einsum("jaQ,jiQ->ia", gamma, Boo, optimize=True)   # L''_ai = sum_jQ G^Q_ja B^Q_ji
    d = np.einsum("klQ,kl->Q", Boo, pij, optimize=True)
    e = np.einsum("bcQ,bc->Q", Bvv, pab, optimize=True)
    U = np.einsum("ikQ,kl->ilQ", Boo, pij, optimize=True)
    V = np.einsum("ibQ,bc->icQ", Bov, pab, optimize=True)
    g_oo = 2.0 * np.einsum("iaQ,Q->ia", Bov, d, optimize=True) - \
        np.einsum("laQ,ilQ->ia", Bov, U, optimize=True)
    g_vv = 2.0 * np.einsum("iaQ,Q->ia", Bov, e, optimize=True) - \
        np.einsum("acQ,icQ->ia", Bvv, V, optimize=True)
    return Lpp_ai - Lp_ia - g_oo - g_vv


def lagrangian_elem(gamma, Bf, jmh, nocc, which, row, q):
    """One element L'_{row,q} (which = "lp", row = i) or L''_{row,q} (which = "lpp",
    row = a) from the three-centre form, for fragments too large for lagrangian()."""
    o = nocc
    jh = np.linalg.inv(jmh)
    if which == "lp":
        gP = gamma[row] @ jmh.T                                    # Gamma^P_ia, [a][P]
        T3 = Bf[q, o:, :] @ jh                                     # (P|q a), [a][P]
        return float(np.sum(gP * T3))
    gP = gamma[:, row, :] @ jmh.T                                  # Gamma^P_ia for all i, [i][P]
    T3 = Bf[:o, q, :] @ jh                                         # (P|i q), [i][P]
    return float(np.sum(gP * T3))
