"""Pins of the CPU oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: exact rational
arithmetic, a NumPy 4-index brute force, closed forms, finite differences (the
paper validates its analytic gradients the same way, Sec. "Measurement
methodology"), invariances and identities of the Appendix definitions, and the MBE
inclusion-exclusion of Eq. mbe3.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import brute, exact, mbe, oracle
from paper_2410_21888_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def frag(o, v, X, seed=0):
    f = synth.fragment_inputs(o, v, X, seed=seed)
    return f.B, f.eo, f.ev


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# ---------------------------------------------------------------- exact / brute force

@pytest.mark.parametrize("name", ["o1v1x3", "o2v2x3", "o3v2x1"])
def test_golden_exact(name):
    """Oracle vs exact rational results (golden fixtures, Appendix definitions)."""
    g = json.load(open(os.path.join(GOLDEN, f"exact_{name}.json")))
    B = np.array(g["inputs"]["B"], dtype=np.float64)
    r = oracle.fragment(B, np.array(g["inputs"]["eo"]), np.array(g["inputs"]["ev"]))
    assert r["energy"] == pytest.approx(g["energy"], rel=1e-15, abs=0)
    for k in ("gamma", "pij", "pab", "epair"):
        np.testing.assert_allclose(r[k], np.array(g[k]), rtol=2e-15, atol=1e-18)


def test_exact_module_closed_form_o1v1():
    """o = v = 1: E = (sum_Q B_Q^2)^2 / (2 (e_i - e_a)), Gamma_Q = E-derived closed form."""
    Bq = [Fraction(1, 4), Fraction(-3, 8), Fraction(5, 16), Fraction(1, 2)]
    ei, ea = Fraction(-3, 4), Fraction(5, 4)
    r = exact.everything([[Bq]], [ei], [ea])
    s = sum(b * b for b in Bq)
    D = 2 * (ei - ea)
    assert r["energy"] == s * s / D
    assert r["gamma"][0][0] == [s * b / D for b in Bq]
    assert r["pij"][0][0] == -(s / D) ** 2
    assert r["pab"][0][0] == (s / D) ** 2


@pytest.mark.parametrize("dims,seed", [((3, 5, 7), 0), ((1, 4, 3), 1), ((4, 1, 6), 2),
                                       ((2, 3, 1), 3), ((5, 6, 11), 4)])
def test_c_oracle_vs_numpy_brute_force(dims, seed):
    """C loops vs explicitly formed (ia|jb) (Eq. MP2_ints) contracted by einsum."""
    B, eo, ev = frag(*dims, seed=seed)
    a = oracle.fragment(B, eo, ev)
    b = brute.everything(B, eo, ev)
    assert a["energy"] == pytest.approx(b["energy"], rel=1e-13)
    for k in ("gamma", "pij", "pab", "epair"):
        assert rel(a[k], b[k]) < 1e-13, k


def test_single_output_routines_match_full():
    B, eo, ev = frag(6, 9, 13, seed=5)
    r = oracle.fragment(B, eo, ev)
    for (i, a, Q) in [(0, 0, 0), (5, 8, 12), (2, 3, 7)]:
        assert oracle.gamma_elem(B, eo, ev, i, a, Q) == pytest.approx(r["gamma"][i, a, Q], rel=1e-12)
    for (a, b) in [(0, 0), (8, 1), (4, 4)]:
        assert oracle.pab_elem(B, eo, ev, a, b) == pytest.approx(r["pab"][a, b], rel=1e-12)
    for (i, j) in [(0, 0), (5, 1), (3, 3)]:
        assert oracle.pij_elem(B, eo, ev, i, j) == pytest.approx(r["pij"][i, j], rel=1e-12)
        assert oracle.pair_energy(B, eo, ev, i, j) == pytest.approx(r["epair"][i, j], rel=1e-12)


def test_k_range_partitions_the_sum():
    B, eo, ev = frag(5, 7, 9, seed=6)
    full = oracle.fragment(B, eo, ev)
    parts = [oracle.fragment(B, eo, ev, k_range=(k0, k1)) for k0, k1 in [(0, 2), (2, 5)]]
    assert sum(p["energy"] for p in parts) == pytest.approx(full["energy"], rel=1e-14)
    for k in ("gamma", "pij", "pab"):
        assert rel(parts[0][k] + parts[1][k], full[k]) < 1e-14


def test_thread_count_does_not_change_result():
    B, eo, ev = frag(6, 8, 10, seed=7)
    a = oracle.fragment(B, eo, ev, nthreads=1)
    b = oracle.fragment(B, eo, ev, nthreads=4)
    assert a["energy"] == b["energy"]
    for k in ("gamma", "pij", "pab", "epair"):
        np.testing.assert_array_equal(a[k], b[k])


# ---------------------------------------------------------------- finite differences

def test_fd_energy_wrt_B_is_4_gamma():
    """dE/dB^Q_ia = 4 Gamma^Q_ia: the 4 Gamma term of the 3c coefficient Z (Appendix)."""
    B, eo, ev = frag(3, 4, 5, seed=8)
    g = oracle.fragment(B, eo, ev)["gamma"]
    h = 1e-5
    for idx in [(0, 0, 0), (2, 3, 4), (1, 2, 1), (0, 3, 2)]:
        Bp, Bm = B.copy(), B.copy()
        Bp[idx] += h
        Bm[idx] -= h
        d = (oracle.fragment(Bp, eo, ev, want=())["energy"]
             - oracle.fragment(Bm, eo, ev, want=())["energy"]) / (2 * h)
        assert d == pytest.approx(4 * g[idx], rel=1e-7, abs=1e-12)


def test_fd_energy_wrt_orbital_energies_is_2_diag_p():
    """dE/de_k = 2 P_kk and dE/de_c = 2 P_cc (D^MP2_ij, D^MP2_ab of the Appendix)."""
    B, eo, ev = frag(4, 5, 6, seed=9)
    r = oracle.fragment(B, eo, ev)
    h = 1e-6
    for k in range(4):
        p, m = eo.copy(), eo.copy()
        p[k] += h
        m[k] -= h
        d = (oracle.fragment(B, p, ev, want=())["energy"]
             - oracle.fragment(B, m, ev, want=())["energy"]) / (2 * h)
        assert d == pytest.approx(2 * r["pij"][k, k], rel=1e-7)
    for c in range(5):
        p, m = ev.copy(), ev.copy()
        p[c] += h
        m[c] -= h
        d = (oracle.fragment(B, eo, p, want=())["energy"]
             - oracle.fragment(B, eo, m, want=())["energy"]) / (2 * h)
        assert d == pytest.approx(2 * r["pab"][c, c], rel=1e-7)


def _energy_with_offdiag_fock(B, eo, ev, block, p, q, eps):
    """E after a symmetric Fock perturbation eps (E_pq + E_qp) in one block; the block
    is re-diagonalised with LAPACK eigh and B rotated into the new orbitals."""
    if block == "occ":
        F = np.diag(eo).copy()
        F[p, q] += eps
        F[q, p] += eps
        w, U = np.linalg.eigh(F)
        return oracle.fragment(np.einsum("iI,iaQ->IaQ", U, B), w, ev, want=())["energy"]
    F = np.diag(ev).copy()
    F[p, q] += eps
    F[q, p] += eps
    w, U = np.linalg.eigh(F)
    return oracle.fragment(np.einsum("aA,iaQ->iAQ", U, B), eo, w, want=())["energy"]


def test_fd_offdiagonal_densities_from_fock_perturbation():
    """Off-diagonal P: dE/deps = 4 P_kl for F = diag(e) + eps (E_kl + E_lk), in both
    the occupied and the virtual block (stationarity of the MP2 Hylleraas functional)."""
    B, eo, ev = frag(4, 6, 9, seed=3)
    r = oracle.fragment(B, eo, ev)
    h = 1e-5
    for (k, l) in [(0, 1), (1, 3), (0, 2)]:
        d = (_energy_with_offdiag_fock(B, eo, ev, "occ", k, l, h)
             - _energy_with_offdiag_fock(B, eo, ev, "occ", k, l, -h)) / (2 * h)
        assert d == pytest.approx(4 * r["pij"][k, l], rel=1e-6)
    for (c, d_) in [(0, 2), (3, 5), (1, 4)]:
        d = (_energy_with_offdiag_fock(B, eo, ev, "vir", c, d_, h)
             - _energy_with_offdiag_fock(B, eo, ev, "vir", c, d_, -h)) / (2 * h)
        assert d == pytest.approx(4 * r["pab"][c, d_], rel=1e-6)


# ---------------------------------------------------------------- identities / invariants

def test_homogeneity_B_dot_gamma_equals_energy():
    B, eo, ev = frag(5, 8, 12, seed=10)
    r = oracle.fragment(B, eo, ev)
    assert float(np.sum(B * r["gamma"])) == pytest.approx(r["energy"], rel=1e-12)


def test_euler_identity_orbital_energies():
    """E is homogeneous of degree -1 in the orbital energies:
    -E = 2 (sum_i e_i P_ii + sum_a e_a P_aa)."""
    B, eo, ev = frag(5, 7, 9, seed=11)
    r = oracle.fragment(B, eo, ev)
    lhs = -r["energy"]
    rhs = 2.0 * (eo @ np.diag(r["pij"]) + ev @ np.diag(r["pab"]))
    assert rhs == pytest.approx(lhs, rel=1e-12)


def test_aux_rotation_invariance():
    """E, P_ij, P_ab invariant and Gamma covariant under B -> B O (O orthogonal on Q)."""
    B, eo, ev = frag(4, 6, 10, seed=12)
    O, _ = np.linalg.qr(np.random.default_rng(0).normal(size=(10, 10)))
    a = oracle.fragment(B, eo, ev)
    b = oracle.fragment(B @ O, eo, ev)
    assert b["energy"] == pytest.approx(a["energy"], rel=1e-12)
    assert rel(b["pij"], a["pij"]) < 1e-12
    assert rel(b["pab"], a["pab"]) < 1e-12
    assert rel(b["gamma"], a["gamma"] @ O) < 1e-12


def test_scaling_laws():
    B, eo, ev = frag(3, 5, 6, seed=13)
    a = oracle.fragment(B, eo, ev)
    s = 1.75
    b = oracle.fragment(s * B, eo, ev)
    assert b["energy"] == pytest.approx(s ** 4 * a["energy"], rel=1e-13)
    assert rel(b["gamma"], s ** 3 * a["gamma"]) < 1e-13
    assert rel(b["pij"], s ** 4 * a["pij"]) < 1e-13
    assert rel(b["pab"], s ** 4 * a["pab"]) < 1e-13
    lam = 2.5
    c = oracle.fragment(B, lam * eo, lam * ev)
    assert c["energy"] == pytest.approx(a["energy"] / lam, rel=1e-13)


def test_density_trace_symmetry_and_signs():
    B, eo, ev = frag(6, 9, 14, seed=14)
    r = oracle.fragment(B, eo, ev)
    assert np.trace(r["pij"]) == pytest.approx(-np.trace(r["pab"]), rel=1e-12)
    assert rel(r["pij"], r["pij"].T) < 1e-13
    assert rel(r["pab"], r["pab"].T) < 1e-13
    assert np.all(np.diag(r["pij"]) <= 0)
    assert np.all(np.diag(r["pab"]) >= 0)
    assert rel(r["epair"], r["epair"].T) < 1e-13


@pytest.mark.parametrize("seed", range(5))
def test_energy_negative_for_negative_denominators(seed):
    B, eo, ev = frag(4, 6, 8, seed=seed)
    assert oracle.fragment(B, eo, ev, want=())["energy"] < 0


def _planted(B, eo, ev, mistake=None):
    """Copy of the brute force with one plausible mistake planted (or none)."""
    iajb = brute.integrals(B)
    D = brute.denominators(eo, ev)
    if mistake == "denominator_sign":          # e_i + e_j - e_a + e_b
        D = (eo[:, None, None, None] + eo[None, None, :, None]
             - ev[None, :, None, None] + ev[None, None, None, :])
    T = iajb / D
    Tt = 2.0 * T - T.transpose(0, 3, 2, 1)
    if mistake == "no_exchange":
        Tt = 2.0 * T
    if mistake == "exchange_factor":
        Tt = T - T.transpose(0, 3, 2, 1)
    E = float(np.sum(Tt * iajb))
    g = np.einsum("iajb,jbQ->iaQ", Tt, B)
    if mistake == "gamma_transposed":
        g = np.einsum("ibja,jbQ->iaQ", Tt, B)
    pij = -np.einsum("iakb,jakb->ij", Tt, T)
    if mistake == "pij_index":
        pij = -np.einsum("iakb,jbka->ij", Tt, T)
    pab = np.einsum("iajc,ibjc->ab", Tt, T)
    if mistake == "pab_factor2":
        pab = 2.0 * pab
    return E, g, pij, pab


def _pins_pass(fn):
    """Run the FD / identity / closed-form pins on an arbitrary implementation."""
    B, eo, ev = frag(3, 4, 5, seed=8)
    E, g, pij, pab = fn(B, eo, ev)
    ok = True
    h = 1e-5
    for idx in [(0, 0, 0), (2, 3, 4), (1, 2, 1)]:
        Bp, Bm = B.copy(), B.copy()
        Bp[idx] += h
        Bm[idx] -= h
        d = (fn(Bp, eo, ev)[0] - fn(Bm, eo, ev)[0]) / (2 * h)
        ok &= abs(d - 4 * g[idx]) <= 1e-6 * abs(d) + 1e-12
    for k in range(3):
        p, m = eo.copy(), eo.copy()
        p[k] += h
        m[k] -= h
        d = (fn(B, p, ev)[0] - fn(B, m, ev)[0]) / (2 * h)
        ok &= abs(d - 2 * pij[k, k]) <= 1e-6 * abs(d)
    for (k, l) in [(0, 1), (1, 2)]:
        def e_of(eps):
            F = np.diag(eo).copy()
            F[k, l] += eps
            F[l, k] += eps
            w, U = np.linalg.eigh(F)
            return fn(np.einsum("iI,iaQ->IaQ", U, B), w, ev)[0]
        d = (e_of(h) - e_of(-h)) / (2 * h)
        ok &= abs(d - 4 * pij[k, l]) <= 1e-5 * abs(d)
    for c in range(4):
        p, m = ev.copy(), ev.copy()
        p[c] += h
        m[c] -= h
        d = (fn(B, eo, p)[0] - fn(B, eo, m)[0]) / (2 * h)
        ok &= abs(d - 2 * pab[c, c]) <= 1e-6 * abs(d)
    # closed form o = v = 1
    b1 = B[:1, :1, :]
    s = float(np.sum(b1 * b1))
    ok &= abs(fn(b1, eo[:1], ev[:1])[0] - s * s / (2 * (eo[0] - ev[0]))) < 1e-12
    return bool(ok)


def test_pins_reject_planted_mistakes():
    """The pin suite passes the genuine definitions and fails every planted mistake
    (dropped exchange, wrong exchange factor, flipped denominator sign, transposed
    Gamma, wrong P index, doubled P_ab)."""
    assert _pins_pass(lambda B, eo, ev: _planted(B, eo, ev))
    for m in ("no_exchange", "exchange_factor", "denominator_sign", "gamma_transposed",
              "pij_index", "pab_factor2"):
        assert not _pins_pass(lambda B, eo, ev, m=m: _planted(B, eo, ev, m)), m


# ---------------------------------------------------------------- MBE3 (Eq. mbe3)

def _fragment_energy(sys_, monomers):
    f = sys_.fragment(monomers)
    return oracle.fragment(f.B, f.eo, f.ev, want=())["energy"]


def test_mbe3_exact_for_three_monomers():
    s = synth.MonomerSystem(n_monomers=3, box=6.0, seed=1, nocc_range=(1, 2))
    mons, dims, tris = mbe.all_polymers(3)
    E = {}
    for p in [(m,) for m in mons] + dims + tris:
        E[p] = _fragment_energy(s, p)
    assert mbe.mbe3(E, mons, dims, tris) == pytest.approx(E[(0, 1, 2)], rel=1e-13)


def test_mbe3_exact_when_four_body_terms_vanish():
    """With B^Q_ia nonzero only when a and Q sit on the same monomer, every energy term
    touches at most three monomers (owners of i, j and of a = b = Q), so the MBE3
    truncation of Eq. mbe3 reproduces the full-system energy for any monomer count."""
    n = 5
    s = synth.MonomerSystem(n_monomers=n, box=8.0, seed=2, nocc_range=(1, 2))
    orig = s.block

    def block(I, J, K):
        b = orig(I, J, K)
        return b if J == K else np.zeros_like(b)

    s.block = block
    mons, dims, tris = mbe.all_polymers(n)
    E = {}
    for p in [(m,) for m in mons] + dims + tris:
        E[p] = _fragment_energy(s, p)
    full = _fragment_energy(s, tuple(range(n)))
    assert mbe.mbe3(E, mons, dims, tris) == pytest.approx(full, rel=1e-12)
    # and the 4-body remainder really is nonzero without the restriction
    s.block = orig
    E2 = {p: _fragment_energy(s, p) for p in E}
    full2 = _fragment_energy(s, tuple(range(n)))
    assert abs(mbe.mbe3(E2, mons, dims, tris) - full2) > 1e-10 * abs(full2)


def test_mbe_corrections_vanish_without_coupling():
    s = synth.MonomerSystem(n_monomers=3, box=10.0, seed=3, nocc_range=(1, 3))
    orig = s.block
    s.block = lambda I, J, K: orig(I, J, K) if I == J == K else np.zeros_like(orig(I, J, K))
    E = {p: _fragment_energy(s, p) for p in [(0,), (1,), (2,), (0, 1), (0, 2), (1, 2), (0, 1, 2)]}
    for d in [(0, 1), (0, 2), (1, 2)]:
        assert abs(mbe.dimer_correction(E, *d)) < 1e-13 * abs(E[d])
    assert abs(mbe.trimer_correction(E, 0, 1, 2)) < 1e-13 * abs(E[(0, 1, 2)])


def test_mbe3_combine_on_three_body_function():
    """Combine code alone: a fragment 'energy' that is a sum of <=3-body terms is
    reproduced exactly by MBE3 for any N."""
    rng = np.random.default_rng(4)
    n = 7
    e1 = rng.normal(size=n)
    e2 = rng.normal(size=(n, n))
    e3 = rng.normal(size=(n, n, n))
    import itertools

    def f(p):
        return (sum(e1[i] for i in p) + sum(e2[i, j] for i, j in itertools.combinations(p, 2))
                + sum(e3[i, j, k] for i, j, k in itertools.combinations(p, 3)))

    mons, dims, tris = mbe.all_polymers(n)
    E = {p: f(p) for p in [(m,) for m in mons] + dims + tris}
    assert mbe.mbe3(E, mons, dims, tris) == pytest.approx(f(tuple(range(n))), rel=1e-12)


# ---------------------------------------------------------------- spin components

@pytest.mark.parametrize("dims,seed", [((3, 5, 7), 0), ((2, 4, 6), 1), ((4, 3, 5), 2)])
def test_spin_components_vs_spin_orbital_brute_force(dims, seed):
    """The oracle's spatial-orbital sums against the spin-orbital form (alpha-beta pairs
    with (ia|jb)^2, same-spin pairs with antisymmetrised integrals)."""
    B, eo, ev = frag(*dims, seed=seed)
    e_os, e_ss = oracle.spin_components(B, eo, ev)
    b_os, b_ss = brute.spin_components(B, eo, ev)
    assert e_os == pytest.approx(b_os, rel=1e-12)
    assert e_ss == pytest.approx(b_ss, rel=1e-12)
    assert e_os + e_ss == pytest.approx(oracle.fragment(B, eo, ev, want=())["energy"], rel=1e-12)


def test_spin_components_closed_forms_and_signs():
    # nocc = nvir = 1: E_OS = (sum_Q B^2)^2 / (2 (e_i - e_a)) and no same-spin pair exists
    B, eo, ev = frag(1, 1, 5)
    e_os, e_ss = oracle.spin_components(B, eo, ev)
    s2 = float(np.sum(B * B))
    assert e_os == pytest.approx(s2 * s2 / (2.0 * (eo[0] - ev[0])), rel=1e-14)
    assert e_ss == 0.0
    # one virtual: a = b only, so E_SS = 0 exactly; one occupied: V_ii(a,b) is symmetric
    # in (a,b), so E_SS vanishes up to the rounding of the denominators
    B, eo, ev = frag(4, 1, 6, seed=3)
    assert oracle.spin_components(B, eo, ev)[1] == 0.0
    B, eo, ev = frag(1, 6, 9, seed=4)
    e_os, e_ss = oracle.spin_components(B, eo, ev)
    assert abs(e_ss) <= 1e-14 * abs(e_os)
    # both components are sums of squares over negative denominators
    for seed in range(4):
        e_os, e_ss = oracle.spin_components(*frag(3, 5, 6, seed=seed))
        assert e_os < 0 and e_ss < 0


def test_pair_spin_components_sum_and_symmetry():
    B, eo, ev = frag(3, 4, 5, seed=5)
    pairs = {(i, j): oracle.pair_spin(B, eo, ev, i, j) for i in range(3) for j in range(3)}
    e_os, e_ss = oracle.spin_components(B, eo, ev)
    assert sum(p[0] for p in pairs.values()) == pytest.approx(e_os, rel=1e-13)
    assert sum(p[1] for p in pairs.values()) == pytest.approx(e_ss, rel=1e-13)
    for (i, j), p in pairs.items():
        assert p[0] == pytest.approx(pairs[(j, i)][0], rel=1e-13)
        assert p[1] == pytest.approx(pairs[(j, i)][1], rel=1e-13)
    ep = oracle.fragment(B, eo, ev, want=("epair",))["epair"]
    for (i, j), p in pairs.items():
        assert p[0] + p[1] == pytest.approx(ep[i, j], rel=1e-12)
