"""Pins of the oracle's MBE3 assembly of gradient intermediates (CPU): finite differences
of the MBE3 energy E = sum_f c_f E_f with respect to the system's global inputs, the
restriction of which every fragment sees.  dE/dB_global = 4 Gamma_sys (blocks with one,
two and three distinct monomers), dE/de = 2 diag P_sys, and an off-diagonal Fock coupling
between orbitals of two different monomers (applied in every fragment that holds both,
re-diagonalised with LAPACK eigh) gives 4 P_sys[k, l]."""
import numpy as np
import pytest

from oracle import mbe, oracle
from paper_2410_21888_gb300 import synth


def _system():
    s = synth.MonomerSystem(n_monomers=4, box=6.0, seed=11, nocc_range=(1, 2),
                            vir_per_occ=2, aux_per_orb=1)
    blocks = {}
    orig = s.block

    def block(I, J, K):
        if (I, J, K) not in blocks:
            blocks[(I, J, K)] = orig(I, J, K)
        return blocks[(I, J, K)]

    s.block = block
    return s, blocks


def _polymers(s):
    mons, dims, tris = mbe.all_polymers(s.n)
    dims, tris = dims[:4], tris[:3]          # a partial expansion: coefficients != trivial
    frags = [(m,) for m in mons] + dims + tris
    coeff = {f: 0 for f in frags}
    for t in tris:
        coeff[t] += 1
        for d in [(t[0], t[1]), (t[0], t[2]), (t[1], t[2])]:
            coeff[d] = coeff.get(d, 0) - 1
        for m in t:
            coeff[(m,)] += 1
    for d in dims:
        coeff[d] += 1
        for m in d:
            coeff[(m,)] -= 1
    for m in mons:
        coeff[(m,)] += 1
    frags = sorted(set(frags) | {d for d in coeff if coeff[d] != 0}, key=lambda f: (len(f), f))
    return mons, dims, tris, frags, coeff


def _energy_mbe(s, frags, coeff, fock=None):
    tot = 0.0
    for f in frags:
        x = s.fragment(f)
        B, eo, ev = x.B, x.eo, x.ev
        if fock is not None:
            blk, (I, k), (J, l), h = fock
            if I in f and J in f:
                n_of = s.nocc if blk == "occ" else s.nvir
                off = {m: int(np.sum(n_of[list(f[:p])])) for p, m in enumerate(f)}
                kk, ll = off[I] + k, off[J] + l
                if blk == "occ":
                    F = np.diag(eo).copy(); F[kk, ll] += h; F[ll, kk] += h
                    w, U = np.linalg.eigh(F)
                    B, eo = np.einsum("iI,iaQ->IaQ", U, B), w
                else:
                    F = np.diag(ev).copy(); F[kk, ll] += h; F[ll, kk] += h
                    w, U = np.linalg.eigh(F)
                    B, ev = np.einsum("aA,iaQ->iAQ", U, B), w
        tot += coeff[f] * oracle.fragment(B, eo, ev, want=())["energy"]
    return tot


@pytest.fixture(scope="module")
def assembled():
    s, blocks = _system()
    mons, dims, tris, frags, coeff = _polymers(s)
    outs = []
    for f in frags:
        x = s.fragment(f)
        outs.append((f, coeff[f], oracle.fragment(x.B, x.eo, x.ev)))
    pij, pab, gamma = mbe.assemble(s.nocc, s.nvir, s.naux, outs)
    return s, blocks, frags, coeff, pij, pab, gamma


def test_fd_mbe_energy_wrt_global_B_is_4_gamma_sys(assembled):
    s, blocks, frags, coeff, _, _, gamma = assembled
    h = 1e-5
    keys = [k for k in gamma if len(set(k)) == 1][:1] + [k for k in gamma if len(set(k)) == 2][:2] \
        + [k for k in gamma if len(set(k)) == 3][:2]
    assert len(keys) == 5
    for key in keys:
        blk = blocks[key]
        idx = tuple(d - 1 for d in blk.shape)
        old = blk[idx]
        blk[idx] = old + h
        ep = _energy_mbe(s, frags, coeff)
        blk[idx] = old - h
        em = _energy_mbe(s, frags, coeff)
        blk[idx] = old
        assert (ep - em) / (2 * h) == pytest.approx(4 * gamma[key][idx], rel=1e-6, abs=1e-11), key


def test_fd_mbe_energy_wrt_orbital_energies_is_2_diag_p_sys(assembled):
    s, _, frags, coeff, pij, pab, _ = assembled
    h = 1e-6
    oo = np.concatenate([[0], np.cumsum(s.nocc)])
    vo = np.concatenate([[0], np.cumsum(s.nvir)])
    for I in range(s.n):
        eo, ev = s.eps(I)
        for arr, base, P in ((eo, oo[I], pij), (ev, vo[I], pab)):
            old = arr[0]
            arr[0] = old + h
            ep = _energy_mbe(s, frags, coeff)
            arr[0] = old - h
            em = _energy_mbe(s, frags, coeff)
            arr[0] = old
            assert (ep - em) / (2 * h) == pytest.approx(2 * P[base, base], rel=1e-6)


def test_fd_intermonomer_fock_coupling_is_4_p_sys(assembled):
    s, _, frags, coeff, pij, pab, _ = assembled
    h = 1e-5
    oo = np.concatenate([[0], np.cumsum(s.nocc)])
    vo = np.concatenate([[0], np.cumsum(s.nvir)])
    for blk, P, base in (("occ", pij, oo), ("vir", pab, vo)):
        for (I, J) in [(0, 1), (1, 3), (0, 2)]:
            d = (_energy_mbe(s, frags, coeff, (blk, (I, 0), (J, 0), h))
                 - _energy_mbe(s, frags, coeff, (blk, (I, 0), (J, 0), -h))) / (2 * h)
            want = 4 * P[base[I], base[J]]
            assert d == pytest.approx(want, rel=1e-5, abs=1e-10), (blk, I, J)
            assert abs(want) > 1e-8
