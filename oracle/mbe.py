"""Reference many-body expansion (MBE3) combine.  TEST INFRASTRUCTURE ONLY.

Eq. mbe3: E = sum_I E_I + sum_{I<J} dE_IJ + sum_{I<J<K} dE_IJK, with the pair
correction dE_IJ = E_IJ - E_I - E_J given in Sec. "Molecular Fragmentation".  The
trimer correction is the standard inclusion-exclusion the paper describes in words
("subtract lower-order contributions"):
    dE_IJK = E_IJK - E_IJ - E_IK - E_JK + E_I + E_J + E_K.
Dimers/trimers absent from the polymer list contribute nothing.  Sums use math.fsum.
"""
from __future__ import annotations

import itertools
import math


def dimer_correction(E, I, J):
    return E[(I, J)] - E[(I,)] - E[(J,)]


def trimer_correction(E, I, J, K):
    return (E[(I, J, K)] - E[(I, J)] - E[(I, K)] - E[(J, K)]
            + E[(I,)] + E[(J,)] + E[(K,)])


def mbe3(E, monomers, dimers, trimers):
    """E maps sorted monomer tuples to fragment energies."""
    terms = [E[(I,)] for I in monomers]
    terms += [dimer_correction(E, *d) for d in dimers]
    terms += [trimer_correction(E, *t) for t in trimers]
    return math.fsum(terms)


def all_polymers(n):
    mons = list(range(n))
    return mons, list(itertools.combinations(mons, 2)), list(itertools.combinations(mons, 3))


def polymers(centroids, r_dimer, r_trimer, rule="max"):
    """Brute-force polymer lists: dimers with centroid distance <= r_dimer; trimers with
    all pair distances <= r_trimer ("max") or at least two of them ("two_pairs")."""
    import numpy as np
    c = np.asarray(centroids, dtype=float)
    n = len(c)

    def d(a, b):
        return float(np.sqrt(np.sum((c[a] - c[b]) ** 2)))

    dimers = [(a, b) for a, b in itertools.combinations(range(n), 2) if d(a, b) <= r_dimer]
    trimers = []
    for a, b, e in itertools.combinations(range(n), 3):
        ds = [d(a, b), d(a, e), d(b, e)]
        ok = max(ds) <= r_trimer if rule == "max" else sum(x <= r_trimer for x in ds) >= 2
        if ok:
            trimers.append((a, b, e))
    return dimers, trimers


def assemble(nocc, nvir, naux, fragments):
    """MBE3 assembly of the fragments' gradient intermediates over the system's index
    spaces (occupied, virtual and auxiliary orbitals of all monomers, monomer by monomer):
        P_ij_sys[(I,i),(J,j)]          = sum_f c_f P_ij,f[(I,i),(J,j)]
        P_ab_sys[(I,a),(J,b)]          = sum_f c_f P_ab,f[(I,a),(J,b)]
        Gamma_sys[(I,J,K)][i][a][Q]    = sum_f c_f Gamma_f[(I,i)][(J,a)][(K,Q)]
    over the fragments f containing the monomers involved.  Because E_MBE3 = sum_f c_f E_f
    with every fragment seeing a restriction of one global B and orbital-energy set,
    these are the MBE3 derivatives dE/dB = 4 Gamma_sys, dE/de = 2 diag(P_sys) and the
    off-diagonal Fock couplings 4 P_sys.  The trimer coefficients are all 1 (Sec.
    "Asynchronous time steps" accumulates trimer gradients directly for that reason).
    `fragments`: list of (monomer tuple, coefficient, dict with gamma, pij, pab)."""
    import numpy as np
    nocc, nvir, naux = (np.asarray(x, dtype=int) for x in (nocc, nvir, naux))
    oo = np.concatenate([[0], np.cumsum(nocc)])
    vo = np.concatenate([[0], np.cumsum(nvir)])
    pij = np.zeros((oo[-1], oo[-1]))
    pab = np.zeros((vo[-1], vo[-1]))
    gamma = {}
    for mons, c, out in fragments:
        m = list(mons)
        fo = np.concatenate([[0], np.cumsum(nocc[m])])
        fv = np.concatenate([[0], np.cumsum(nvir[m])])
        fx = np.concatenate([[0], np.cumsum(naux[m])])
        for p, I in enumerate(m):
            for q, J in enumerate(m):
                pij[oo[I]:oo[I + 1], oo[J]:oo[J + 1]] += c * out["pij"][fo[p]:fo[p + 1], fo[q]:fo[q + 1]]
                pab[vo[I]:vo[I + 1], vo[J]:vo[J + 1]] += c * out["pab"][fv[p]:fv[p + 1], fv[q]:fv[q + 1]]
                for r, K in enumerate(m):
                    blk = gamma.setdefault((I, J, K), np.zeros((nocc[I], nvir[J], naux[K])))
                    blk += c * out["gamma"][fo[p]:fo[p + 1], fv[q]:fv[q + 1], fx[r]:fx[r + 1]]
    return pij, pab, gamma
