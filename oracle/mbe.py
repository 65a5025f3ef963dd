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
