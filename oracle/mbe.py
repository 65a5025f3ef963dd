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
