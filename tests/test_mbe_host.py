"""MBE3 host logic of the library (polymer formation, inclusion-exclusion coefficients)
against the oracle's brute force; CPU only (no compute call needs a GPU)."""
import math

import numpy as np
import pytest

from oracle import mbe as ombe
from paper_2410_21888_gb300 import build as libbuild
from paper_2410_21888_gb300 import rimp2, synth


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()


@pytest.mark.parametrize("rule", ["max", "two_pairs"])
@pytest.mark.parametrize("seed", [0, 1])
def test_polymers_match_brute_force(rule, seed):
    s = synth.MonomerSystem(n_monomers=20, box=20.0, seed=seed)
    d, t = rimp2.mbe_polymers(s.centroids, 9.0, 7.5, rule)
    bd, bt = ombe.polymers(s.centroids, 9.0, 7.5, rule)
    assert [tuple(x) for x in d] == bd
    assert [tuple(x) for x in t] == bt


def test_polymers_counts_for_the_64_monomer_box():
    """64 monomers in a 40-bohr box: dimers within 12 bohr, trimers with every pair
    within 10 bohr (the stated cutoffs), and the two-pair rule used for count-matched
    batches."""
    s = synth.MonomerSystem(n_monomers=64, box=40.0, seed=0)
    d, t = rimp2.mbe_polymers(s.centroids, 12.0, 10.0, "max")
    bd, bt = ombe.polymers(s.centroids, 12.0, 10.0, "max")
    assert len(d) == len(bd) and len(t) == len(bt)
    d2, t2 = rimp2.mbe_polymers(s.centroids, 16.0, 15.0, "two_pairs")
    assert len(d2) > len(d) and len(t2) > len(t)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_coefficients_reproduce_inclusion_exclusion(seed):
    s = synth.MonomerSystem(n_monomers=12, box=14.0, seed=seed)
    d, t = rimp2.mbe_polymers(s.centroids, 8.0, 7.0, "two_pairs")
    frags, coeff = rimp2.mbe_coefficients(s.n, d, t)
    fs = set(frags)
    for tri in t:                       # every sub-pair of a kept trimer is present
        a, b, c = (int(x) for x in tri)
        assert {(a, b), (a, c), (b, c)} <= fs
    rng = np.random.default_rng(seed)
    E = {f: float(rng.normal()) for f in frags}
    mons = list(range(s.n))
    ref = ombe.mbe3(E, mons, [tuple(int(x) for x in p) for p in d],
                    [tuple(int(x) for x in p) for p in t])
    got = math.fsum(c * E[f] for f, c in zip(frags, coeff))
    assert got == pytest.approx(ref, abs=1e-12)


def test_coefficients_reject_bad_ids():
    with pytest.raises(rimp2.Rimp2Error):
        rimp2.mbe_coefficients(3, [[0, 3]], [])
    with pytest.raises(rimp2.Rimp2Error):
        rimp2.mbe_coefficients(3, [], [[0, 1, 1]])
