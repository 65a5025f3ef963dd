"""Seeded synthetic inputs for the RI-MP2 hot path.

This module only draws inputs: orbital energies, MO-basis three-index tensors
B[nocc][nvir][naux] (naux fastest) and monomer geometries.  It holds none of the
method's arithmetic.  The CPU oracle tests and the GPU path both take their inputs
from here; the oracle itself never imports it.

The paper's molecular systems (urea/paracetamol crystal sections, PDB 6PQ5 and
2BEG, cc-pVDZ / cc-pVDZ-RIFIT; Sec. "Benchmark molecular systems") are not
available, so these seeded draws stand in for them:

* single fragment: eps_occ ~ U[-1.5, -0.3] Eh, eps_vir ~ U[0.2, 3.0] Eh,
  B^Q_ia ~ N(0, 0.05^2) i.i.d.;
* MBE3 system: monomer centroids ~ U[0, L]^3 bohr, nocc ~ U{8..20},
  nvir = 4 nocc, naux = 3 (nocc + nvir).  The system's B is one global tensor over
  the concatenated occupied, virtual and auxiliary sets of all monomers.  It is drawn
  block by block, one seed per (occ-owner, vir-owner, aux-owner) monomer triple, and
  a block whose owners span the monomer set S is multiplied by
  exp(-sum_{pairs in S} |R_I - R_K| / 3 bohr).  A fragment's B is the restriction of
  that global tensor to the fragment's monomers, so all MBE terms see one system.
"""
from __future__ import annotations

import copy
import itertools
from dataclasses import dataclass

import numpy as np

EPS_OCC = (-1.5, -0.3)
EPS_VIR = (0.2, 3.0)
B_SIGMA = 0.05
DECAY_BOHR = 3.0

# stream tags keep the per-monomer and per-block seed sequences apart
_TAG_EPS = 11
_TAG_BLOCK = 23
_TAG_GEOM = 37
_TAG_FULLMO = 41


@dataclass
class FragmentInputs:
    """One fragment's inputs: B[o][v][X] (float64, C order), eps_occ[o], eps_vir[v]."""

    B: np.ndarray
    eo: np.ndarray
    ev: np.ndarray

    @property
    def shape(self):
        return self.B.shape


def fragment_inputs(nocc: int, nvir: int, naux: int, seed: int = 0,
                    sigma: float = B_SIGMA) -> FragmentInputs:
    """Single seeded fragment (the tiny and the large single-fragment workloads)."""
    rng = np.random.default_rng(seed)
    eo = rng.uniform(EPS_OCC[0], EPS_OCC[1], size=nocc)
    ev = rng.uniform(EPS_VIR[0], EPS_VIR[1], size=nvir)
    B = rng.normal(0.0, sigma, size=(nocc, nvir, naux))
    return FragmentInputs(np.ascontiguousarray(B), eo, ev)


@dataclass
class FullMOInputs:
    """Inputs of the gradient step after the densities: the full MO-basis three-index
    tensor Bf[p][q][Q] (occupied orbitals first, symmetric in p, q), orbital energies
    eps[n], a symmetric positive definite J^{-1/2}[Q][P], and the fragment whose
    occupied-virtual block Bf[i][nocc + a] is frag.B[i][a]."""

    Bf: np.ndarray
    eps: np.ndarray
    jmh: np.ndarray
    frag: FragmentInputs


def full_mo_inputs(nocc: int, nvir: int, naux: int, seed: int = 0,
                   sigma: float | None = None, jmh_range=(0.5, 2.0)) -> FullMOInputs:
    """Seeded full-MO inputs around fragment_inputs(nocc, nvir, naux, seed, sigma): the
    occupied-occupied and virtual-virtual blocks of B are symmetrised normal draws of
    the same spread, J^{-1/2} = U diag(lambda) U^T with U orthogonal (QR of a normal
    matrix) and lambda ~ U[jmh_range].

    sigma defaults to 0.25 (nocc nvir naux)^(-1/4).  The Z-vector operator
    (e_a - e_i)/2 + 2 (ai|bj) - (aj|bi) is positive definite for a stable closed-shell
    reference, whose exchange integrals stay bounded; i.i.d. draws make the exchange
    part's spectrum grow like sigma^2 sqrt(nocc nvir naux), and at the hot path's
    sigma = 0.05 it already turns the operator indefinite at nocc=10, nvir=40, naux=150
    (lowest eigenvalue -0.29).  With the default the spectrum stays within about
    [0.25, 2.3] up to the nocc=100 nvir=500 naux=1500 fragment."""
    if sigma is None:
        sigma = 0.25 / max(1.0, float(nocc) * nvir * naux) ** 0.25
    frag = fragment_inputs(nocc, nvir, naux, seed, sigma)
    rng = np.random.default_rng([seed, _TAG_FULLMO])
    n = nocc + nvir
    Bf = np.zeros((n, n, naux))
    for lo, hi in ((0, nocc), (nocc, n)):
        m = hi - lo
        D = rng.normal(0.0, sigma, size=(m, m, naux))
        Bf[lo:hi, lo:hi] = (D + D.transpose(1, 0, 2)) / np.sqrt(2.0)
    Bf[:nocc, nocc:] = frag.B
    Bf[nocc:, :nocc] = frag.B.transpose(1, 0, 2)
    U, R = np.linalg.qr(rng.normal(size=(naux, naux)) if naux > 0 else np.zeros((0, 0)))
    U = U * np.sign(np.diag(R))[None, :] if naux > 0 else U
    lam = rng.uniform(jmh_range[0], jmh_range[1], size=naux)
    jmh = (U * lam[None, :]) @ U.T
    jmh = 0.5 * (jmh + jmh.T)
    eps = np.concatenate([frag.eo, frag.ev])
    return FullMOInputs(np.ascontiguousarray(Bf), eps, np.ascontiguousarray(jmh), frag)


class MonomerSystem:
    """Seeded monomer system for MBE3 batches (uneven monomer/dimer/trimer fragments)."""

    def __init__(self, n_monomers: int = 64, box: float = 40.0, seed: int = 0,
                 nocc_range=(8, 20), vir_per_occ: int = 4, aux_per_orb: int = 3,
                 decay: float = DECAY_BOHR, sigma: float = B_SIGMA):
        self.seed = int(seed)
        self.n = int(n_monomers)
        self.box = float(box)
        self.decay = float(decay)
        self.sigma = float(sigma)
        rng = np.random.default_rng([self.seed, _TAG_GEOM])
        self.centroids = rng.uniform(0.0, self.box, size=(self.n, 3))
        self.nocc = rng.integers(nocc_range[0], nocc_range[1] + 1, size=self.n)
        self.nvir = vir_per_occ * self.nocc
        self.naux = aux_per_orb * (self.nocc + self.nvir)
        self._eps = {}
        self.step = 0

    def at_step(self, step: int) -> "MonomerSystem":
        """The same system (geometry, orbital counts and energies) with the B blocks of
        time step `step` (fresh seeds per step; step 0 is this system)."""
        other = copy.copy(self)
        other.step = int(step)
        return other

    def distance(self, I: int, K: int) -> float:
        return float(np.linalg.norm(self.centroids[I] - self.centroids[K]))

    def eps(self, I: int):
        """Orbital energies of monomer I (seeded per monomer)."""
        if I not in self._eps:
            rng = np.random.default_rng([self.seed, _TAG_EPS, I])
            eo = rng.uniform(EPS_OCC[0], EPS_OCC[1], size=int(self.nocc[I]))
            ev = rng.uniform(EPS_VIR[0], EPS_VIR[1], size=int(self.nvir[I]))
            self._eps[I] = (eo, ev)
        return self._eps[I]

    def block_scale(self, owners) -> float:
        s = sorted(set(int(x) for x in owners))
        d = sum(self.distance(a, b) for a, b in itertools.combinations(s, 2))
        return float(np.exp(-d / self.decay))

    def block(self, I: int, J: int, K: int) -> np.ndarray:
        """Global-B block with occupied rows of I, virtual rows of J, aux columns of K."""
        key = [self.seed, _TAG_BLOCK, I, J, K] + ([self.step] if self.step else [])
        rng = np.random.default_rng(key)
        blk = rng.normal(0.0, self.sigma,
                         size=(int(self.nocc[I]), int(self.nvir[J]), int(self.naux[K])))
        return blk * self.block_scale((I, J, K))

    def fragment_dims(self, monomers):
        m = list(monomers)
        return (int(sum(self.nocc[m])), int(sum(self.nvir[m])), int(sum(self.naux[m])))

    def fragment(self, monomers) -> FragmentInputs:
        """Restriction of the global tensor to a polymer (tuple of monomer ids)."""
        m = [int(x) for x in monomers]
        o, v, X = self.fragment_dims(m)
        B = np.empty((o, v, X))
        oo = np.concatenate([[0], np.cumsum(self.nocc[m])])
        vo = np.concatenate([[0], np.cumsum(self.nvir[m])])
        xo = np.concatenate([[0], np.cumsum(self.naux[m])])
        for p, I in enumerate(m):
            for q, J in enumerate(m):
                for r, K in enumerate(m):
                    B[oo[p]:oo[p + 1], vo[q]:vo[q + 1], xo[r]:xo[r + 1]] = self.block(I, J, K)
        eo = np.concatenate([self.eps(I)[0] for I in m])
        ev = np.concatenate([self.eps(I)[1] for I in m])
        return FragmentInputs(B, eo, ev)


def pack_batch(frags):
    """Concatenate fragments into flat pools.

    Returns (B_pool, eps_pool, dims, offsets) with dims[f] = (o, v, X) and
    offsets[f] = (b_off, eo_off, ev_off, gamma_off, pij_off, pab_off, epair_off) in
    elements.  Gamma shares B's layout and offsets; P_ij, P_ab and the pair energies
    get pools of their own.  Pure bookkeeping, no arithmetic of the method.
    """
    dims, offs = [], []
    b = e = pij = pab = 0
    for fr in frags:
        o, v, X = fr.B.shape
        dims.append((o, v, X))
        offs.append((b, e, e + o, b, pij, pab, pij))
        b += o * v * X
        e += o + v
        pij += o * o
        pab += v * v
    B_pool = np.concatenate([fr.B.ravel() for fr in frags]) if frags else np.zeros(0)
    eps_pool = np.concatenate([np.concatenate([fr.eo, fr.ev]) for fr in frags]) if frags else np.zeros(0)
    return B_pool, eps_pool, dims, offs, (b, pij, pab)
