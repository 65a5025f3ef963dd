"""NumPy brute force of the RI-MP2 energy and intermediates from the explicit 4-index
integrals (ia|jb).  TEST INFRASTRUCTURE ONLY, for tiny sizes.

It forms the whole (ia|jb) array (Eq. MP2_ints) and the amplitudes of the Appendix
with einsum, independently of the C loops in rimp2_oracle.c, so the two check each
other.  Definitions are the ones listed in that file's header.
"""
from __future__ import annotations

import numpy as np


def integrals(B):
    """(ia|jb)_RI = sum_Q B^Q_ia B^Q_jb as an array [i, a, j, b]."""
    return np.einsum("iaQ,jbQ->iajb", B, B)


def denominators(eo, ev):
    """D[i, a, j, b] = e_i + e_j - e_a - e_b."""
    return (eo[:, None, None, None] + eo[None, None, :, None]
            - ev[None, :, None, None] - ev[None, None, None, :])


def everything(B, eo, ev):
    """Dict with energy, gamma, pij, pab, epair (brute force)."""
    iajb = integrals(B)
    T = iajb / denominators(eo, ev)                 # X^ab_ij stored as T[i, a, j, b]
    Tt = 2.0 * T - T.transpose(0, 3, 2, 1)          # 2 X^ab_ij - X^ba_ij
    epair = np.einsum("iajb,iajb->ij", Tt, iajb)
    energy = float(np.sum(epair))
    gamma = np.einsum("iajb,jbQ->iaQ", Tt, B)
    pij = -np.einsum("iakb,jakb->ij", Tt, T)
    pab = np.einsum("iajc,ibjc->ab", Tt, T)
    return {"energy": energy, "gamma": gamma, "pij": pij, "pab": pab, "epair": epair}


def energy(B, eo, ev) -> float:
    return everything(B, eo, ev)["energy"]


def spin_components(B, eo, ev):
    """(E_OS, E_SS) in the spin-orbital form, independent of the spatial-orbital sums of
    rimp2_oracle.c: the alpha-beta pairs give E_OS = sum_ijab (ia|jb)^2 / D_ijab; the
    alpha-alpha and beta-beta pairs give, with antisymmetrised integrals
    <ij||ab> = (ia|jb) - (ib|ja), E_SS = 2 sum_{i<j} sum_{a<b} <ij||ab>^2 / D_ijab."""
    iajb = integrals(B)
    D = denominators(eo, ev)
    e_os = float(np.sum(iajb * iajb / D))
    o, v = len(eo), len(ev)
    e_ss = 0.0
    for i in range(o):
        for j in range(i + 1, o):
            for a in range(v):
                for b in range(a + 1, v):
                    anti = iajb[i, a, j, b] - iajb[i, b, j, a]
                    e_ss += 2.0 * anti * anti / D[i, a, j, b]
    return e_os, e_ss
