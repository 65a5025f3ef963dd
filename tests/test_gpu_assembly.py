"""MBE3 assembly of Gamma / P_ij / P_ab over the system's index spaces on the GPU against
the oracle's assembly (tests/test_mbe_assembly_pins.py pins the oracle by finite
differences of the MBE3 energy), for the FP64 and BF16 paths; level-by-level
accumulation equals the one-shot assembly bit for bit (same summation order)."""
import numpy as np
import pytest
import torch

from oracle import mbe as ombe
from oracle import oracle
from paper_2410_21888_gb300 import rimp2, synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def case():
    s = synth.MonomerSystem(n_monomers=6, box=10.0, seed=4, nocc_range=(2, 4))
    d, t = rimp2.mbe_polymers(s.centroids, 8.0, 7.0, "max")
    frags, coeff = rimp2.mbe_coefficients(s.n, d, t)
    frags = [tuple(int(x) for x in f) for f in frags]
    outs = []
    for f, c in zip(frags, coeff):
        x = s.fragment(f)
        outs.append((f, int(c), oracle.fragment(x.B, x.eo, x.ev)))
    ref = ombe.assemble(s.nocc, s.nvir, s.naux, outs)
    assert len(t) > 0 and len(d) > len(t)
    return s, frags, np.asarray(coeff), ref


def _engine(s, frags, precision):
    eng = rimp2.Engine([s.fragment_dims(f) for f in frags], precision=precision, want_epair=False)
    eng.set_inputs([s.fragment(f) for f in frags])
    eng.run()
    torch.cuda.synchronize()
    eng.check_status()
    return eng


def _assembly(s, frags, coeff, eng):
    offs = eng.offsets
    return rimp2.MBEAssembly(s.nocc, s.nvir, s.naux, frags, coeff, [o[0] for o in offs],
                             [o[2] for o in offs], [o[3] for o in offs])


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("bf16", 1e-9)])
def test_assembly_matches_oracle(case, precision, tol):
    s, frags, coeff, (pij_ref, pab_ref, gam_ref) = case
    eng = _engine(s, frags, precision)
    asm = _assembly(s, frags, coeff, eng)
    g, pij, pab = asm.outputs()
    asm.run(eng.gamma, eng.pij, eng.pab, g, pij, pab)
    torch.cuda.synchronize()
    assert rel(pij.cpu().numpy(), pij_ref) <= tol
    assert rel(pab.cpu().numpy(), pab_ref) <= tol
    assert set(gam_ref) == {tuple(k) for k in np.argwhere(asm.block_index >= 0)}
    num = den = 0.0
    for (I, J, K), blk in gam_ref.items():
        got = asm.block(g, I, J, K, s.nocc, s.nvir, s.naux).cpu().numpy()
        num += float(np.sum((got - blk) ** 2))
        den += float(np.sum(blk ** 2))
    assert np.sqrt(num / den) <= tol


def test_level_by_level_accumulation_equals_one_shot(case):
    s, frags, coeff, _ = case
    eng = _engine(s, frags, "bf16")
    asm = _assembly(s, frags, coeff, eng)
    g1, p1, q1 = asm.outputs()
    asm.run(eng.gamma, eng.pij, eng.pab, g1, p1, q1)
    g2, p2, q2 = asm.outputs()
    for level in (1, 2, 3):
        idx = [k for k, f in enumerate(frags) if len(f) == level]
        part = rimp2.MBEAssembly(s.nocc, s.nvir, s.naux, [frags[k] for k in idx], coeff[idx],
                                 [eng.offsets[k][0] for k in idx], [eng.offsets[k][2] for k in idx],
                                 [eng.offsets[k][3] for k in idx])
        # same block layout needs the same block set: map through the full index
        gp, _, _ = part.outputs()
        part.run(eng.gamma, eng.pij, eng.pab, gp, p2, q2, accumulate=level > 1)
        for I, J, K in np.argwhere(part.block_index >= 0):
            src = part.block(gp, I, J, K, s.nocc, s.nvir, s.naux)
            dst = asm.block(g2, I, J, K, s.nocc, s.nvir, s.naux)
            dst += src
    torch.cuda.synchronize()
    assert torch.equal(p1, p2) and torch.equal(q1, q2)
    assert torch.allclose(g1, g2, rtol=1e-13, atol=1e-15)
