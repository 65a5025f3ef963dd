"""MBE3 through the GPU engine (one plan per MBE level, device combine) against the
oracle's fragment energies combined by the oracle's inclusion-exclusion (Eq. mbe3).

Tolerance: every fragment energy within 1e-8 Eh (split path target) or 1e-10 relative
(FP64 path); the MBE3 total within sum_f |c_f| x that per-fragment tolerance.
"""
import numpy as np
import pytest
import torch

from oracle import mbe as ombe
from oracle import oracle
from paper_2410_21888_gb300 import mbe, rimp2, synth

pytestmark = pytest.mark.gpu


def _system():
    return synth.MonomerSystem(n_monomers=7, box=11.0, seed=4, nocc_range=(2, 4))


@pytest.mark.parametrize("precision", ["fp64", "bf16"])
def test_mbe3_total_matches_oracle(precision):
    s = _system()
    run = mbe.MBE3(s, r_dimer=8.0, r_trimer=7.0, trimer_rule="two_pairs", precision=precision)
    res = run.run(timing=False)
    assert res.level_counts[3] > 0 and res.level_counts[2] > 0
    E = {}
    for f in res.fragments:
        x = s.fragment(f)
        E[f] = oracle.fragment(x.B, x.eo, x.ev, want=())["energy"]
    ref_frag = np.array([E[f] for f in res.fragments])
    tol = 1e-8 if precision == "bf16" else 1e-10 * np.abs(ref_frag) + 1e-12
    assert np.all(np.abs(res.frag_energy - ref_frag) <= tol)
    ref_total = ombe.mbe3(E, list(range(s.n)), [tuple(map(int, d)) for d in res.dimers],
                          [tuple(map(int, t)) for t in res.trimers])
    bound = float(np.sum(np.abs(res.coeff)) * (1e-8 if precision == "bf16" else 1e-10 *
                                                 np.max(np.abs(ref_frag))))
    assert abs(res.energy - ref_total) <= bound + 1e-12


def test_mbe_combine_is_deterministic_and_exact_on_integers():
    e = torch.arange(1, 5001, dtype=torch.float64, device="cuda") * 0.5
    c = torch.tensor([(-1) ** k * (1 + k % 3) for k in range(5000)], dtype=torch.int32,
                     device="cuda")
    a = rimp2.mbe_combine(e, c)
    b = rimp2.mbe_combine(e, c)
    torch.cuda.synchronize()
    ref = float(np.sum(c.cpu().numpy().astype(np.int64) * np.arange(1, 5001)) * 0.5)
    assert float(a.item()) == ref == float(b.item())


def test_mbe3_with_waves_matches_single_wave():
    s = _system()
    a = mbe.MBE3(s, 8.0, 7.0, "two_pairs", precision="bf16").run(timing=False)
    b = mbe.MBE3(s, 8.0, 7.0, "two_pairs", precision="bf16",
                 max_workspace_bytes=8 << 20).run(timing=False)
    assert np.allclose(a.frag_energy, b.frag_energy, rtol=1e-13, atol=1e-14)
