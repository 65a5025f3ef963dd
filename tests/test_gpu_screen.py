"""End to end learned screen on small monomer systems: labels computed by the engine
(split path with 8 slices, FP64-level), the network trained by the library's kernels,
then candidate trimers of an unseen system screened at 1e-7 Eh.  The test shows the gain
(trimers and trimer FLOPs skipped) and that the MBE3 total moves by at most 1e-6 Eh; a
5% sample of the skipped trimers is recomputed by the FP64 path as the audit; and, at
the same 1e-6 Eh budget, the learned ordering skips more trimers than the best distance
cutoff, the rule the screen replaces.
"""
import numpy as np
import pytest
import torch

from oracle import oracle
from paper_2410_21888_gb300 import screen, synth

pytestmark = pytest.mark.gpu


def _sys(seed):
    # 24 small monomers in a 40-bohr box; candidate trimers have two pairs within 20 bohr,
    # so their corrections span about 1e-12 .. 1e-3 Eh
    return synth.MonomerSystem(n_monomers=24, box=40.0, seed=seed, nocc_range=(2, 4))


def test_device_block_inputs_match_host_generator_structure():
    """Device-drawn fragments are restrictions of one global tensor: the (I,I,I) blocks
    of a dimer equal the monomer's, and block scaling follows the host generator."""
    from paper_2410_21888_gb300 import rimp2
    s = _sys(1)
    frags = [(0,), (0, 1)]
    eng = rimp2.Engine([s.fragment_dims(f) for f in frags], precision="fp64")
    screen.DeviceBlockInputs(s).fill(eng, frags)
    o0, v0, X0 = s.fragment_dims((0,))
    o1, v1, X1 = s.fragment_dims((0, 1))
    B0 = eng.B[:o0 * v0 * X0].view(o0, v0, X0)
    b = eng.offsets[1][0]
    B1 = eng.B[b:b + o1 * v1 * X1].view(o1, v1, X1)
    assert torch.equal(B0, B1[:o0, :v0, :X0])
    ratio = float(B1[:o0, :v0, X0:].abs().mean() / B0.abs().mean())
    assert ratio == pytest.approx(s.block_scale((0, 1)), rel=0.2)


def test_labels_match_oracle_on_host_inputs():
    s = synth.MonomerSystem(n_monomers=5, box=9.0, seed=2, nocc_range=(2, 3))
    ts = screen.trimer_set(s, None, device_inputs=False, trimers=[[0, 1, 2], [1, 3, 4]])
    E = {}
    for f in [(0,), (1,), (2,), (3,), (4,), (0, 1), (0, 2), (1, 2), (1, 3), (1, 4), (3, 4),
              (0, 1, 2), (1, 3, 4)]:
        x = s.fragment(f)
        E[f] = oracle.fragment(x.B, x.eo, x.ev, want=())["energy"]
    ref = [E[(0, 1, 2)] - E[(0, 1)] - E[(0, 2)] - E[(1, 2)] + E[(0,)] + E[(1,)] + E[(2,)],
           E[(1, 3, 4)] - E[(1, 3)] - E[(1, 4)] - E[(3, 4)] + E[(1,)] + E[(3,)] + E[(4,)]]
    assert np.allclose(ts.dE.cpu().numpy(), ref, rtol=0, atol=1e-9)


def test_screen_gain_and_error_bound():
    train = [screen.trimer_set(_sys(seed), 20.0) for seed in (10, 11, 12)]
    feats = torch.cat([t.feats for t in train])
    labels = torch.cat([t.labels for t in train])
    sc = screen.TrimerScreen(seed=0)
    sc.set_normalization(feats)
    l0 = sc.loss(feats, labels)
    sc.fit(feats, labels, epochs=150, batch=256, lr=3e-3)
    assert sc.loss(feats, labels) < 0.1 * l0
    test = screen.trimer_set(_sys(20), 20.0)
    res, skip = screen.screen_and_audit(_sys(20), sc, test, threshold=1e-7, margin_decades=1.0)
    assert res["skipped"] > 0.2 * res["candidates"], res
    assert abs(res["skipped_sum_Eh"]) <= 1e-6, res
    assert res["audit_count"] >= 1 and res["audit_max_abs_Eh"] < 1e-6, res
    assert res["audit_vs_method_max_diff_Eh"] < 1e-9, res
    # against the method without the screen: the best distance cutoff (max-pair or
    # two-pair distance, threshold chosen in hindsight) at the same 1e-6 Eh budget skips
    # fewer trimers than the learned ordering; no ordering beats the exact one
    cmp = screen.compare_with_distance_cutoff(_sys(20), test, sc.predict(test.feats).cpu().numpy(),
                                              1e-6)
    best_d = max(cmp["distance_max"]["skipped"], cmp["distance_two"]["skipped"])
    assert cmp["learned"]["skipped"] > best_d, cmp
    assert cmp["learned_gain_over_best_distance"] > 0, cmp
    assert cmp["exact"]["skipped"] >= cmp["learned"]["skipped"], cmp
    for k in ("distance_max", "distance_two", "learned", "exact"):
        assert abs(cmp[k]["skipped_sum_Eh"]) <= 1e-6, cmp
