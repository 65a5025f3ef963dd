"""GPU parity of the FP64 path against the CPU oracle, through the C ABI.

Tolerance: both sides are FP64 with different summation orders, so results agree to
about 1e-14 relative; the tests allow 1e-11 relative (energy) and 1e-11 relative
Frobenius (Gamma, P_ij, P_ab, pair energies).
"""
import numpy as np
import pytest
import torch

from oracle import oracle
from paper_2410_21888_gb300 import rimp2, synth

pytestmark = pytest.mark.gpu

TOL_E = 1e-11
TOL_A = 1e-11


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def check(out, ref, tol_e=TOL_E, tol_a=TOL_A):
    E = float(out["energy"].item())
    assert abs(E - ref["energy"]) <= tol_e * abs(ref["energy"]) + 1e-300, (E, ref["energy"])
    for k in ("gamma", "pij", "pab", "epair"):
        if k in out:
            g = out[k].detach().cpu().numpy()
            assert g.shape == ref[k].shape
            assert rel(g, ref[k]) <= tol_a, (k, rel(g, ref[k]))


@pytest.mark.parametrize("dims,seed", [
    ((10, 40, 150), 0),      # tiny single fragment
    ((1, 1, 1), 1),
    ((3, 5, 7), 2),
    ((2, 70, 33), 3),        # nvir crosses two 32-wide amplitude tiles, ov not multiple of 64
    ((7, 13, 129), 4),
    ((5, 31, 1), 5),         # naux = 1 (rank-1 V)
    ((13, 37, 17), 6),       # prime sizes, several GEMM tiles and a ragged tail
])
def test_fp64_fragment_parity(dims, seed):
    f = synth.fragment_inputs(*dims, seed=seed)
    ref = oracle.fragment(f.B, f.eo, f.ev)
    out = rimp2.energy_grad(f.B, f.eo, f.ev, precision="fp64")
    check(out, ref)


def test_fp64_degenerate_sizes():
    for dims in [(3, 0, 5), (0, 4, 5), (3, 4, 0)]:
        o, v, X = dims
        f = synth.fragment_inputs(*dims, seed=0)
        out = rimp2.energy_grad(f.B, f.eo, f.ev, precision="fp64")
        assert float(out["energy"].item()) == 0.0
        assert torch.count_nonzero(out["gamma"]).item() == 0
        assert torch.count_nonzero(out["pij"]).item() == 0
        assert torch.count_nonzero(out["pab"]).item() == 0


def _mbe_batch(seed=0, n=6, box=14.0):
    s = synth.MonomerSystem(n_monomers=n, box=box, seed=seed, nocc_range=(2, 5))
    polys = [(0,), (3,), (0, 1), (2, 4), (1, 3, 5), (0, 2, 4), (5,)]
    return [s.fragment(p) for p in polys]


@pytest.mark.parametrize("use_graph", [True, False])
def test_fp64_uneven_batch_one_call(use_graph):
    frags = _mbe_batch()
    eng = rimp2.Engine([f.B.shape for f in frags], precision="fp64", use_graph=use_graph)
    eng.set_inputs(frags)
    eng.run()
    torch.cuda.synchronize()
    eng.check_status()
    for k, f in enumerate(frags):
        check(eng.views(k), oracle.fragment(f.B, f.eo, f.ev))
    # replay gives identical energies
    e1 = eng.energy.clone()
    eng.run()
    torch.cuda.synchronize()
    assert torch.equal(e1, eng.energy)


def test_fp64_waves_match_single_wave():
    frags = _mbe_batch(seed=1)
    dims = [f.B.shape for f in frags]
    a = rimp2.Engine(dims, precision="fp64")
    b = rimp2.Engine(dims, precision="fp64", max_workspace_bytes=1 << 20)
    assert b.plan.stats().waves > 1
    for e in (a, b):
        e.set_inputs(frags)
        e.run()
    torch.cuda.synchronize()
    for k in range(len(frags)):
        va, vb = a.views(k), b.views(k)
        assert float(va["energy"]) == pytest.approx(float(vb["energy"]), rel=1e-13)
        assert rel(vb["gamma"].cpu(), va["gamma"].cpu()) < 1e-13


def test_status_denominator_and_nonfinite():
    f = synth.fragment_inputs(3, 4, 5, seed=0)
    eo = f.eo.copy()
    eo[1] = 0.5          # above min(eps_vir) = ... ensure violation
    ev = f.ev.copy()
    ev[0] = 0.25
    with pytest.raises(rimp2.Rimp2Error) as ei:
        rimp2.energy_grad(f.B, eo, ev, precision="fp64")
    assert ei.value.code == -3
    B = f.B.copy()
    B[1, 2, 3] = np.nan
    with pytest.raises(rimp2.Rimp2Error) as ei:
        rimp2.energy_grad(B, f.eo, f.ev, precision="fp64")
    assert ei.value.code == -4
    # the status word was cleared: a good call afterwards succeeds
    out = rimp2.energy_grad(f.B, f.eo, f.ev, precision="fp64")
    assert np.isfinite(float(out["energy"].item()))


def test_host_side_errors():
    eng = rimp2.Engine([(3, 4, 5)], precision="fp64")
    b = eng._batch
    b.nfrag = 2
    with pytest.raises(rimp2.Rimp2Error) as ei:
        eng.run()
    assert ei.value.code == -2
    b.nfrag = 1
    energy = b.energy
    b.energy = None
    with pytest.raises(rimp2.Rimp2Error) as ei:
        eng.run()
    assert ei.value.code == -1
    b.energy = energy
    small = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(rimp2.Rimp2Error) as ei:
        eng.plan.energy_grad(b, small)
    assert ei.value.code == -5
