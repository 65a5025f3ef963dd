"""Opposite-/same-spin energy components (SCS-MP2, named in the paper's Introduction) on
the GPU against the oracle: E_OS = sum T V from the amplitude stage of every path, with
E_SS = E - E_OS; single fragments with ragged tiles and an uneven batch.  Tolerances as
for the energy: 1e-8 Eh (split paths), 1e-11 relative (FP64)."""
import numpy as np
import pytest
import torch

from oracle import oracle
from paper_2410_21888_gb300 import rimp2, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,seed", [((5, 20, 30), 0), ((13, 37, 17), 6), ((4, 130, 300), 7),
                                       ((1, 9, 12), 2)])
@pytest.mark.parametrize("precision", ["fp64", "bf16", "fp8"])
def test_spin_components_match_oracle(dims, seed, precision):
    f = synth.fragment_inputs(*dims, seed=seed)
    e_os, e_ss = oracle.spin_components(f.B, f.eo, f.ev)
    out = rimp2.energy_grad(f.B, f.eo, f.ev, precision=precision, want_gamma=False, want_p=False)
    E, Eos = float(out["energy"].item()), float(out["energy_os"].item())
    tol = 1e-11 * abs(e_os) if precision == "fp64" else 1e-8
    assert abs(Eos - e_os) <= tol, (Eos, e_os)
    assert abs((E - Eos) - e_ss) <= tol + 1e-11 * abs(e_ss), (E - Eos, e_ss)
    # SCS-MP2 combination formed by the library: default (Grimme) and SOS-MP2 weights
    scs = float(out["energy_scs"].item())
    assert scs == pytest.approx(1.2 * e_os + e_ss / 3.0, abs=2 * tol + 1e-12)
    sos = float(rimp2.scs_energy(f.B, f.eo, f.ev, precision=precision, c_os=1.3,
                                 c_ss=0.0).item())
    assert sos == pytest.approx(1.3 * e_os, abs=2 * tol + 1e-12)


@pytest.mark.parametrize("precision", ["fp64", "bf16"])
def test_spin_components_uneven_batch(precision):
    s = synth.MonomerSystem(n_monomers=6, box=14.0, seed=0, nocc_range=(2, 5))
    polys = [(0,), (3,), (0, 1), (2, 4), (1, 3, 5), (0, 2, 4), (5,)]
    frags = [s.fragment(p) for p in polys]
    eng = rimp2.Engine([f.B.shape for f in frags], precision=precision)
    eng.set_inputs(frags)
    eng.run()
    torch.cuda.synchronize()
    eng.check_status()
    Eos = eng.energy_os[:len(frags)].cpu().numpy()
    for k, f in enumerate(frags):
        ref = oracle.spin_components(f.B, f.eo, f.ev)[0]
        tol = 1e-11 * abs(ref) if precision == "fp64" else 1e-8
        assert abs(Eos[k] - ref) <= tol, (k, Eos[k], ref)
    assert np.all(Eos < 0)
