"""rimp2_energy_fp64_noalloc: the entry point for callers that cannot allocate device
memory (its scratch is a static device array inside the library).  Checked through the
C ABI against rimp2_energy_grad on the same inputs, on two calls in a row, with the
FP64 tolerance of the other GPU tests.  Collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2410_21888_gb300 import rimp2, synth

pytestmark = pytest.mark.gpu

TOL = 1e-11


def _noalloc():
    lib = rimp2.load()
    f = lib.rimp2_energy_fp64_noalloc
    f.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def _call(fn, o, v, X, B, eps, energy, epair):
    stream = torch.cuda.current_stream().cuda_stream
    return fn(o, v, X, B.data_ptr(), eps.data_ptr(), energy.data_ptr(),
              None if epair is None else epair.data_ptr(), stream)


@pytest.mark.parametrize("dims", [(10, 40, 150), (7, 13, 29)])
def test_noalloc_matches_energy_grad_twice(dims):
    fn = _noalloc()
    o, v, X = dims
    for seed in (0, 1):   # two calls in a row, different inputs: no stale scratch
        f = synth.fragment_inputs(o, v, X, seed=seed)
        ref = rimp2.energy_grad(f.B, f.eo, f.ev, precision="fp64")
        B = torch.as_tensor(f.B, device="cuda").contiguous()
        eps = torch.as_tensor(np.concatenate([f.eo, f.ev]), device="cuda")
        energy = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
        epair = torch.full((o, o), np.nan, dtype=torch.float64, device="cuda")
        assert _call(fn, o, v, X, B, eps, energy, epair) == 0
        torch.cuda.synchronize()
        E_ref = float(ref["energy"].item())
        assert abs(float(energy.item()) - E_ref) <= TOL * abs(E_ref)
        ep_ref = ref["epair"].cpu().numpy()
        ep = epair.cpu().numpy()
        assert np.linalg.norm(ep - ep_ref) <= TOL * np.linalg.norm(ep_ref)


def test_noalloc_rejects_oversize_and_bad_args():
    fn = _noalloc()
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    # nocc * nvir = 2000 exceeds the static scratch: rejected before any launch
    assert _call(fn, 20, 100, 8, dummy, dummy, dummy, None) == -5
    assert _call(fn, -1, 4, 4, dummy, dummy, dummy, None) == -1
    stream = torch.cuda.current_stream().cuda_stream
    assert fn(2, 3, 4, dummy.data_ptr(), dummy.data_ptr(), None, None, stream) == -1
