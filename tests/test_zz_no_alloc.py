"""rimp2_energy_fp64_noalloc: the entry point for callers that cannot allocate device
memory (an allocator that owns the whole device, a loop that cannot afford cudaMalloc's
synchronisation, a host that audits allocations); its scratch is a static device array
inside the library.  Checked through the C ABI against rimp2_energy_grad and against the
CPU oracle on the same inputs, on two calls in a row, with the FP64 tolerance of the
other GPU tests; then the capacity limit on both sides of its edge, and the NaN it
returns for inputs the device check rejects.  Collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import oracle
from paper_2410_21888_gb300 import rimp2, synth

pytestmark = pytest.mark.gpu

TOL = 1e-11
SCRATCH = 32 << 20


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


def _run(fn, B_np, eo, ev, with_epair=True):
    o, v, X = B_np.shape
    B = torch.as_tensor(B_np, device="cuda").contiguous()
    eps = torch.as_tensor(np.concatenate([eo, ev]), device="cuda")
    energy = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    epair = torch.full((o, o), np.nan, dtype=torch.float64, device="cuda") if with_epair else None
    rc = _call(fn, o, v, X, B, eps, energy, epair)
    torch.cuda.synchronize()
    return rc, float(energy.item()), (epair.cpu().numpy() if with_epair else None)


def _scratch_bytes(o, v):
    a256 = lambda x: (x + 255) // 256 * 256   # noqa: E731
    return 4096 + a256(8 * (o * v) ** 2) + a256(8 * o * o)


@pytest.mark.parametrize("dims", [(10, 40, 150), (7, 13, 29)])
def test_noalloc_matches_energy_grad_and_oracle_twice(dims):
    fn = _noalloc()
    o, v, X = dims
    for seed in (0, 1):   # two calls in a row, different inputs: no stale scratch
        f = synth.fragment_inputs(o, v, X, seed=seed)
        ref = rimp2.energy_grad(f.B, f.eo, f.ev, precision="fp64")
        orc = oracle.fragment(f.B, f.eo, f.ev, want=("epair",))
        rc, E, ep = _run(fn, f.B, f.eo, f.ev)
        assert rc == 0
        E_ref = float(ref["energy"].item())
        assert abs(E - E_ref) <= TOL * abs(E_ref)
        assert abs(E - orc["energy"]) <= TOL * abs(orc["energy"])
        ep_ref = ref["epair"].cpu().numpy()
        assert np.linalg.norm(ep - ep_ref) <= TOL * np.linalg.norm(ep_ref)
        assert np.linalg.norm(ep - orc["epair"]) <= TOL * np.linalg.norm(orc["epair"])


def test_noalloc_capacity_edge():
    """nocc=1, nvir=2047 is the widest single-occupied fragment the 32 MiB array holds
    (8 (nocc nvir)^2 bytes of T); nvir=2048 is rejected before any launch."""
    fn = _noalloc()
    assert _scratch_bytes(1, 2047) <= SCRATCH < _scratch_bytes(1, 2048)
    f = synth.fragment_inputs(1, 2047, 8, seed=3)
    rc, E, ep = _run(fn, f.B, f.eo, f.ev)
    assert rc == 0
    ref = oracle.fragment(f.B, f.eo, f.ev, want=("epair",))
    assert abs(E - ref["energy"]) <= TOL * abs(ref["energy"])
    assert ep[0, 0] == pytest.approx(ref["epair"][0, 0], rel=TOL)
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    assert _call(fn, 1, 2048, 8, dummy, dummy, dummy, None) == -5


def test_noalloc_rejects_oversize_and_bad_args():
    fn = _noalloc()
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    # nocc * nvir = 2100 exceeds the static scratch: rejected before any launch
    assert _scratch_bytes(21, 100) > SCRATCH
    assert _call(fn, 21, 100, 8, dummy, dummy, dummy, None) == -5
    assert _call(fn, -1, 4, 4, dummy, dummy, dummy, None) == -1
    stream = torch.cuda.current_stream().cuda_stream
    assert fn(2, 3, 4, dummy.data_ptr(), dummy.data_ptr(), None, None, stream) == -1


def test_noalloc_flags_rejected_inputs_as_nan_then_recovers():
    """An occupied energy above a virtual one (a non-negative denominator) and a NaN in B
    make the energy NaN; the next call with good inputs clears the shared status word."""
    fn = _noalloc()
    f = synth.fragment_inputs(4, 9, 20, seed=5)
    eo = f.eo.copy()
    eo[2] = f.ev.max() + 0.5
    rc, E, _ = _run(fn, f.B, eo, f.ev, with_epair=False)
    assert rc == 0 and np.isnan(E)
    B = f.B.copy()
    B[1, 3, 7] = np.nan
    rc, E, _ = _run(fn, B, f.eo, f.ev, with_epair=False)
    assert rc == 0 and np.isnan(E)
    rc, E, _ = _run(fn, f.B, f.eo, f.ev, with_epair=False)
    ref = oracle.fragment(f.B, f.eo, f.ev, want=())
    assert rc == 0 and abs(E - ref["energy"]) <= TOL * abs(ref["energy"])
