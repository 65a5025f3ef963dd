"""Failure detection in the tensor-core contraction kernel without a GPU fault: the test
hook rimp2_testing_set_wait_limit shortens the consumer-side mbarrier waits (MMA issuer
and epilogue) to zero, so that they expire while their data is still in flight.  The
kernel then takes its abort path (status bit, MMAs and TMA loads in flight drained with
the normal 2 s bound, TMEM freed) and the plan reports RIMP2_ERR_TIMEOUT; with the normal
limit restored the next call on the same plan and graph is correct again (checked against
the oracle).  No wait is left unbounded, nothing traps.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import oracle
from paper_2410_21888_gb300 import rimp2, synth

pytestmark = pytest.mark.gpu


def _set_limit():
    f = rimp2.load().rimp2_testing_set_wait_limit
    f.argtypes = [ctypes.c_int64]
    f.restype = ctypes.c_int
    return f


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_expired_waits_report_timeout_and_plan_recovers(precision):
    set_limit = _set_limit()
    f = synth.fragment_inputs(20, 80, 240, seed=3)
    ref = oracle.fragment(f.B, f.eo, f.ev)
    eng = rimp2.Engine([f.B.shape], precision=precision)
    eng.set_inputs([f])
    eng.run()                                  # captures the graph with the normal limit
    torch.cuda.synchronize()
    assert eng.plan.status() == 0
    try:
        assert set_limit(0) == 0
        eng.run()
        torch.cuda.synchronize()
        assert eng.plan.status() == -7         # RIMP2_ERR_TIMEOUT, then the word is clear
    finally:
        assert set_limit(-1) == 0
    for _ in range(2):
        eng.run()
        torch.cuda.synchronize()
        assert eng.plan.status() == 0
        v = eng.views(0)
        assert abs(float(v["energy"].item()) - ref["energy"]) <= 1e-8
        for k in ("gamma", "pij", "pab"):
            g = v[k].cpu().numpy()
            assert np.linalg.norm(g - ref[k]) <= 1e-9 * np.linalg.norm(ref[k]), k
