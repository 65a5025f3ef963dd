"""Asynchronous MBE3 time steps on the GPU: the async schedule (each wave of step t+1
waits only for the step-t waves sharing its monomers) gives exactly the numbers of the
synchronous one, and every step's fragment energies and MBE3 totals match the oracle on
that step's inputs (two small systems, three steps, host-drawn inputs)."""
import math

import numpy as np
import pytest

from oracle import oracle
from paper_2410_21888_gb300 import pipeline, synth

pytestmark = pytest.mark.gpu


def test_async_equals_sync_and_oracle():
    systems = [synth.MonomerSystem(n_monomers=8, box=12.0, seed=s, nocc_range=(2, 4))
               for s in (0, 1)]
    pipe = pipeline.AsyncMBE3(systems, 9.0, 8.0, "max", n_waves=4, precision="bf16",
                              workspace_budget=8 * 2 ** 30, inputs="host")
    assert len(pipe.waves) == 4
    pipe.prepare_steps(3)
    e_sync, tot_sync, _ = pipe.run("sync")
    e_async, tot_async, _ = pipe.run("async")
    assert np.array_equal(e_sync.cpu().numpy(), e_async.cpu().numpy())
    assert np.array_equal(tot_sync.cpu().numpy(), tot_async.cpu().numpy())
    E = e_async.cpu().numpy()
    T = tot_async.cpu().numpy()
    for t in range(3):
        ref = []
        for it in pipe.items:
            x = systems[it.system].at_step(t).fragment(it.monomers)
            ref.append(oracle.fragment(x.B, x.eo, x.ev, want=())["energy"])
        assert np.max(np.abs(E[t] - np.array(ref))) <= 1e-8
        for s_idx, (a, b) in enumerate(pipe.sys_slices):
            want = math.fsum(pipe.items[k].coeff * ref[k] for k in range(a, b))
            assert abs(T[t, s_idx] - want) <= 1e-8 * (b - a)
    # inputs really change from step to step
    assert not np.allclose(E[0], E[1])
