"""In-situ autotuning of the contraction stage (the analogue of the paper's runtime GEMM
variant selection, Sec. "GEMM runtime auto-tuning"): the first calls of a plan each run
one variant, timed with CUDA events; later calls use the fastest; the choice is cached
per (precision, slices, shapes) key.  Every variant computes the same quantities.
"""
import os
import tempfile

import numpy as np
import pytest
import torch

from oracle import oracle
from paper_2410_21888_gb300 import rimp2, synth

pytestmark = pytest.mark.gpu


def _frags():
    s = synth.MonomerSystem(n_monomers=6, box=12.0, seed=5, nocc_range=(2, 5))
    return [s.fragment(p) for p in [(0,), (1, 2), (0, 3, 4), (5,)]]


@pytest.mark.parametrize("precision,nvar,tol", [("bf16", 4, 1e-9), ("fp64", 3, 1e-11)])
def test_trials_then_best_variant_and_identical_results(precision, nvar, tol):
    frags = _frags()
    cache = os.path.join(tempfile.mkdtemp(), "tune.txt")
    eng = rimp2.Engine([f.B.shape for f in frags], precision=precision, autotune=True,
                       autotune_cache=cache)
    eng.set_inputs(frags)
    outs = []
    for call in range(nvar + 2):
        eng.run()
        torch.cuda.synchronize()
        eng.check_status()
        outs.append([{k: t.detach().cpu().numpy().copy() for k, t in eng.views(i).items()}
                     for i in range(len(frags))])
    st = eng.plan.stats()
    assert st.tune_done == 1
    ms = [st.tune_ms[v] for v in range(nvar)]
    assert all(m > 0 for m in ms)
    assert st.tune_variant == int(np.argmin(ms))
    for i, f in enumerate(frags):
        ref = oracle.fragment(f.B, f.eo, f.ev)
        for o in outs:
            for k in ("pij", "pab", "gamma"):
                err = np.linalg.norm(o[i][k] - ref[k]) / np.linalg.norm(ref[k])
                assert err <= tol, (precision, k, err)
    assert open(cache).read().split()[1] == str(st.tune_variant)
    # a second plan with the same key starts from the cached variant, no trials
    eng2 = rimp2.Engine([f.B.shape for f in frags], precision=precision, autotune=True,
                        autotune_cache=cache)
    st2 = eng2.plan.stats()
    assert st2.tune_done == 1 and st2.tune_variant == st.tune_variant
