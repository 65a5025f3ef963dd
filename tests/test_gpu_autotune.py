"""In-situ autotuning (the analogue of the paper's runtime GEMM variant selection, Sec.
"GEMM runtime auto-tuning"): the first calls of a plan each run one trial, timed with
CUDA events between the stages; later calls use the fastest.  Split paths trial the tile
shapes first (n_tile x K per stage, per launch: V, P_ab / P_ij, Gamma), then the
contraction-stage variants with each launch's fastest shape; FP64 trials its split-K
variants.  The choice is cached per (precision, slices, shapes) key.  Every trial
computes the same quantities.
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


@pytest.mark.parametrize("precision,nvar,tol", [("bf16", 4, 1e-9), ("fp8", 4, 1e-9),
                                                ("fp64", 3, 1e-11)])
def test_trials_then_best_and_identical_results(precision, nvar, tol):
    frags = _frags()
    cache = os.path.join(tempfile.mkdtemp(), "tune.txt")
    eng = rimp2.Engine([f.B.shape for f in frags], precision=precision, autotune=True,
                       autotune_cache=cache)
    eng.set_inputs(frags)
    ntrials = eng.plan.stats().tune_trials
    if precision == "fp64":
        assert ntrials == nvar
    else:   # several tile shapes, then the other nvar - 1 variants
        assert ntrials > nvar
    outs = []
    shapes = set()
    for call in range(ntrials + 2):
        eng.run()
        torch.cuda.synchronize()
        eng.check_status()
        st = eng.plan.stats()
        shapes.add(tuple(st.n_tile) + tuple(st.stage_k))
        outs.append([{k: t.detach().cpu().numpy().copy() for k, t in eng.views(i).items()}
                     for i in range(len(frags))])
    st = eng.plan.stats()
    assert st.tune_done == 1
    ms = [st.tune_ms[v] for v in range(nvar)]
    assert all(m > 0 for m in ms)
    assert st.tune_variant == int(np.argmin(ms))
    if precision != "fp64":
        assert len(shapes) > 2          # the trials did run different tile shapes
        for nt, bk in zip(st.n_tile, st.stage_k):
            assert nt in (32, 48, 64, 80, 96) and bk in (16, 32, 64)
    for i, f in enumerate(frags):
        ref = oracle.fragment(f.B, f.eo, f.ev)
        for o in outs:
            assert abs(float(o[i]["energy"]) - ref["energy"]) <= 1e-8
            for k in ("pij", "pab", "gamma"):
                err = np.linalg.norm(o[i][k] - ref[k]) / np.linalg.norm(ref[k])
                assert err <= tol, (precision, k, err)
    rec = open(cache).read().split()
    assert rec[1] == str(st.tune_variant) and len(rec) == 5
    # a second plan with the same key starts from the cached variant and shapes, no trials
    eng2 = rimp2.Engine([f.B.shape for f in frags], precision=precision, autotune=True,
                        autotune_cache=cache)
    st2 = eng2.plan.stats()
    assert st2.tune_done == 1 and st2.tune_variant == st.tune_variant
    assert list(st2.n_tile) == list(st.n_tile) and list(st2.stage_k) == list(st.stage_k)
    eng2.set_inputs(frags)
    eng2.run()
    torch.cuda.synchronize()
    eng2.check_status()
    assert np.allclose(eng2.energy[:len(frags)].cpu().numpy(),
                       eng.energy[:len(frags)].cpu().numpy(), rtol=1e-12, atol=1e-9)
