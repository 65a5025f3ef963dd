"""Precision sweep of the split path: the digit-slice count s (used for V, P_ab / P_ij and
Gamma alike) from the fewest slices to past the double-float floor, BF16 (9-bit digits)
and FP8 (5-bit digits), on

* the single fragment nocc=10 nvir=40 naux=150 (seed 0): energy error against the
  oracle and relative Frobenius errors of Gamma, P_ij, P_ab;
* the MBE3 batch of a 64-monomer, 40-bohr system (seed 0; dimers within 12 bohr,
  trimers with every pair within 10 bohr): the largest per-fragment energy difference to
  the plain FP64 path (itself checked against the oracle by the other GPU tests), the
  MBE3 total's difference, and fragments/s of the whole batch (all outputs, CUDA-graph
  replay timed with CUDA events) next to the FP64 path's.

Asserts that each added slice shrinks the error until the double-float floor, and that
the library's default slice counts meet 1e-8 Eh per fragment and 1e-9 relative on
Gamma / P.  Prints one JSON line with the table (run with -s to keep it).
"""
import json
import math

import numpy as np
import pytest
import torch

from oracle import oracle
from paper_2410_21888_gb300 import rimp2, synth

pytestmark = pytest.mark.gpu

VARIANTS = ([("bf16", s) for s in range(3, 9)] + [("fp8", s) for s in (6, 7, 8, 9, 10, 12)])


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _batch(system, frags, prec, opts, reps=3):
    eng = rimp2.Engine([system.fragment_dims(f) for f in frags], precision=prec,
                       want_epair=False, **opts)
    eng.set_inputs([system.fragment(f) for f in frags])
    eng.run()
    torch.cuda.synchronize()
    eng.check_status()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        eng.run()
    e1.record()
    torch.cuda.synchronize()
    E = eng.energy[:len(frags)].cpu().numpy().copy()
    ms = e0.elapsed_time(e1) / reps
    del eng
    torch.cuda.empty_cache()
    return ms, E


def test_precision_sweep():
    f0 = synth.fragment_inputs(10, 40, 150, seed=0)
    ref0 = oracle.fragment(f0.B, f0.eo, f0.ev)
    system = synth.MonomerSystem(n_monomers=64, box=40.0, seed=0)
    dimers, trimers = rimp2.mbe_polymers(system.centroids, 12.0, 10.0, "max")
    frags, coeff = rimp2.mbe_coefficients(system.n, dimers, trimers)
    ms64, E64 = _batch(system, frags, "fp64", {}, reps=1)
    mbe64 = math.fsum(float(c) * float(e) for c, e in zip(coeff, E64))
    rows = []
    for prec, s in VARIANTS + [("bf16", 0), ("fp8", 0)]:     # s = 0: library defaults
        opts = {} if s == 0 else {"slices_v": s, "slices_t": s, "slices_g": s}
        out = rimp2.energy_grad(f0.B, f0.eo, f0.ev, precision=prec, **opts)
        row = {"precision": prec, "slices": s or "default",
               "c0_abs_err_E_Eh": abs(float(out["energy"].item()) - ref0["energy"])}
        for k in ("gamma", "pij", "pab"):
            row[f"c0_rel_err_{k}"] = _rel(out[k].cpu().numpy(), ref0[k])
        del out
        ms, E = _batch(system, frags, prec, opts)
        row["c2_max_abs_fragment_diff_vs_fp64_Eh"] = float(np.max(np.abs(E - E64)))
        row["c2_mbe3_diff_vs_fp64_Eh"] = math.fsum(float(c) * float(e) for c, e in zip(coeff, E)) - mbe64
        row["c2_ms"] = ms
        row["c2_fragments_per_s"] = len(frags) / (ms * 1e-3)
        row["c2_speedup_vs_fp64"] = ms64 / ms
        rows.append(row)
    print(json.dumps({"fragments": len(frags), "fp64_ms": ms64, "fp64_mbe3_Eh": mbe64,
                      "rows": rows}))
    for prec in ("bf16", "fp8"):
        r = [x for x in rows if x["precision"] == prec and x["slices"] != "default"]
        g = [x["c0_rel_err_gamma"] for x in r]
        e = [x["c2_max_abs_fragment_diff_vs_fp64_Eh"] for x in r]
        # each slice buys bits until the double-float floor (~1e-12 relative, ~1e-10 Eh)
        for a, b in zip(g, g[1:]):
            assert b < a or b < 1e-11, (prec, g)
        for a, b in zip(e, e[1:]):
            assert b < a or b < 1e-9, (prec, e)
        d = [x for x in rows if x["precision"] == prec and x["slices"] == "default"][0]
        assert d["c0_abs_err_E_Eh"] <= 1e-8 and d["c2_max_abs_fragment_diff_vs_fp64_Eh"] <= 1e-8
        for k in ("gamma", "pij", "pab"):
            assert d[f"c0_rel_err_{k}"] <= 1e-9, (prec, k, d)
