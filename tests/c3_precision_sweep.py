"""Precision sweep: the single fragment nocc=10 nvir=40 naux=150 (seed 0) and the MBE3 batch
of a 64-monomer, 40-bohr system (seed 0; dimers within 12 bohr, trimers with every pair
within 10 bohr: 256 fragment energies) through the FP64 path, the BF16 split with
s = 3..8 slices and the FP8 split with s = 6..16 slices (s for V and for Gamma/P).

Per variant: the largest per-fragment |E - E_oracle| over the batch and the error of the
MBE3 total (oracle energies computed here on the host cores), for the single fragment
also the relative Frobenius errors of Gamma, P_ij and P_ab, and the throughput of the
256-fragment batch (all outputs; CUDA-graph replays timed with CUDA events) in
fragments/s next to the FP64 path's.

  python tests/c3_precision_sweep.py [--reps 3]

Needs a GPU.  Test infrastructure: it runs the oracle.  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import numpy as np  # noqa: E402
import torch  # noqa: E402

from oracle import oracle  # noqa: E402
from paper_2410_21888_gb300 import rimp2, synth  # noqa: E402

VARIANTS = ([("fp64", 0)] + [("bf16", s) for s in range(3, 9)]
            + [("fp8", s) for s in range(6, 17)])


def rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def batch_run(system, frags, prec, s, reps):
    opts = {} if prec == "fp64" else {"slices_v": s, "slices_t": s}
    eng = rimp2.Engine([system.fragment_dims(f) for f in frags], precision=prec,
                       want_epair=False, max_workspace_bytes=int(100e9), **opts)
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
    eng.check_status()
    ms = e0.elapsed_time(e1) / reps
    E = eng.energy[:len(frags)].cpu().numpy().copy()
    del eng
    torch.cuda.empty_cache()
    return ms, E


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args()
    nthr = oracle.threads()
    rep = {"workload": "precision sweep: fragment (10, 40, 150) seed 0; MBE3 batch 64 monomers, "
                       "40-bohr box, seed 0, dimers <= 12 bohr, trimers max <= 10 bohr",
           "oracle_threads": nthr}
    # single fragment: full outputs from the oracle
    f0 = synth.fragment_inputs(10, 40, 150, seed=0)
    ref0 = oracle.fragment(f0.B, f0.eo, f0.ev, nthreads=nthr)
    # MBE3 batch: oracle energies of every fragment
    system = synth.MonomerSystem(n_monomers=64, box=40.0, seed=0)
    dimers, trimers = rimp2.mbe_polymers(system.centroids, 12.0, 10.0, "max")
    frags, coeff = rimp2.mbe_coefficients(system.n, dimers, trimers)
    t0 = time.perf_counter()
    Eref = np.array([oracle.fragment(x.B, x.eo, x.ev, want=(), nthreads=nthr)["energy"]
                     for x in (system.fragment(f) for f in frags)])
    rep["oracle_seconds"] = time.perf_counter() - t0
    rep["fragments"] = len(frags)
    mbe_ref = math.fsum(float(c) * float(e) for c, e in zip(coeff, Eref))
    rep["mbe3_oracle_Eh"] = mbe_ref
    rows = []
    fp64_rate = None
    for prec, s in VARIANTS:
        opts = {} if prec == "fp64" else {"slices_v": s, "slices_t": s}
        out = rimp2.energy_grad(f0.B, f0.eo, f0.ev, precision=prec, **opts)
        row = {"precision": prec, "slices": s,
               "c0_abs_err_E_Eh": abs(float(out["energy"].item()) - ref0["energy"]),
               "c0_rel_err_gamma": rel(out["gamma"].cpu().numpy(), ref0["gamma"]),
               "c0_rel_err_pij": rel(out["pij"].cpu().numpy(), ref0["pij"]),
               "c0_rel_err_pab": rel(out["pab"].cpu().numpy(), ref0["pab"])}
        del out
        ms, E = batch_run(system, frags, prec, s, a.reps)
        row["c2_max_abs_fragment_err_Eh"] = float(np.max(np.abs(E - Eref)))
        row["c2_mbe3_err_Eh"] = math.fsum(float(c) * float(e) for c, e in zip(coeff, E)) - mbe_ref
        row["c2_ms"] = ms
        row["c2_fragments_per_s"] = len(frags) / (ms * 1e-3)
        if prec == "fp64":
            fp64_rate = row["c2_fragments_per_s"]
        row["c2_speedup_vs_fp64"] = row["c2_fragments_per_s"] / fp64_rate if fp64_rate else None
        rows.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    rep["variants"] = rows
    print(json.dumps(rep))


if __name__ == "__main__":
    main()
