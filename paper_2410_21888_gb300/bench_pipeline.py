"""Throughput of asynchronous MBE3 time steps (Sec. "Asynchronous time steps") against
step-by-step execution on one GPU.

  python -m paper_2410_21888_gb300.bench_pipeline [--systems 2] [--steps 4] [--waves 8]

Systems: 64 monomers in a 40-bohr box each by default (seeds 0, 1, ...), dimers within 12 bohr,
trimers with every pair within 10 bohr.  Every step draws fresh B blocks on the GPU
(per-block, per-step seeds; same geometry).  All outputs (energy, Gamma, P) per
fragment.  One warm-up pass captures the wave graphs; then each mode runs every step
once.  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import numpy as np  # noqa: E402

from paper_2410_21888_gb300 import pipeline, synth  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--systems", type=int, default=2)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--waves", type=int, default=8)
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp8", "fp64"])
    ap.add_argument("--workspace-gb", type=float, default=160.0)
    ap.add_argument("--monomers", type=int, default=64)
    ap.add_argument("--box", type=float, default=40.0)
    a = ap.parse_args()
    systems = [synth.MonomerSystem(n_monomers=a.monomers, box=a.box, seed=s)
               for s in range(a.systems)]
    t0 = time.perf_counter()
    pipe = pipeline.AsyncMBE3(systems, 12.0, 10.0, "max", n_waves=a.waves, precision=a.precision,
                              workspace_budget=int(a.workspace_gb * 2 ** 30), inputs="device")
    pipe.prepare_steps(a.steps)
    setup_s = time.perf_counter() - t0
    pipe.run("sync")                       # warm-up: captures every wave graph
    flop = sum(it.cost for it in pipe.items) * a.steps
    rep = {"workload": f"{a.systems} x MBE3 system ({a.monomers} monomers, {a.box:g}-bohr box, "
                       f"dimers <= 12 bohr, "
                       f"trimers max <= 10 bohr), {a.steps} time steps, fresh B per step",
           "fragments_per_step": len(pipe.items), "waves": len(pipe.waves),
           "precision": a.precision, "setup_s": setup_s,
           "wave_fragments": [len(w) for w in pipe.waves],
           "wave_dependencies": [len(d) for d in pipe.deps]}
    res = {}
    for mode in ("sync", "async"):
        E, T, ms = pipe.run(mode)
        res[mode] = (E.cpu().numpy(), T.cpu().numpy())
        rep[mode] = {"ms": ms, "ms_per_step": ms / a.steps,
                     "fragments_per_s": len(pipe.items) * a.steps / (ms * 1e-3),
                     "tflops": flop / (ms * 1e-3) / 1e12}
    rep["async_speedup"] = rep["sync"]["ms"] / rep["async"]["ms"]
    rep["max_abs_diff_fragment_Eh"] = float(np.max(np.abs(res["sync"][0] - res["async"][0])))
    rep["mbe3_totals_Eh"] = res["async"][1].tolist()
    print(json.dumps(rep))


if __name__ == "__main__":
    main()
