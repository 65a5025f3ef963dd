"""Split-precision accuracy and speed on the single-fragment workload for several seeds.

  python -m paper_2410_21888_gb300.bench_seeds [--dims 100 500 1500] [--seeds 1 2 3 4]

Per seed: the BF16 split path and the FP64 path on the same seeded inputs; the energy
difference (Eh), the relative Frobenius differences of Gamma, P_ij, P_ab, and the device
time per call of each path (CUDA events, after one warm-up call).  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch  # noqa: E402

from paper_2410_21888_gb300 import rimp2, synth  # noqa: E402


def timed(eng, reps):
    eng.run()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(reps):
        eng.run()
    t1.record()
    torch.cuda.synchronize()
    eng.check_status()
    return t0.elapsed_time(t1) / reps


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", type=int, nargs=3, default=[100, 500, 1500])
    ap.add_argument("--seeds", type=int, nargs="+", default=[1, 2, 3, 4])
    a = ap.parse_args()
    o, v, X = a.dims
    rows = []
    for seed in a.seeds:
        f = synth.fragment_inputs(o, v, X, seed=seed)
        out = {}
        for prec, reps in (("bf16", 3), ("fp64", 1)):
            eng = rimp2.Engine([(o, v, X)], precision=prec, want_epair=False)
            eng.set_inputs([f])
            ms = timed(eng, reps)
            out[prec] = {"ms": ms, "energy": float(eng.energy[0].item()),
                         **{k: getattr(eng, k).clone() for k in ("gamma", "pij", "pab")}}
            del eng
            torch.cuda.empty_cache()
        b, r = out["bf16"], out["fp64"]
        rel = {k: float(torch.linalg.norm(b[k] - r[k]) / torch.linalg.norm(r[k]))
               for k in ("gamma", "pij", "pab")}
        rows.append({"seed": seed, "bf16_ms": b["ms"], "fp64_ms": r["ms"],
                     "energy_Eh": r["energy"], "energy_diff_Eh": b["energy"] - r["energy"],
                     "rel_frobenius": rel})
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    print(json.dumps({"workload": f"single fragment nocc={o} nvir={v} naux={X}", "seeds": rows}))


if __name__ == "__main__":
    main()
