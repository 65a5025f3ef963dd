"""Throughput of the gradient step after the densities (Gamma^P, L', L'', Z-vector D_ai)
on one GB300, FP64.

  python -m paper_2410_21888_gb300.bench_zvector [--dims 100 500 1500] [--steps 3]

The fragment's Gamma, P_ij and P_ab come from the hot path (rimp2_energy_grad, BF16 split)
on the seeded full-MO inputs; the step is then timed alone with CUDA events on its stream
(inputs resident in HBM, B alone 4.3 GB at the default size: no L2 flush needed).  FLOPs
are the 2mnk counts of the step's contractions:
  Gamma^P 2 ov X^2; L' and L'' 2 o n v X each; right-hand side 2 o^3 X + 2 o^2 v X
  + 4 o v^2 X; per conjugate-gradient iteration 4 o^2 v X.
Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch  # noqa: E402

from paper_2410_21888_gb300 import rimp2, synth  # noqa: E402

FP64_PEAK_TFLOPS = 1.199   # measured DFMA throughput of this GB300


def step_flops(o, v, X, iters, with_jmh=True):
    n = o + v
    f = 2.0 * o * n * v * X * 2
    f += 2.0 * o ** 3 * X + 2.0 * o * o * v * X + 4.0 * o * v * v * X
    f += iters * 4.0 * o * o * v * X
    if with_jmh:
        f += 2.0 * o * v * X * X
    return f


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", type=int, nargs=3, default=[100, 500, 1500])
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args()
    o, v, X = a.dims
    f = synth.full_mo_inputs(o, v, X, seed=a.seed)
    hot = rimp2.energy_grad(f.frag.B, f.frag.eo, f.frag.ev, precision="bf16")
    gamma = hot["gamma"].reshape(o, v, X)
    pij, pab = hot["pij"].reshape(o, o), hot["pab"].reshape(v, v)
    Bf = torch.as_tensor(f.Bf).cuda()
    eps = torch.as_tensor(f.eps).cuda()
    jmh = torch.as_tensor(f.jmh).cuda()
    ws = torch.empty(rimp2.zvector_workspace_size(o, v, X), dtype=torch.uint8, device="cuda")
    for _ in range(a.warmup):
        out = rimp2.zvector(Bf, eps, gamma, pij, pab, jmh=jmh, workspace=ws)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    for _ in range(a.steps):
        t0.record()
        out = rimp2.zvector(Bf, eps, gamma, pij, pab, jmh=jmh, workspace=ws, sync=False)
        t1.record()
        torch.cuda.synchronize()
        ms.append(t0.elapsed_time(t1))
    info = out["info"].cpu().tolist()
    iters = int(info[0])
    F = step_flops(o, v, X, iters)
    best = min(ms)
    tf = F / (best * 1e-3) / 1e12
    print(json.dumps({
        "workload": f"gradient step after the densities, nocc={o} nvir={v} naux={X}, seed "
                    f"{a.seed}: Gamma^P, L', L'', Z-vector D_ai (FP64)",
        "ms": best, "ms_all": ms, "cg_iterations": iters, "rel_residual": info[1],
        "flops": F, "tflops": tf, "fp64_peak_tflops": FP64_PEAK_TFLOPS,
        "frac_of_fp64_peak": tf / FP64_PEAK_TFLOPS,
        "note": "FLOPs: contractions only (2mnk); row and column sums and the CG vector "
                "updates (O(ov X) each) are not counted"}))


if __name__ == "__main__":
    main()
