"""Throughput of the engine on MBE3-shaped uneven batches (64 monomers, 40-bohr box).

  python -m paper_2410_21888_gb300.bench_mbe --cutoffs stated --precision both
  python -m paper_2410_21888_gb300.bench_mbe --cutoffs matched --precision bf16 --device-inputs

stated:  dimers within 12 bohr, trimers with every pair within 10 bohr
matched: dimers within 16 bohr, trimers with two of three pairs within 15 bohr (about 300
         dimers and 1,200-1,400 trimers, the batch size of the uneven-batch workload)

One plan per MBE level: every fragment of a level runs in the same grouped persistent
launches, captured once into a CUDA graph and replayed for the timed run.  With
--device-inputs the fragment B tensors are drawn on the GPU (same distribution and
inter-monomer block scaling as the host generator, different random stream); use it for
throughput on large batches.  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import numpy as np  # noqa: E402
import torch  # noqa: E402

from paper_2410_21888_gb300 import rimp2, synth  # noqa: E402

CUTOFFS = {"stated": (12.0, 10.0, "max"), "matched": (16.0, 15.0, "two_pairs")}


def flops(o, v, X):
    return float(o * (o + 1) * v * v * X + 2 * o * o * v * v * X + 2 * o * o * v ** 3
                 + 2 * o ** 3 * v * v)


def fill_device_inputs(eng, system, frags, gen):
    for k, f in enumerate(frags):
        o, v, X = eng.dims[k]
        b, e, _, _ = eng.offsets[k]
        Bf = eng.B[b:b + o * v * X].view(o, v, X)
        Bf.normal_(0.0, system.sigma, generator=gen)
        m = list(f)
        oo = np.concatenate([[0], np.cumsum(system.nocc[m])])
        vo = np.concatenate([[0], np.cumsum(system.nvir[m])])
        xo = np.concatenate([[0], np.cumsum(system.naux[m])])
        for p, I in enumerate(m):
            for q, J in enumerate(m):
                for r, K in enumerate(m):
                    sc = system.block_scale((I, J, K))
                    if sc != 1.0:
                        Bf[oo[p]:oo[p + 1], vo[q]:vo[q + 1], xo[r]:xo[r + 1]].mul_(sc)
        eo = np.concatenate([system.eps(I)[0] for I in m])
        ev = np.concatenate([system.eps(I)[1] for I in m])
        eng.eps[e:e + o].copy_(torch.from_numpy(eo))
        eng.eps[e + o:e + o + v].copy_(torch.from_numpy(ev))


def run_level(frags, system, precision, device_inputs, ws_budget, reps, seed, asm_out=None,
              coeff=None, accumulate=False):
    eng = rimp2.Engine([system.fragment_dims(f) for f in frags], precision=precision,
                       want_epair=False, max_workspace_bytes=ws_budget)
    if device_inputs:
        gen = torch.Generator(device="cuda")
        gen.manual_seed(seed)
        fill_device_inputs(eng, system, frags, gen)
    else:
        eng.set_inputs([system.fragment(f) for f in frags])
    t0 = time.perf_counter()
    eng.run()                                   # capture + first run
    torch.cuda.synchronize()
    eng.check_status()
    first_s = time.perf_counter() - t0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        eng.run()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    st = eng.plan.stats()
    energies = eng.energy[:len(frags)].cpu().numpy().copy()
    out = {"fragments": len(frags), "ms": ms, "first_call_s": first_s, "waves": st.waves,
           "launches_per_call": st.launches_per_call, "tiles_per_call": st.tiles_per_call}
    if asm_out is not None:
        # MBE3 assembly of this level's Gamma / P into the system arrays (added to the
        # previous levels'), timed after one untimed pass on scratch outputs
        offs = eng.offsets
        asm = rimp2.MBEAssembly(system.nocc, system.nvir, system.naux, frags, coeff,
                                [o[0] for o in offs], [o[2] for o in offs], [o[3] for o in offs])
        g_lvl, p_lvl, q_lvl = asm.outputs()
        asm.run(eng.gamma, eng.pij, eng.pab, g_lvl, p_lvl, q_lvl)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record()
        asm.run(eng.gamma, eng.pij, eng.pab, g_lvl, asm_out[1], asm_out[2], accumulate=accumulate)
        a1.record()
        torch.cuda.synchronize()
        n_in = sum(o * v * x + o * o + v * v for o, v, x in eng.dims)
        out["assembly_ms"] = a0.elapsed_time(a1)
        out["assembly_gamma_sys_elems"] = int(asm.gamma_elems)
        out["assembly_gb_moved"] = 8.0 * (n_in + asm.gamma_elems + 2 * (asm.o_total ** 2 + asm.v_total ** 2)) / 1e9
        del asm, g_lvl, p_lvl, q_lvl
    del eng
    torch.cuda.empty_cache()
    return out, energies


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--cutoffs", default="stated", choices=list(CUTOFFS))
    ap.add_argument("--precision", default="both", choices=["bf16", "fp64", "both"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--device-inputs", action="store_true")
    ap.add_argument("--workspace-gb", type=float, default=120.0)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--assemble", action="store_true",
                    help="also time the MBE3 assembly of Gamma / P over the system (bf16 path)")
    a = ap.parse_args()
    system = synth.MonomerSystem(n_monomers=64, box=40.0, seed=a.seed)
    rd, rt, rule = CUTOFFS[a.cutoffs]
    dimers, trimers = rimp2.mbe_polymers(system.centroids, rd, rt, rule)
    frags, coeff = rimp2.mbe_coefficients(system.n, dimers, trimers)
    precs = ["bf16", "fp64"] if a.precision == "both" else [a.precision]
    report = {"workload": f"MBE3 batch, 64 monomers, 40-bohr box, seed {a.seed}, cutoffs "
                          f"{a.cutoffs} (dimers <= {rd} bohr, trimers {rule} <= {rt} bohr)",
              "dimers_kept": int(len(dimers)), "trimers_kept": int(len(trimers)),
              "fragments": len(frags), "inputs": "device" if a.device_inputs else "host",
              "paths": {}}
    all_E = {}
    for prec in precs:
        levels, E = {}, np.zeros(len(frags))
        tot_ms, tot_fl = 0.0, 0.0
        for level in (1, 2, 3):
            idx = [k for k, f in enumerate(frags) if len(f) == level]
            if not idx:
                continue
            lf = [frags[k] for k in idx]
            fl = sum(flops(*system.fragment_dims(f)) for f in lf)
            asm_out = None
            if a.assemble and prec == "bf16":
                if level == 1:
                    O, V = int(np.sum(system.nocc)), int(np.sum(system.nvir))
                    asm_state = (None, torch.zeros((O, O), dtype=torch.float64, device="cuda"),
                                 torch.zeros((V, V), dtype=torch.float64, device="cuda"))
                asm_out = asm_state
            r, en = run_level(lf, system, prec, a.device_inputs, int(a.workspace_gb * 2**30),
                              a.reps if prec == "bf16" else 1, a.seed, asm_out=asm_out,
                              coeff=np.asarray(coeff)[idx], accumulate=level > 1)
            E[idx] = en
            r["tflop"] = fl / 1e12
            r["tflops"] = fl / (r["ms"] * 1e-3) / 1e12
            r["fragments_per_s"] = len(lf) / (r["ms"] * 1e-3)
            levels[level] = r
            tot_ms += r["ms"]
            tot_fl += fl
        total = rimp2.mbe_combine(torch.as_tensor(E, device="cuda"),
                                  torch.as_tensor(coeff, dtype=torch.int32, device="cuda"))
        all_E[prec] = E
        report["paths"][prec] = {"levels": levels, "ms": tot_ms, "tflops": tot_fl / (tot_ms * 1e-3) / 1e12,
                                 "fragments_per_s": len(frags) / (tot_ms * 1e-3),
                                 "mbe3_energy_Eh": float(total.item())}
    if len(all_E) == 2:
        d = np.abs(all_E["bf16"] - all_E["fp64"])
        report["bf16_vs_fp64_max_abs_fragment_error_Eh"] = float(d.max())
        report["bf16_vs_fp64_mbe3_diff_Eh"] = (report["paths"]["bf16"]["mbe3_energy_Eh"]
                                              - report["paths"]["fp64"]["mbe3_energy_Eh"])
        report["speedup_fragments_per_s"] = (report["paths"]["bf16"]["fragments_per_s"]
                                             / report["paths"]["fp64"]["fragments_per_s"])
    print(json.dumps(report))


if __name__ == "__main__":
    main()
