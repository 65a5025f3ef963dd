"""Benchmark of the RI-MP2 energy + gradient-intermediate hot path on one GB300.

Workload: one large fragment, nocc=100, nvir=500, naux=1500 (seeded synthetic B and
orbital energies), energy + Gamma + P_ij + P_ab per step.  A step is one full pass of
the hot path.  Inputs (600 MB) and workspace (tens of GB) are far larger than L2, so no
flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision auto|fp64|bf16]
  python bench.py --impl reference ...   (the CPU oracle on a bounded sample)

Under torchrun each rank runs its own replica (weak scaling, no collective on the data
path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RI-MP2 energy+grad TFLOP/s and fragments/s on 1 GB300, vs plain FP64 at <=1e-8 Eh"
WORKLOAD = {"workload": "single fragment RI-MP2 energy+Gamma+P_ab+P_ij, nocc=100 nvir=500 "
                        "naux=1500, seed 0", "nocc": 100, "nvir": 500, "naux": 1500}
DIMS = (100, 500, 1500)
# dram__bytes_read.sum + dram__bytes_write.sum per launch at nocc=100 nvir=500
# naux=1500 (BF16 defaults), keyed by (precision, launch: V, P = P_ab / P_ij, G = Gamma),
# from an ncu capture of these two metrics alone on this fragment (one pass per launch,
# which a small-fragment capture showed first).  An entry is removed (traffic null)
# whenever its kernel or its launch's tile order changes, until it is captured again.
TRAFFIC_PER_LAUNCH = {("bf16", "G"): 96_830_000_000 + 1_890_000_000,
                      ("bf16", "P"): 133_130_000_000 + 27_020_000,
                      ("bf16", "V"): 10_790_000_000 + 10_180_000_000}


def flops(o, v, X):
    """2mnk count (V over i<=j, Gamma, P_ab, P_ij)."""
    return float(o * (o + 1) * v * v * X + 2 * o * o * v * v * X + 2 * o * o * v ** 3
                 + 2 * o ** 3 * v * v)


def fp64_peak():
    """FP64 throughput of this GPU measured in place by the library's test hook:
    CUDA-core DFMA and the FP64 tensor path (mma.sync m8n8k4), TFLOP/s."""
    import ctypes
    from paper_2410_21888_gb300 import rimp2
    f = rimp2.load().rimp2_testing_fp64_peak
    f.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]
    f.restype = ctypes.c_int
    out = {}
    for kind, name in ((0, "dfma_tflops"), (1, "dmma_tflops")):
        t = ctypes.c_double(0.0)
        out[name] = t.value if f(kind, ctypes.byref(t)) == 0 else None
    return out


def oracle_golden():
    """The oracle's full result for this fragment (seed 0), stored by
    tests/golden/make_c1_golden.py; None when absent."""
    p = os.path.join(ROOT, "tests", "golden", "c1_seed0.json")
    return json.load(open(p)) if os.path.exists(p) else None


def mbe3_leg(seed=0, reps=3):
    """The MBE3-shaped uneven batch: 64 monomers in a 40-bohr box (seed 0), dimers within
    12 bohr, trimers with every pair within 10 bohr; one plan per MBE level, its launch
    sequence captured once and replayed; inputs drawn on the device.  Split path (library
    defaults) timed over `reps` replays, the plain FP64 path once on the same inputs."""
    import numpy as np
    import torch
    from paper_2410_21888_gb300 import bench_mbe, rimp2, synth
    system = synth.MonomerSystem(n_monomers=64, box=40.0, seed=seed)
    rd, rt, rule = bench_mbe.CUTOFFS["stated"]
    dimers, trimers = rimp2.mbe_polymers(system.centroids, rd, rt, rule)
    frags, coeff = rimp2.mbe_coefficients(system.n, dimers, trimers)
    out = {"workload": f"MBE3 batch, 64 monomers (nocc 8..20, nvir 4 nocc, naux 3 (nocc+nvir)), "
                       f"40-bohr box, seed {seed}; dimers within {rd} bohr, trimers with every "
                       f"pair within {rt} bohr; energy + Gamma + P_ab + P_ij per fragment",
           "fragments": len(frags),
           "per_level": {lvl: sum(1 for f in frags if len(f) == lvl) for lvl in (1, 2, 3)}}
    E = {}
    for prec, r in (("bf16", reps), ("fp64", 1)):
        En = np.zeros(len(frags))
        tot_ms = tot_fl = 0.0
        for level in (1, 2, 3):
            idx = [k for k, f in enumerate(frags) if len(f) == level]
            if not idx:
                continue
            lf = [frags[k] for k in idx]
            res, en = bench_mbe.run_level(lf, system, prec, True, 120 << 30, r, seed)
            En[idx] = en
            tot_ms += res["ms"]
            tot_fl += sum(flops(*system.fragment_dims(f)) for f in lf)
        total = rimp2.mbe_combine(torch.as_tensor(En, device="cuda"),
                                  torch.as_tensor(coeff, dtype=torch.int32, device="cuda"))
        E[prec] = En
        out[prec] = {"ms": tot_ms, "fragments_per_s": len(frags) / (tot_ms * 1e-3),
                     "tflops_fp64_equivalent": tot_fl / (tot_ms * 1e-3) / 1e12,
                     "mbe3_energy_Eh": float(total.item()), "timed_replays": r}
    out["max_fragment_diff_vs_fp64_path_Eh"] = float(np.max(np.abs(E["bf16"] - E["fp64"])))
    out["mbe3_total_diff_vs_fp64_path_Eh"] = out["bf16"]["mbe3_energy_Eh"] - out["fp64"]["mbe3_energy_Eh"]
    out["speedup_fragments_per_s"] = out["bf16"]["fragments_per_s"] / out["fp64"]["fragments_per_s"]
    return out


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_baseline(B, eo, ev, max_seconds=25.0):
    """The oracle, as it stands, on a bounded sample of the workload: a slice of the
    second pair index k (each k is 1/nocc of the pairs), scaled to TFLOP/s."""
    from oracle import oracle
    o, v, X = B.shape
    nthr = oracle.threads()
    t0 = time.perf_counter()
    k = 0
    while k < o:
        oracle.fragment(B, eo, ev, k_range=(k, k + 1), nthreads=nthr)
        k += 1
        if time.perf_counter() - t0 > max_seconds:
            break
    dt = time.perf_counter() - t0
    val = flops(o, v, X) * k / o / dt / 1e12
    return {"value": val, "unit": "TFLOP/s", "cores": nthr, "kind": "oracle",
            "sample": f"pairs (i,k) for k in [0,{k}) of nocc={o} nvir={v} naux={X} "
                      f"(energy, Gamma, P_ij, P_ab contributions; {dt:.1f} s)",
            "seconds": dt, "k_done": k}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2410_21888_gb300 import synth
    o, v, X = DIMS
    f = synth.fragment_inputs(o, v, X, seed=0)
    vals = []
    for _ in range(max(args.warmup, 0)):
        cpu_baseline(f.B, f.eo, f.ev, max_seconds=2.0)
    cb = None
    for _ in range(args.steps):
        cb = cpu_baseline(f.B, f.eo, f.ev, max_seconds=max(5.0, 60.0 / max(args.steps, 1)))
        vals.append(cb["value"])
    value = statistics.median(vals)
    ms = flops(o, v, X) / (value * 1e12) * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(WORKLOAD, l2="CPU run"),
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cb["cores"],
                             "kind": "oracle", "sample": cb["sample"]},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def measure_e2e(eng, f, steps, barrier):
    """End to end through the public API: every step copies its inputs from pinned host
    memory and reads the energy back (device -> host); ms per step.  The inputs of step
    k+1 are copied host -> device into a staging buffer on a second stream while step k
    runs (a double-buffered input pool), then moved into the engine's pool on the
    compute stream before step k+1."""
    import numpy as np
    import torch
    pinned_B = torch.from_numpy(f.B.reshape(-1)).pin_memory()
    pinned_eps = torch.from_numpy(np.concatenate([f.eo, f.ev])).pin_memory()
    stream = torch.cuda.current_stream()
    copy_stream = torch.cuda.Stream()
    stage_B = torch.empty_like(eng.B[:pinned_B.numel()])
    stage_eps = torch.empty_like(eng.eps[:pinned_eps.numel()])
    nb, ne = pinned_B.numel(), pinned_eps.numel()

    def run_steps(n):
        copied, consumed = torch.cuda.Event(), torch.cuda.Event()
        copy_stream.wait_stream(stream)   # the first copy starts inside the timed region
        with torch.cuda.stream(copy_stream):
            stage_B.copy_(pinned_B, non_blocking=True)
            stage_eps.copy_(pinned_eps, non_blocking=True)
            copied.record(copy_stream)
        for k in range(n):
            stream.wait_event(copied)
            eng.B[:nb].copy_(stage_B, non_blocking=True)
            eng.eps[:ne].copy_(stage_eps, non_blocking=True)
            consumed.record(stream)
            if k + 1 < n:   # the next step's inputs, during this step
                copied = torch.cuda.Event()
                copy_stream.wait_event(consumed)
                with torch.cuda.stream(copy_stream):
                    stage_B.copy_(pinned_B, non_blocking=True)
                    stage_eps.copy_(pinned_eps, non_blocking=True)
                    copied.record(copy_stream)
                consumed = torch.cuda.Event()
            eng.run()
            float(eng.energy[0].item())   # device -> host read of the step's result

    run_steps(2)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    run_steps(steps)
    e1.record(stream)
    barrier()
    return e0.elapsed_time(e1) / steps, nb * 8 + ne * 8


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", "fp64", "bf16", "fp8"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--stage-k", type=int, default=0, choices=[0, 16, 32],
                    help="K per tensor-core pipeline stage (0: library default)")
    ap.add_argument("--n-tile", type=int, default=0, choices=[0, 48, 64, 80, 96])
    ap.add_argument("--slices-t", type=int, default=0,
                    help="slices of the P_ab / P_ij operands; 0: precision default (6 for bf16)")
    ap.add_argument("--slices-g", type=int, default=0,
                    help="slices of the Gamma operands; 0: as --slices-t")
    ap.add_argument("--no-mbe3", action="store_true",
                    help="skip the MBE3 uneven-batch leg (reported under \"mbe3\")")
    ap.add_argument("--fp64-steps", type=int, default=1,
                    help="timed steps of the plain FP64 path reported beside the split path")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2410_21888_gb300 import rimp2, synth

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    o, v, X = DIMS
    F = flops(o, v, X)
    f = synth.fragment_inputs(o, v, X, seed=0)

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    precs = ["bf16", "fp64"] if args.precision == "auto" else [args.precision]
    results = {}
    e2e_ms = e2e_h2d = e2e_clocks = None
    for prec in precs:
        def make(profile):
            return rimp2.Engine([(o, v, X)], precision=prec, device=dev, profile_stages=profile,
                                stage_k=args.stage_k, n_tile=args.n_tile,
                                slices_t=args.slices_t, slices_g=args.slices_g)
        # the timed engine records no stage events: its steps run back to back
        eng = make(False)
        eng.set_inputs([f])
        head_run = prec == precs[0] or args.precision != "auto"
        steps = args.steps if head_run else args.fp64_steps
        warm = args.warmup if head_run else 1
        for _ in range(warm):
            eng.run()
        barrier()
        eng.check_status()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            barrier()
            e0.record(stream)
            for _ in range(steps):
                eng.run()
            e1.record(stream)
            barrier()
        eng.check_status()
        ms = e0.elapsed_time(e1) / steps
        if ws > 1:
            t = torch.tensor([ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        st = eng.plan.stats()
        if head_run:   # end to end right after the device-timed loop, same engine
            e2e_steps = max(1, min(args.steps, 5))
            with ClockSampler(local) as clk_e2e:
                e2e_ms, e2e_h2d = measure_e2e(eng, f, e2e_steps, barrier)
            e2e_clocks = clk_e2e.summary()
        # stage split from a second engine that records events between the stages (its own
        # untimed steps: the event records and the per-step read of their times would slow
        # the timed loop)
        prof = make(True)
        prof.set_inputs([f])
        prof.run()
        stage = [0.0, 0.0, 0.0, 0.0]
        launch = [0.0, 0.0]
        nprof = max(1, min(steps, 3))
        for _ in range(nprof):
            prof.run()
            pst = prof.plan.stats()        # waits for the step; reads its stage timers
            for k in range(4):
                stage[k] += pst.stage_ms[k] / nprof
            for k in range(2):
                launch[k] += pst.launch_ms[k] / nprof
        del prof
        torch.cuda.empty_cache()
        results[prec] = {"ms": ms, "steps": steps, "warmup": warm, "engine": eng,
                         "clocks": clk.summary(), "launches": st.launches_per_call,
                         "energy": float(eng.energy[0].item()),
                         "energy_os": float(eng.energy_os[0].item()), "stage_ms": stage,
                         "launch_ms": launch, "slices": list(st.slices),
                         "tc_flops": list(st.tc_flops)}
        if not head_run:
            del eng
    if not results:
        raise RuntimeError("no precision path available")
    head = precs[0] if precs[0] in results else list(results)[0]
    R = results[head]
    eng = R["engine"]
    if e2e_ms is None:
        e2e_ms, e2e_h2d = measure_e2e(eng, f, max(1, min(args.steps, 5)), barrier)


    peaks, peak_src = load_peaks()
    value = ws * F / (R["ms"] * 1e-3) / 1e12
    sm, lm = R["stage_ms"], R["launch_ms"]
    F_v = float(o * (o + 1) * v * v * X)
    F_g = float(2 * o * o * v * v * X)
    F_p = F - F_v - F_g
    sv = stt = sg = 0
    if head == "fp64":
        peak = fp64_peak()
        k = 3 if sm[3] >= sm[1] else 1
        Fk = F - F_v if k == 3 else F_v
        ach = Fk / (sm[k] * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": peak["dfma_tflops"], "unit": "TFLOP/s",
                "frac": ach / peak["dfma_tflops"], "traffic": None,
                "kernel": "k_gemm_f64 (" + ("Gamma/P_ab/P_ij" if k == 3 else "V") + ")",
                "peak_source": "DFMA throughput measured in this run (rimp2_testing_fp64_peak)",
                "fp64_peaks_tflops": peak}
    else:
        fp8 = head == "fp8"
        sv, stt, sg = R["slices"]
        prod = {"V": sv * (sv + 1) // 2, "P": stt * (stt + 1) // 2, "G": sg * (sg + 1) // 2}
        tc = R["tc_flops"]
        # launches of one step: V (stage 1), the P_ab / P_ij launch (with Gamma when it has
        # their slice count) and the separate Gamma launch (stage 3)
        launches = {"V": (sm[1], F_v * prod["V"], tc[0], F_v, f"V, {prod['V']} slice products")}
        if sg != stt:
            launches["P"] = (lm[0], F_p * prod["P"], tc[1], F_p,
                             f"P_ab/P_ij, {prod['P']} slice products")
            launches["G"] = (lm[1], F_g * prod["G"], tc[2], F_g,
                             f"Gamma, {prod['G']} slice products")
        else:
            launches["P"] = (lm[0], (F_p + F_g) * prod["P"], tc[1], F_p + F_g,
                             f"Gamma/P_ab/P_ij, {prod['P']} slice products")
        kname = max(launches, key=lambda n: launches[n][0])
        t_ms, alg_fl, tc_fl, f64_fl, desc = launches[kname]
        # FP8 dense peak: the measured BF16 peak x the nominal FP8:BF16 ratio (4.5 / 2.25)
        peak = float(peaks["bf16_tflops_sustained"]) * (2.0 if fp8 else 1.0)
        ach = alg_fl / (t_ms * 1e-3) / 1e12
        issued = tc_fl / (t_ms * 1e-3) / 1e12
        roof = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": TRAFFIC_PER_LAUNCH.get((head, kname)),
                "kernel": f"k_split_gemm ({desc})", "launch_ms": t_ms,
                "achieved_convention": "algorithmic 2mnk FLOPs of the launch's contractions x "
                                       "digit products / launch time",
                "issued_tflops": issued, "issued_frac": issued / peak,
                "issued_convention": "tensor-core FLOPs the launch issues (2 x 128 x n_tile x K "
                                     "per computed tile, padding included, skipped symmetric "
                                     "tiles excluded) / launch time",
                "peak_source": f"{peak_src} bf16 dense sustained (kernel inside a long step)"
                               + (" x 2 (nominal fp8:bf16)" if fp8 else ""),
                "fp64_equivalent_tflops": f64_fl / (t_ms * 1e-3) / 1e12,
                "launches": {n: {"ms": l[0],
                                 "algorithmic_tflops": l[1] / (l[0] * 1e-3) / 1e12 if l[0] > 0 else None,
                                 "issued_tflops": l[2] / (l[0] * 1e-3) / 1e12 if l[0] > 0 else None}
                             for n, l in launches.items()}}
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws,
        "steps": R["steps"], "warmup": R["warmup"], "ms_per_step": R["ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if head == "fp64" else head,
        "data": "synthetic",
        "config": dict(WORKLOAD, precision=head if head == "fp64" else
                       (f"{head} split, {sv} slices for V, {stt} for Gamma/P" if sg == stt else
                        f"{head} split, {sv} slices for V, {stt} for P_ab/P_ij, {sg} for Gamma"),
                       digit_bits=None if head == "fp64" else (5 if head == "fp8" else 9),
                       l2="inputs larger than L2 (B 600 MB, workspace >> 129 MB); no flush",
                       fragments_per_s=ws * 1000.0 / R["ms"], energy_Eh=R["energy"]),
        "roofline": roof,
        "stage_ms": {"slice_check": sm[0], "V_gemm": sm[1], "amplitudes_energy": sm[2],
                     "gamma_p_gemm": sm[3]},
        "e2e": {"value": ws * F / (e2e_ms * 1e-3) / 1e12, "unit": "TFLOP/s",
                "h2d_bytes_per_step": int(e2e_h2d),
                "d2h_bytes_per_step": 8, "ms_per_step": e2e_ms, "clocks": e2e_clocks},
        "gpu_launches": int(R["launches"] * R["steps"]),
        "clocks": R["clocks"],
        "paths": {p: {"ms_per_step": r["ms"], "tflops": F / (r["ms"] * 1e-3) / 1e12,
                      "fragments_per_s": 1000.0 / r["ms"], "energy_Eh": r["energy"],
                      "stage_ms": r["stage_ms"]}
                  for p, r in results.items()},
        "peaks": {"source": peak_src},
    }
    if "fp64" in results and head != "fp64":
        line["config"]["energy_diff_vs_fp64_path_Eh"] = R["energy"] - results["fp64"]["energy"]
    gold = oracle_golden()
    if gold is not None:
        for p_, r_ in results.items():
            line["paths"][p_]["energy_diff_vs_oracle_Eh"] = r_["energy"] - gold["energy"]
            line["paths"][p_]["energy_os_diff_vs_oracle_Eh"] = r_["energy_os"] - gold["energy_os"]
        line["config"]["energy_diff_vs_oracle_Eh"] = R["energy"] - gold["energy"]
    if head != "fp64":
        line["fp64_peaks_tflops"] = fp64_peak()
    if rank == 0 and not args.no_mbe3 and args.precision in ("auto", "bf16"):
        del eng, R, results
        torch.cuda.empty_cache()
        line["mbe3"] = mbe3_leg()
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = {k: val for k, val in cpu_baseline(f.B, f.eo, f.ev).items()
                                if k in ("value", "unit", "cores", "kind", "sample")}
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
