"""Runs one fragment through the library a few times (for profiler captures).

  python -m paper_2410_21888_gb300.profile_case --nocc 24 --nvir 200 --naux 600 \
      --precision bf16 --calls 1

Seeded synthetic inputs; exits 0 after checking the device status.
"""
import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch  # noqa: E402

from paper_2410_21888_gb300 import rimp2, synth  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nocc", type=int, default=24)
    ap.add_argument("--nvir", type=int, default=200)
    ap.add_argument("--naux", type=int, default=600)
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp8", "fp64"])
    ap.add_argument("--calls", type=int, default=1)
    ap.add_argument("--slices-v", type=int, default=0, help="0: the library default")
    ap.add_argument("--slices-t", type=int, default=0, help="0: the library default")
    a = ap.parse_args()
    f = synth.fragment_inputs(a.nocc, a.nvir, a.naux, seed=0)
    eng = rimp2.Engine([f.B.shape], precision=a.precision, slices_v=a.slices_v,
                       slices_t=a.slices_t)
    eng.set_inputs([f])
    for _ in range(a.calls):
        eng.run()
    torch.cuda.synchronize()
    eng.check_status()
    print(f"E = {float(eng.energy[0]):.12f}  workspace {eng.workspace.numel() / 2**30:.2f} GiB")
    return 0


if __name__ == "__main__":
    sys.exit(main())
