"""Writes the full-size oracle fixture of the single large fragment
(nocc=100, nvir=500, naux=1500, seed 0): c1_seed0.json (scalars) and c1_seed0.npz
(arrays).

Calls only oracle/ (the plain FP64 C loops over the Appendix definitions: RI integrals of
Eq. MP2_ints, amplitudes X^ab_ij, the closed-shell energy, Gamma^Q_ia in the MO-B basis,
D^MP2_ij, D^MP2_ab, and the opposite-spin part of the energy).  The inputs come from the
seeded generator in paper_2410_21888_gb300/synth.py, which holds no arithmetic of the
method.  Nothing here touches a GPU.

Stored: the energy, its opposite-spin part, every pair energy e_ij, all of P_ij and P_ab,
the Frobenius norm of Gamma per occupied index i, and 512 Gamma elements at seeded
(i, a, Q).  The whole of Gamma (600 MB) is not stored.

Run (about 15-25 minutes on 8 cores):  python tests/golden/make_c1_golden.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle  # noqa: E402
from paper_2410_21888_gb300 import synth  # noqa: E402

DIMS = (100, 500, 1500)
SEED = 0
N_GAMMA_SAMPLES = 512
SAMPLE_SEED = 20241021


def gamma_sample_indices(o, v, X, n=N_GAMMA_SAMPLES, seed=SAMPLE_SEED):
    """Seeded (i, a, Q) triples at which Gamma is stored (also used by the tests)."""
    rng = np.random.default_rng(seed)
    return np.stack([rng.integers(0, o, n), rng.integers(0, v, n), rng.integers(0, X, n)],
                    axis=1).astype(np.int64)


def main():
    o, v, X = DIMS
    f = synth.fragment_inputs(o, v, X, seed=SEED)
    nthr = oracle.threads()
    t0 = time.time()
    r = oracle.fragment(f.B, f.eo, f.ev, nthreads=nthr)
    t1 = time.time()
    e_os, e_ss = oracle.spin_components(f.B, f.eo, f.ev, nthreads=nthr)
    t2 = time.time()
    idx = gamma_sample_indices(o, v, X)
    g = r["gamma"]
    meta = {
        "citation": "Appendix: RI integrals (Eq. MP2_ints), amplitudes X^ab_ij, Gamma^P_ia "
                    "(MO-B basis), D^MP2_ij, D^MP2_ab; closed-shell energy "
                    "E = sum X^ab_ij [2(ia|jb) - (ib|ja)]; opposite-spin part "
                    "E_OS = sum X^ab_ij (ia|jb) (SCS-MP2, Introduction)",
        "generator": "tests/golden/make_c1_golden.py via oracle/oracle.py "
                     "(oracle/rimp2_oracle.c, plain FP64 loops, Neumaier-compensated "
                     "cross-pair energy sums)",
        "inputs": {"nocc": o, "nvir": v, "naux": X, "seed": SEED,
                   "generator": "paper_2410_21888_gb300.synth.fragment_inputs"},
        "energy": r["energy"],
        "energy_os": e_os,
        "energy_ss": e_ss,
        "gamma_frobenius": float(np.linalg.norm(g)),
        "gamma_samples": {"n": N_GAMMA_SAMPLES, "seed": SAMPLE_SEED},
        "oracle_threads": nthr,
        "oracle_seconds": {"fragment": round(t1 - t0, 1), "spin_components": round(t2 - t1, 1)},
    }
    np.savez_compressed(
        os.path.join(HERE, "c1_seed0.npz"),
        epair=r["epair"], pij=r["pij"], pab=r["pab"],
        gamma_row_norm=np.sqrt(np.einsum("iaq,iaq->i", g, g)),
        gamma_idx=idx, gamma_val=g[idx[:, 0], idx[:, 1], idx[:, 2]])
    with open(os.path.join(HERE, "c1_seed0.json"), "w") as fh:
        json.dump(meta, fh, indent=1)
        fh.write("\n")
    print(json.dumps(meta, indent=1))


if __name__ == "__main__":
    main()
