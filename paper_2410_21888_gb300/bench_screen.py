"""Learned trimer screen at full size.

  python -m paper_2410_21888_gb300.bench_screen [--train-systems 4] [--n-candidates 20000]

Training: candidate trimers (two of three centroid distances within the screening
radius) of 64-monomer, 40-bohr systems with nocc ~ U{8..20} (seeds 100, 101, ...),
randomly subsampled to about 5,000 trimers; labels log10|dE_IJK| from the engine
(split path, 8 slices for V: FP64-level energies), network trained by the library
kernels (90/10 train/validation split).
Screening: a 256-monomer, 80-bohr box; the candidate radius (two-pair rule) is the
smallest 0.5-bohr step giving at least --n-candidates trimers.  Every candidate's
correction is computed (to measure the exact effect of the screen on the MBE3 total);
two rules are reported: the per-trimer rule (skip if the predicted |dE| < threshold/10)
and the budgeted rule (skip the smallest predictions first while their predicted sum
stays below budget/safety, by default 1e-6 Eh / 2); 5% of the skipped ones are recomputed with
the FP64 path as the audit.  The method without the screen, a distance cutoff, is
compared at the same error budget: the best cutoff in hindsight on the max-pair and on
the two-pair distance, the learned ordering with the same hindsight stop, and the exact
ordering that bounds them all.  Inputs are drawn on the GPU from per-block
seeds (device_inputs).  Prints one JSON line.
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

from paper_2410_21888_gb300 import rimp2, screen, synth  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train-systems", type=int, default=4)
    ap.add_argument("--train-target", type=int, default=5000)
    ap.add_argument("--n-candidates", type=int, default=20000)
    ap.add_argument("--threshold", type=float, default=1e-7)
    ap.add_argument("--margin", type=float, default=1.0)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--budget", type=float, default=1e-6)
    ap.add_argument("--safety", type=float, default=2.0)
    a = ap.parse_args()
    t_all = time.perf_counter()
    rep = {"workload": "learned trimer screen: train on C2-style trimers, screen a "
                       "256-monomer 80-bohr box", "threshold_Eh": a.threshold}
    # ---- screening geometry first: the training candidates use the same radius
    big = synth.MonomerSystem(n_monomers=256, box=80.0, seed=7)
    r = 16.0
    while True:
        _, tri = rimp2.mbe_polymers(big.centroids, 0.0, r, "two_pairs")
        if len(tri) >= a.n_candidates or r > 40:
            break
        r += 0.5
    rep["candidate_radius_bohr"] = r
    # ---- training set
    sets, n = [], 0
    t0 = time.perf_counter()
    per = max(1, a.train_target // a.train_systems)
    rng = np.random.default_rng(1)
    for k in range(a.train_systems):
        s = synth.MonomerSystem(n_monomers=64, box=40.0, seed=100 + k)
        _, cand = rimp2.mbe_polymers(s.centroids, 0.0, r, "two_pairs")
        if len(cand) > per:
            cand = cand[np.sort(rng.choice(len(cand), per, replace=False))]
        sets.append(screen.trimer_set(s, None, trimers=cand))
        n += len(sets[-1].trimers)
    feats = torch.cat([x.feats for x in sets])
    labels = torch.cat([x.labels for x in sets])
    rep["train_trimers"] = int(feats.shape[0])
    rep["train_label_seconds"] = time.perf_counter() - t0
    sc = screen.TrimerScreen(seed=0)
    sc.set_normalization(feats)
    ntr = int(0.9 * feats.shape[0])
    perm = np.random.default_rng(0).permutation(feats.shape[0]).astype(np.int32)
    tr = torch.as_tensor(perm[:ntr], device="cuda")
    va = torch.as_tensor(perm[ntr:], device="cuda")
    t0 = time.perf_counter()
    sc.fit(feats, labels, epochs=a.epochs, batch=512, lr=2e-3, rows=tr)
    torch.cuda.synchronize()
    rep["train_seconds"] = time.perf_counter() - t0
    rep["train_rmse_decades"] = float(np.sqrt(sc.loss(feats, labels, tr)))
    rep["val_rmse_decades"] = float(np.sqrt(sc.loss(feats, labels, va)))
    t0 = time.perf_counter()
    ts = screen.trimer_set(big, r, "two_pairs")
    rep["candidate_set_seconds"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    feats_t = ts.feats
    pred = sc.predict(feats_t)
    torch.cuda.synchronize()
    rep["predict_seconds"] = time.perf_counter() - t0
    rep["test_rmse_decades"] = float(np.sqrt(np.mean((pred.cpu().numpy() - ts.labels.cpu().numpy()) ** 2)))
    res, _ = screen.screen_and_audit(big, sc, ts, threshold=a.threshold, margin_decades=a.margin)
    rep["threshold_rule"] = res
    resb, _ = screen.screen_and_audit(big, sc, ts, threshold=a.threshold, margin_decades=a.margin,
                                      budget_Eh=a.budget, safety=a.safety)
    rep["budget_rule"] = resb
    rep["budget_rule_within_1e-6_of_unscreened"] = bool(abs(resb["skipped_sum_Eh"]) <= 1e-6)
    # the method without the screen: the best distance cutoff at the same error budget,
    # next to the learned ordering, and the self-budgeted rule at several safety factors
    rep["vs_distance_cutoff"] = screen.compare_with_distance_cutoff(big, ts, pred.cpu().numpy(),
                                                                    a.budget)
    rep["budget_rule_by_safety"] = {}
    for sf in (1.0, 2.0, 5.0, 10.0):
        rs, _ = screen.screen_and_audit(big, sc, ts, threshold=a.threshold,
                                        margin_decades=a.margin, budget_Eh=a.budget, safety=sf,
                                        audit_fraction=0.05 if sf == a.safety else 0.0)
        rep["budget_rule_by_safety"][str(sf)] = {
            k: rs[k] for k in ("skipped", "trimer_flop_fraction_skipped", "skipped_sum_Eh",
                               "predicted_skipped_sum_Eh")}
    dE = np.abs(ts.dE.cpu().numpy())
    rep["exact_dE_quantiles_Eh"] = [float(x) for x in np.quantile(dE, [0.01, 0.1, 0.25, 0.5, 0.75, 0.9])]
    srt = np.sort(dE)
    rep["oracle_best_skip_count_within_budget"] = int(np.searchsorted(np.cumsum(srt), a.budget))
    rep["total_seconds"] = time.perf_counter() - t_all
    print(json.dumps(rep))


if __name__ == "__main__":
    main()
