"""Learned trimer screen: an MLP (include/rimp2_mlp.h) trained on trimer corrections
dE_IJK that the engine itself computed predicts log10|dE_IJK| for candidate trimers;
trimers predicted below a threshold are skipped, a random sample of the skipped ones is
recomputed by the plain method as the audit, and the plain method stays the fallback
(screen=None).

Host code here is bookkeeping (polymer lists, index tables, minibatch permutations);
features, labels, gradients, optimiser steps and predictions run in library kernels.
"""
from __future__ import annotations

import time
import zlib
from dataclasses import dataclass

import numpy as np
import torch

from . import rimp2

TRIMER_SIGNS = (1, -1, -1, -1, 1, 1, 1)
DIMER_SIGNS = (1, -1, -1)


class DeviceBlockInputs:
    """Fragment inputs restricted from one global B, with each (occ-owner, vir-owner,
    aux-owner) block drawn on the GPU from its own seed, so every fragment containing a
    block sees the same values (MBE differences cancel exactly as on the host
    generator).  Same distribution and block scaling as synth.MonomerSystem."""

    def __init__(self, system, step: int = 0):
        self.s = system
        self.step = int(step)     # time step: fresh block seeds, same geometry
        self.gen = torch.Generator(device="cuda")

    def _seed(self, I, J, K):
        key = [self.s.seed, 97, I, J, K] + ([self.step] if self.step else [])
        return zlib.crc32(np.array(key, dtype=np.int64).tobytes())

    def fill(self, eng, frags):
        s = self.s
        for k, f in enumerate(frags):
            o, v, X = eng.dims[k]
            b, e, _, _ = eng.offsets[k]
            Bf = eng.B[b:b + o * v * X].view(o, v, X)
            m = list(f)
            oo = np.concatenate([[0], np.cumsum(s.nocc[m])])
            vo = np.concatenate([[0], np.cumsum(s.nvir[m])])
            xo = np.concatenate([[0], np.cumsum(s.naux[m])])
            for p, I in enumerate(m):
                for q, J in enumerate(m):
                    for r, K in enumerate(m):
                        self.gen.manual_seed(self._seed(I, J, K))
                        blk = Bf[oo[p]:oo[p + 1], vo[q]:vo[q + 1], xo[r]:xo[r + 1]]
                        blk.normal_(0.0, s.sigma, generator=self.gen)
                        sc = s.block_scale((I, J, K))
                        if sc != 1.0:
                            blk.mul_(sc)
            eo = np.concatenate([s.eps(I)[0] for I in m])
            ev = np.concatenate([s.eps(I)[1] for I in m])
            eng.eps[e:e + o].copy_(torch.from_numpy(eo))
            eng.eps[e + o:e + o + v].copy_(torch.from_numpy(ev))


def fragment_energies(system, frags, precision="bf16", slices_v=8, device_inputs=True,
                      chunk_bytes=48 << 30, ws_budget=64 << 30):
    """Energies of `frags` (tuples of monomer ids), energy only, one plan per chunk of
    same-order fragments; returns (device FP64 tensor, seconds of GPU work)."""
    out = torch.zeros(len(frags), dtype=torch.float64, device="cuda")
    filler = DeviceBlockInputs(system) if device_inputs else None
    gpu_s = 0.0
    order = sorted(range(len(frags)), key=lambda k: (len(frags[k]), frags[k]))
    chunk, bytes_ = [], 0
    pending = []

    def flush(idx):
        nonlocal gpu_s
        if not idx:
            return
        fl = [frags[k] for k in idx]
        eng = rimp2.Engine([system.fragment_dims(f) for f in fl], precision=precision,
                           want_gamma=False, want_p=False, want_epair=False,
                           max_workspace_bytes=ws_budget, slices_v=slices_v)
        if filler is not None:
            filler.fill(eng, fl)
        else:
            eng.set_inputs([system.fragment(f) for f in fl])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        eng.run()
        e1.record()
        torch.cuda.synchronize()
        eng.check_status()
        gpu_s += e0.elapsed_time(e1) * 1e-3
        out[torch.as_tensor(idx, device="cuda")] = eng.energy[:len(idx)]
        del eng
        torch.cuda.empty_cache()

    for k in order:
        o, v, X = system.fragment_dims(frags[k])
        nb = o * v * X * 8
        if chunk and (bytes_ + nb > chunk_bytes or len(frags[chunk[0]]) != len(frags[k])):
            flush(chunk)
            chunk, bytes_ = [], 0
        chunk.append(k)
        bytes_ += nb
    flush(chunk)
    return out, gpu_s


@dataclass
class TrimerSet:
    trimers: np.ndarray          # [nt, 3]
    feats: torch.Tensor          # [nt, 9] FP32 device
    labels: torch.Tensor         # [nt] FP32 log10|dE_IJK|
    dE: torch.Tensor             # [nt] FP64 dE_IJK
    trimer_seconds: float        # GPU time spent on the trimer energies
    lower_seconds: float         # GPU time on monomers and pairs


def _index(frags):
    return {f: k for k, f in enumerate(frags)}


def trimer_set(system, r_trimer, rule="two_pairs", precision="bf16", slices_v=8,
               device_inputs=True, trimers=None) -> TrimerSet:
    """Candidate trimers (or the given list), their exact-by-the-method corrections, and
    features built from the dimer corrections of their sub-pairs."""
    if trimers is None:
        _, trimers = rimp2.mbe_polymers(system.centroids, 0.0, r_trimer, rule)
    trimers = np.asarray(trimers, dtype=np.int32).reshape(-1, 3)
    mons = [(i,) for i in range(system.n)]
    pairs = sorted({(int(a), int(b)) for t in trimers for a, b in ((t[0], t[1]), (t[0], t[2]), (t[1], t[2]))})
    tris = [tuple(int(x) for x in t) for t in trimers]
    low = mons + pairs
    E_low, s_low = fragment_energies(system, low, precision, slices_v, device_inputs)
    E_tri, s_tri = fragment_energies(system, tris, precision, slices_v, device_inputs)
    E = torch.cat([E_low, E_tri])
    ix = _index(low + tris)
    dterms = torch.tensor([[ix[p], ix[(p[0],)], ix[(p[1],)]] for p in pairs] or
                          np.zeros((0, 3)), dtype=torch.int32)
    dde = rimp2.mbe_corrections(E, dterms, DIMER_SIGNS) if len(pairs) else \
        torch.zeros(0, dtype=torch.float64, device="cuda")
    table = torch.zeros((system.n, system.n), dtype=torch.float64, device="cuda")
    if len(pairs):
        pa = torch.as_tensor(np.array(pairs), device="cuda", dtype=torch.long)
        table[pa[:, 0], pa[:, 1]] = dde
        table[pa[:, 1], pa[:, 0]] = dde
    tterms = torch.tensor([[ix[t], ix[(t[0], t[1])], ix[(t[0], t[2])], ix[(t[1], t[2])],
                            ix[(t[0],)], ix[(t[1],)], ix[(t[2],)]] for t in tris] or
                          np.zeros((0, 7)), dtype=torch.int32)
    dE, lab = rimp2.mbe_corrections(E, tterms, TRIMER_SIGNS, want_log=True)
    cen = torch.as_tensor(system.centroids, dtype=torch.float64, device="cuda")
    nocc = torch.as_tensor(system.nocc, dtype=torch.int32, device="cuda")
    tri_d = torch.as_tensor(trimers, dtype=torch.int32, device="cuda")
    feats = rimp2.screen_features(cen, nocc, tri_d, table)
    return TrimerSet(trimers, feats, lab, dE, s_tri, s_low)


class TrimerScreen:
    """The MLP parameters (FP32 master on the device, BF16 in the forward pass) and its
    Adam state; feature standardisation constants fixed from the training set."""

    def __init__(self, seed: int = 0):
        rng = np.random.default_rng(seed)
        parts = []
        for (o, i) in ((64, 9), (64, 64), (64, 64), (1, 64)):
            parts.append(rng.normal(0.0, np.sqrt(2.0 / i), size=o * i))
            parts.append(np.zeros(o))
        theta = np.concatenate(parts).astype(np.float32)
        assert theta.size == rimp2.MLP_PARAMS
        self.master = torch.as_tensor(theta, device="cuda")
        self.m = torch.zeros_like(self.master)
        self.v = torch.zeros_like(self.master)
        self.t = 0
        self.mean = torch.zeros(9, dtype=torch.float32, device="cuda")
        self.std = torch.ones(9, dtype=torch.float32, device="cuda")

    def set_normalization(self, feats: torch.Tensor):
        f = feats.double().cpu().numpy()
        self.mean = torch.as_tensor(f.mean(0), dtype=torch.float32, device="cuda")
        self.std = torch.as_tensor(f.std(0) + 1e-3, dtype=torch.float32, device="cuda")

    def fit(self, feats, labels, epochs=200, batch=512, lr=2e-3, seed=0, rows=None):
        """Adam on minibatches of `rows` (device int32 row indices; default all rows)."""
        if rows is None:
            rows = torch.arange(feats.shape[0], dtype=torch.int32, device="cuda")
        rows_h = rows.cpu().numpy()
        n = len(rows_h)
        rng = np.random.default_rng(seed)
        hist = []
        for ep in range(epochs):
            perm = torch.as_tensor(rows_h[rng.permutation(n)].astype(np.int32), device="cuda")
            tot = 0.0
            for s0 in range(0, n, batch):
                idx = perm[s0:s0 + batch]
                g, loss = rimp2.mlp_grad(self.master, feats, labels, idx, idx.numel(),
                                         self.mean, self.std)
                self.t += 1
                rimp2.mlp_adam(self.master, g, self.m, self.v, self.t, lr)
                tot += float(loss.item()) * idx.numel()
            hist.append(tot / n)
        return hist

    def predict(self, feats):
        return rimp2.mlp_predict(self.master, feats, self.mean, self.std)

    def loss(self, feats, labels, rows=None):
        n = feats.shape[0] if rows is None else rows.numel()
        idx = None if rows is None else rows.to(torch.int32)
        _, l = rimp2.mlp_grad(self.master, feats, labels, idx, n, self.mean, self.std)
        return float(l.item())


def select_skips(pred_log10, threshold=1e-7, margin_decades=1.0, budget_Eh=None, safety=10.0):
    """Trimers to skip: predicted |dE| below threshold x 10^-margin, taken in ascending
    order of the prediction while the predicted skipped sum stays within
    budget_Eh / safety (no budget: the threshold rule alone)."""
    pred = np.asarray(pred_log10, dtype=np.float64)
    cand = pred < (np.log10(threshold) - margin_decades)
    if budget_Eh is None:
        return cand
    order = np.argsort(pred)
    csum = np.cumsum(10.0 ** pred[order])
    take = order[(csum <= budget_Eh / safety) & cand[order]]
    skip = np.zeros(len(pred), dtype=bool)
    skip[take] = True
    return skip


def screen_and_audit(system, screen: TrimerScreen, ts: TrimerSet, threshold=1e-7,
                     margin_decades=1.0, audit_fraction=0.05, seed=0, audit_precision="fp64",
                     budget_Eh=None, safety=10.0):
    """Applies the screen to the candidate set `ts` (whose exact corrections are known, so
    the effect on the MBE3 total is measured directly) and recomputes a random
    `audit_fraction` of the skipped trimers with the plain method."""
    pred = screen.predict(ts.feats).cpu().numpy()
    skip = select_skips(pred, threshold, margin_decades, budget_Eh, safety)
    dE = ts.dE.cpu().numpy()
    nt = len(dE)
    res = {"candidates": int(nt), "skipped": int(skip.sum()), "kept": int(nt - skip.sum()),
           "threshold_Eh": threshold, "margin_decades": margin_decades,
           "budget_Eh": budget_Eh, "budget_safety": safety,
           "predicted_skipped_sum_Eh": float(np.sum(10.0 ** pred[skip])),
           "skipped_sum_Eh": float(np.sum(dE[skip])),
           "skipped_abs_sum_Eh": float(np.sum(np.abs(dE[skip]))),
           "max_skipped_abs_Eh": float(np.max(np.abs(dE[skip]))) if skip.any() else 0.0,
           "missed_above_threshold": int(np.sum(skip & (np.abs(dE) >= threshold)))}
    # time saved: the trimer-energy GPU time scales with the trimers computed
    fl = np.array([_flops(system, t) for t in ts.trimers])
    res["trimer_flop_fraction_skipped"] = float(fl[skip].sum() / max(fl.sum(), 1.0))
    res["trimer_seconds_all"] = ts.trimer_seconds
    res["trimer_seconds_saved_est"] = ts.trimer_seconds * res["trimer_flop_fraction_skipped"]
    # audit: recompute a held-out random sample of the skipped trimers with the plain method
    sk = np.nonzero(skip)[0]
    rng = np.random.default_rng(seed + 12345)
    nj = int(np.ceil(audit_fraction * len(sk))) if len(sk) else 0
    if nj:
        pick = np.sort(rng.choice(sk, nj, replace=False))
        js = trimer_set(system, None, precision=audit_precision, device_inputs=True,
                        trimers=ts.trimers[pick]) if audit_precision == "fp64" else None
        jd = js.dE.cpu().numpy()
        res["audit_count"] = int(nj)
        res["audit_max_abs_Eh"] = float(np.max(np.abs(jd)))
        res["audit_mean_abs_Eh"] = float(np.mean(np.abs(jd)))
        res["audit_est_skipped_abs_sum_Eh"] = float(np.mean(np.abs(jd)) * len(sk))
        res["audit_vs_method_max_diff_Eh"] = float(np.max(np.abs(jd - dE[pick])))
        res["audit_precision"] = audit_precision
    return res, skip


def _prefix_within(order, dE, budget_Eh):
    """Length of the longest prefix of `order` whose skipped absolute corrections sum to at
    most budget_Eh (a bound on the change of the MBE3 total)."""
    return int(np.searchsorted(np.cumsum(np.abs(dE[order])), budget_Eh, side="right"))


def compare_with_distance_cutoff(system, ts: TrimerSet, pred_log10, budget_Eh=1e-6):
    """The method without the screen is a distance cutoff (the paper's reference-monomer
    cutoff study in Sec. "Molecular Fragmentation"): a trimer is computed when its
    centroid distances are within R_cut.  For each ordering of the candidates, the
    trimers are skipped in that order while the sum of their exact |corrections| (a bound
    on the change of the MBE3 total) stays within budget_Eh, i.e. each rule gets its best
    threshold in hindsight:
      distance_max:  farthest first by the largest pairwise centroid distance (R_cut on
                     the max rule);
      distance_two:  farthest first by the second-largest distance (R_cut on the two-pair
                     rule that formed the candidates);
      learned:       smallest predicted |dE_IJK| first;
      exact:         smallest exact |dE_IJK| first (the most any ordering can skip).
    Returns, per ordering, the trimers skipped, their share of the trimer FLOPs and the
    distance of the last skipped trimer (the equivalent R_cut)."""
    dE = ts.dE.cpu().numpy()
    c = np.asarray(system.centroids)
    t = np.asarray(ts.trimers)
    d = np.stack([np.linalg.norm(c[t[:, 0]] - c[t[:, 1]], axis=1),
                  np.linalg.norm(c[t[:, 0]] - c[t[:, 2]], axis=1),
                  np.linalg.norm(c[t[:, 1]] - c[t[:, 2]], axis=1)], axis=1)
    d.sort(axis=1)
    fl = np.array([_flops(system, x) for x in t])
    orders = {"distance_max": np.argsort(-d[:, 2], kind="stable"),
              "distance_two": np.argsort(-d[:, 1], kind="stable"),
              "learned": np.argsort(np.asarray(pred_log10, dtype=np.float64), kind="stable"),
              "exact": np.argsort(np.abs(dE), kind="stable")}
    out = {"budget_Eh": budget_Eh, "candidates": int(len(dE))}
    for name, order in orders.items():
        k = _prefix_within(order, dE, budget_Eh)
        sk = order[:k]
        r = {"skipped": k, "trimer_flop_fraction_skipped": float(fl[sk].sum() / max(fl.sum(), 1.0)),
             "skipped_sum_Eh": float(dE[sk].sum())}
        if name.startswith("distance") and k:
            col = 2 if name == "distance_max" else 1
            r["equivalent_r_cut_bohr"] = float(d[order[k - 1], col])
        out[name] = r
    best_d = max(out["distance_max"]["skipped"], out["distance_two"]["skipped"])
    out["learned_gain_over_best_distance"] = out["learned"]["skipped"] - best_d
    return out


def _flops(system, t):
    o, v, X = system.fragment_dims(t)
    return float(o * (o + 1) * v * v * X)
