"""MBE3 driver (Eq. mbe3): polymer formation with distance cutoffs, one engine plan per
MBE level (each level's fragments of uneven size run in the same grouped launches under
one CUDA graph), and the inclusion-exclusion total combined on the device.

Host work here is bookkeeping only: polymer lists and coefficients come from the C ABI
(include/rimp2_mbe.h), fragment inputs from the seeded synthetic system.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import rimp2


@dataclass
class MBE3Result:
    energy: float
    fragments: list
    coeff: np.ndarray
    frag_energy: np.ndarray
    level_ms: dict = field(default_factory=dict)
    level_counts: dict = field(default_factory=dict)
    dimers: np.ndarray = None
    trimers: np.ndarray = None


class MBE3:
    """MBE3 over a synth.MonomerSystem (or any object with .n, .centroids and
    .fragment(monomers) -> object with B, eo, ev)."""

    def __init__(self, system, r_dimer: float, r_trimer: float, trimer_rule: str = "max",
                 precision: str = "bf16", want_grad: bool = True, max_workspace_bytes: int = 0,
                 **plan_opts):
        self.system = system
        self.r_dimer, self.r_trimer, self.rule = r_dimer, r_trimer, trimer_rule
        self.precision = precision
        self.want_grad = want_grad
        self.max_ws = max_workspace_bytes
        self.plan_opts = plan_opts

    def polymers(self):
        return rimp2.mbe_polymers(self.system.centroids, self.r_dimer, self.r_trimer, self.rule)

    def run(self, trimer_keep=None, timing: bool = True) -> MBE3Result:
        """trimer_keep: optional boolean mask over the trimer list (learned screen)."""
        dimers, trimers = self.polymers()
        if trimer_keep is not None:
            trimers = trimers[np.asarray(trimer_keep, dtype=bool)]
        frags, coeff = rimp2.mbe_coefficients(self.system.n, dimers, trimers)
        energies = torch.zeros(len(frags), dtype=torch.float64, device="cuda")
        res = MBE3Result(0.0, frags, coeff, None, dimers=dimers, trimers=trimers)
        for level in (1, 2, 3):
            idx = [k for k, f in enumerate(frags) if len(f) == level]
            res.level_counts[level] = len(idx)
            if not idx:
                continue
            inputs = [self.system.fragment(frags[k]) for k in idx]
            eng = rimp2.Engine([x.B.shape for x in inputs], precision=self.precision,
                               want_gamma=self.want_grad, want_p=self.want_grad,
                               want_epair=False, max_workspace_bytes=self.max_ws,
                               **self.plan_opts)
            eng.set_inputs(inputs)
            eng.run()                     # first call captures the level's graph
            torch.cuda.synchronize()
            eng.check_status()
            if timing:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                eng.run()                 # replay, timed
                e1.record()
                torch.cuda.synchronize()
                res.level_ms[level] = e0.elapsed_time(e1)
            energies[torch.tensor(idx, device="cuda")] = eng.energy[:len(idx)]
            del eng
        c = torch.as_tensor(coeff, dtype=torch.int32, device="cuda")
        total = rimp2.mbe_combine(energies, c)
        torch.cuda.synchronize()
        res.energy = float(total.item())
        res.frag_energy = energies.cpu().numpy()
        return res
