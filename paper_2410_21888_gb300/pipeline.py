"""Asynchronous MBE3 time steps on one GPU (Sec. "Asynchronous time steps").

The polymers of a time step are taken in the order of the paper's priority queue: first
by the smallest distance of one of their monomers to a reference monomer at an extremity
of the system (here: the smallest x coordinate), then by decreasing size (2mnk cost).
The ordered list is cut into waves of about equal cost.  Each wave is one engine plan:
all its fragments, of mixed MBE levels, run in the grouped launches replayed from one
CUDA graph.

A monomer is complete for step t when every step-t wave holding one of its polymers has
finished.  A wave of step t+1 may start once every monomer of each of its polymers is
complete for step t.  On one GPU this becomes a static pipeline: even and odd steps run
on two streams, each stream with its own set of wave plans and workspaces, and CUDA
events carry the dependencies.
- "sync": step t+1 waits for the whole of step t.
- "async": each wave of step t+1 waits only for the step-t waves it depends on (and, on
  its own stream, for the step t-1 use of its plan).  The start of step t+1 then fills
  the tail of step t.
Both modes compute the same numbers.  The MBE3 total of each step and system is combined
on the device (compensated FP64).

Host code is bookkeeping: polymer lists and coefficients come from the C ABI, waves and
dependencies are index sets, inputs are drawn per step by the seeded generators.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import rimp2
from .screen import DeviceBlockInputs


def fragment_cost(o: int, v: int, X: int) -> float:
    return float(o * (o + 1) * v * v * X + 2 * o * o * v * v * X + 2 * o * o * v ** 3
                 + 2 * o ** 3 * v * v)


@dataclass
class Item:
    system: int
    monomers: tuple
    coeff: int
    dist: float
    cost: float


def priority_order(items):
    """Indices of `items` in the paper's priority-queue order (distance to the reference
    monomer, then decreasing size)."""
    return sorted(range(len(items)), key=lambda k: (items[k].dist, -items[k].cost, k))


def cut_waves(order, costs, n_waves: int):
    """Contiguous pieces of `order` with about equal total cost (at least one item each)."""
    n_waves = max(1, min(n_waves, len(order)))
    total = float(sum(costs[k] for k in order))
    waves, cur, acc = [], [], 0.0
    for pos, k in enumerate(order):
        cur.append(k)
        acc += costs[k]
        left_items = len(order) - pos - 1
        left_waves = n_waves - len(waves) - 1
        if left_waves > 0 and (acc >= total * (len(waves) + 1) / n_waves or left_items == left_waves):
            waves.append(cur)
            cur = []
    if cur:
        waves.append(cur)
    return waves


def wave_dependencies(items, waves):
    """deps[j]: the waves of the previous step that hold a polymer sharing a monomer with
    a polymer of wave j (those must finish before wave j of the next step starts)."""
    holder = {}
    for j, w in enumerate(waves):
        for k in w:
            for m in items[k].monomers:
                holder.setdefault((items[k].system, m), set()).add(j)
    deps = []
    for w in waves:
        d = set()
        for k in w:
            for m in items[k].monomers:
                d |= holder[(items[k].system, m)]
        deps.append(sorted(d))
    return deps


class AsyncMBE3:
    def __init__(self, systems, r_dimer: float, r_trimer: float, rule: str = "max",
                 n_waves: int = 8, precision: str = "bf16", want_grad: bool = True,
                 workspace_budget: int = 160 * 2 ** 30, inputs: str = "device"):
        self.systems = list(systems)
        self.precision = precision
        self.inputs = inputs
        items = []
        self.coeff = []
        self.sys_slices = []
        for s_idx, sysm in enumerate(self.systems):
            d, t = rimp2.mbe_polymers(sysm.centroids, r_dimer, r_trimer, rule)
            frags, coeff = rimp2.mbe_coefficients(sysm.n, d, t)
            ref = int(np.argmin(sysm.centroids[:, 0]))
            start = len(items)
            for f, c in zip(frags, coeff):
                f = tuple(int(x) for x in f)
                dist = min(sysm.distance(m, ref) for m in f)
                items.append(Item(s_idx, f, int(c), dist, fragment_cost(*sysm.fragment_dims(f))))
            self.sys_slices.append((start, len(items)))
        self.items = items
        self.order = priority_order(items)
        self.waves = cut_waves(self.order, [it.cost for it in items], n_waves)
        self.deps = wave_dependencies(items, self.waves)
        per_engine = int(workspace_budget // (2 * len(self.waves)))
        self.engines = [[rimp2.Engine([self.systems[items[k].system].fragment_dims(items[k].monomers)
                                       for k in w], precision=precision, want_gamma=want_grad,
                                      want_p=want_grad, want_epair=False,
                                      max_workspace_bytes=per_engine)
                         for w in self.waves] for _ in range(2)]
        self.coeff_dev = torch.as_tensor([it.coeff for it in items], dtype=torch.int32,
                                         device="cuda")
        self.wave_index = [torch.as_tensor(w, dtype=torch.int64, device="cuda") for w in self.waves]
        self.streams = [torch.cuda.Stream(), torch.cuda.Stream()]
        self.step_inputs = []

    # ---------------------------------------------------------------- inputs
    def prepare_steps(self, steps: int):
        """Draws the inputs of `steps` time steps (outside any timed region): per step and
        wave, device copies of the engine's B and eps pools."""
        self.step_inputs = []
        for t in range(steps):
            per_wave = []
            for j, w in enumerate(self.waves):
                eng = self.engines[0][j]
                if self.inputs == "device":
                    for s_idx, sysm in enumerate(self.systems):
                        ks = [p for p, k in enumerate(w) if self.items[k].system == s_idx]
                        if not ks:
                            continue
                        gen = DeviceBlockInputs(sysm, step=t)
                        _fill_subset(gen, eng, [self.items[w[p]].monomers for p in ks], ks)
                else:
                    eng.set_inputs([self.systems[self.items[k].system].at_step(t)
                                    .fragment(self.items[k].monomers) for k in w])
                per_wave.append((eng.B.clone(), eng.eps.clone()))
            self.step_inputs.append(per_wave)
        torch.cuda.synchronize()

    # ---------------------------------------------------------------- execution
    def run(self, mode: str = "async"):
        """Runs every prepared step; returns (device energies [steps][items], MBE3 totals
        [steps][systems] as a device tensor, elapsed ms between the first launch and the
        end of the last step)."""
        assert mode in ("sync", "async")
        steps = len(self.step_inputs)
        W = len(self.waves)
        energies = torch.zeros((steps, len(self.items)), dtype=torch.float64, device="cuda")
        totals = torch.zeros((steps, len(self.systems)), dtype=torch.float64, device="cuda")
        done = [[torch.cuda.Event() for _ in range(W)] for _ in range(steps)]
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        main = torch.cuda.current_stream()
        t0.record(main)
        for s in self.streams:
            s.wait_event(t0)
        for t in range(steps):
            st = self.streams[t % 2]
            engs = self.engines[t % 2]
            with torch.cuda.stream(st):
                for j in range(W):
                    if t > 0:
                        for d in ([W - 1] if mode == "sync" else self.deps[j]):
                            st.wait_event(done[t - 1][d])
                    B, eps = self.step_inputs[t][j]
                    engs[j].B.copy_(B, non_blocking=True)
                    engs[j].eps.copy_(eps, non_blocking=True)
                    engs[j].run(stream=st)
                    n = len(self.waves[j])
                    energies[t].index_copy_(0, self.wave_index[j], engs[j].energy[:n])
                    done[t][j].record(st)
                for s_idx, (a, b) in enumerate(self.sys_slices):
                    totals[t, s_idx:s_idx + 1].copy_(
                        rimp2.mbe_combine(energies[t, a:b], self.coeff_dev[a:b], stream=st))
        for s in self.streams:
            main.wait_stream(s)
        t1.record(main)
        torch.cuda.synchronize()
        for row in self.engines:
            for e in row:
                e.check_status()
        return energies, totals, t0.elapsed_time(t1)


def _fill_subset(gen, eng, monomer_lists, positions):
    """DeviceBlockInputs.fill restricted to the engine's fragments at `positions`."""

    class _View:
        pass

    view = _View()
    view.B, view.eps = eng.B, eng.eps
    view.dims = [eng.dims[p] for p in positions]
    view.offsets = [eng.offsets[p] for p in positions]
    gen.fill(view, monomer_lists)
