"""Host logic of the asynchronous MBE3 time-step pipeline (CPU): the priority order of
Sec. "Asynchronous time steps" (distance to the reference monomer, then decreasing size),
waves of about equal cost, and the wave dependencies that decide when a polymer of the
next step may start."""
import itertools

import numpy as np

from paper_2410_21888_gb300 import pipeline


def _items(seed=0, n=9):
    rng = np.random.default_rng(seed)
    items = []
    for m in range(n):
        items.append(pipeline.Item(0, (m,), 1, float(rng.uniform(0, 10)), float(rng.uniform(1, 2))))
    for a, b in itertools.combinations(range(n), 2):
        if rng.uniform() < 0.4:
            items.append(pipeline.Item(0, (a, b), -1, min(items[a].dist, items[b].dist),
                                       float(rng.uniform(5, 10))))
    return items


def test_priority_order_distance_then_decreasing_size():
    items = _items()
    order = pipeline.priority_order(items)
    assert sorted(order) == list(range(len(items)))
    for p, q in zip(order, order[1:]):
        a, b = items[p], items[q]
        assert a.dist < b.dist or (a.dist == b.dist and a.cost >= b.cost)


def test_waves_cover_in_order_with_balanced_cost():
    items = _items(1, 12)
    order = pipeline.priority_order(items)
    costs = [it.cost for it in items]
    for n_waves in (1, 3, 5, 40):
        waves = pipeline.cut_waves(order, costs, n_waves)
        assert [k for w in waves for k in w] == order
        assert all(len(w) > 0 for w in waves) and len(waves) <= n_waves
        if n_waves == 3:
            tot = [sum(costs[k] for k in w) for w in waves]
            assert max(tot) <= sum(costs) / 3 + max(costs)


def test_dependencies_are_exactly_the_waves_sharing_a_monomer():
    items = _items(2, 10)
    order = pipeline.priority_order(items)
    waves = pipeline.cut_waves(order, [it.cost for it in items], 4)
    deps = pipeline.wave_dependencies(items, waves)
    for j, w in enumerate(waves):
        mons = {m for k in w for m in items[k].monomers}
        want = sorted({i for i, u in enumerate(waves)
                       if any(set(items[k].monomers) & mons for k in u)})
        assert deps[j] == want
        assert j in deps[j]
