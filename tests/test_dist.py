"""Multi-rank host logic on CPU (gloo, world size 2): LPT sharding of an uneven MBE3
fragment list and the one FP64 all-reduce of the partial MBE3 sums reproduce the serial
total; the shards cover every fragment exactly once and are balanced."""
import math
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

from oracle import mbe as ombe
from oracle import oracle
from paper_2410_21888_gb300 import build as libbuild
from paper_2410_21888_gb300 import dist, rimp2, synth


def _system():
    return synth.MonomerSystem(n_monomers=6, box=10.0, seed=3, nocc_range=(1, 3))


def _energies(s, frags):
    out = []
    for f in frags:
        x = s.fragment(f)
        out.append(oracle.fragment(x.B, x.eo, x.ev, want=(), nthreads=1)["energy"])
    return np.array(out)


def _worker(rank, world, port, frags, coeff, costs, q):
    import torch.distributed as tdist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    s = _system()
    total, mine = dist.sharded_mbe3_total(lambda fl: _energies(s, fl), frags, coeff, costs,
                                          rank, world)
    q.put((rank, total, mine))
    tdist.destroy_process_group()


def test_lpt_shards_cover_and_balance():
    rng = np.random.default_rng(0)
    costs = list(rng.pareto(1.5, size=300) + 1.0)
    for world in (1, 2, 4, 8):
        sh = dist.shard_lpt(costs, world)
        assert sorted(k for s in sh for k in s) == list(range(300))
        assert dist.imbalance(costs, sh) < 1.05 or world == 8


def test_sharded_total_matches_serial_gloo_two_ranks():
    libbuild.build()
    s = _system()
    d, t = rimp2.mbe_polymers(s.centroids, 7.0, 6.0, "two_pairs")
    frags, coeff = rimp2.mbe_coefficients(s.n, d, t)
    costs = [dist.fragment_cost(*s.fragment_dims(f)) for f in frags]
    E = _energies(s, frags)
    serial = math.fsum(float(c) * float(e) for c, e in zip(coeff, E))
    ref = ombe.mbe3(dict(zip(frags, E)), list(range(s.n)), [tuple(map(int, x)) for x in d],
                    [tuple(map(int, x)) for x in t])
    assert serial == pytest.approx(ref, abs=1e-12)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29000 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, frags, list(coeff), costs, q))
             for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert res[0][1] == pytest.approx(serial, abs=1e-12)
    assert res[1][1] == res[0][1]
    assert sorted(res[0][2] + res[1][2]) == list(range(len(frags)))
