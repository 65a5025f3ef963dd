"""Full-size parity: the single large fragment (nocc=100, nvir=500, naux=1500, seed 0)
in the configuration bench.py times (BF16 split, 5 slices for V, 6 for Gamma/P, CUDA
graph), the FP8 split mode (8 and 10 slices) and the FP64 path.

The oracle cannot run the whole fragment in a test, so it computes sampled outputs one
by one (pair energies, Gamma, P_ab and P_ij elements); identities that hold at any size
check the rest: E = sum_ij e_ij, <B, Gamma> = E (homogeneity), Tr P_ij = -Tr P_ab,
-E = 2 (sum_i e_i P_ii + sum_a e_a P_aa) (Euler), symmetry of P and e_pair, signs.

Tolerances: split path vs oracle 1e-9 relative on sampled elements (pair energies
1e-8 Eh absolute); split vs FP64 path total energy 1e-7 Eh (|E| ~ 1e7 Eh, ~1 ulp is
2e-9); identities 1e-9 relative (split) and 1e-11 (FP64).  The total energy is the
sharpest check of a one-signed error: the diagonal V_ii(a,a) carries a few per cent of
E, so a relative bias of 2^-40 on it moves E by ~1e-6 Eh.
"""
import numpy as np
import pytest
import torch

from oracle import oracle
from paper_2410_21888_gb300 import rimp2, synth

pytestmark = pytest.mark.gpu

DIMS = (100, 500, 1500)


@pytest.fixture(scope="module")
def c1():
    f = synth.fragment_inputs(*DIMS, seed=0)
    res = {}
    for prec in ("bf16", "fp8", "fp64"):
        eng = rimp2.Engine([DIMS], precision=prec)
        eng.set_inputs([f])
        eng.run()
        torch.cuda.synchronize()
        eng.check_status()
        v = eng.views(0)
        res[prec] = {k: (float(t.item()) if k in ("energy", "energy_os") else t.cpu().numpy())
                     for k, t in v.items()}
        del eng
        torch.cuda.empty_cache()
    return f, res


def _identities(f, r, tol):
    E = r["energy"]
    assert E < 0
    assert np.sum(r["epair"]) == pytest.approx(E, rel=tol)
    assert float(np.sum(f.B * r["gamma"])) == pytest.approx(E, rel=tol)
    assert np.trace(r["pij"]) == pytest.approx(-np.trace(r["pab"]), rel=tol)
    euler = 2.0 * (f.eo @ np.diag(r["pij"]) + f.ev @ np.diag(r["pab"]))
    assert euler == pytest.approx(-E, rel=tol)
    for k in ("pij", "pab", "epair"):
        a = r[k]
        assert np.linalg.norm(a - a.T) <= tol * np.linalg.norm(a)
    assert np.all(np.diag(r["pij"]) <= 0) and np.all(np.diag(r["pab"]) >= 0)


def test_c1_identities_split(c1):
    f, r = c1
    _identities(f, r["bf16"], 1e-9)


def test_c1_identities_fp8(c1):
    f, r = c1
    _identities(f, r["fp8"], 1e-9)


def test_c1_identities_fp64(c1):
    f, r = c1
    _identities(f, r["fp64"], 1e-11)


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_c1_split_vs_fp64_energy(c1, prec):
    _, r = c1
    assert abs(r[prec]["energy"] - r["fp64"]["energy"]) <= 1e-7
    # spin components: E_OS < E < 0 side by side, E_SS = E - E_OS < 0
    assert abs(r[prec]["energy_os"] - r["fp64"]["energy_os"]) <= 1e-7
    assert r[prec]["energy_os"] < 0 and r[prec]["energy"] - r[prec]["energy_os"] < 0
    for k in ("gamma", "pij", "pab"):
        a, b = r[prec][k], r["fp64"][k]
        assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(b), k


def test_c1_sampled_outputs_vs_oracle(c1):
    f, r = c1
    rng = np.random.default_rng(42)
    nthr = oracle.threads()
    for prec, tol in (("bf16", 1e-9), ("fp8", 1e-9), ("fp64", 1e-11)):
        g = r[prec]
        for (i, j) in [(0, 0), (3, 77), (99, 12)]:
            ref = oracle.pair_energy(f.B, f.eo, f.ev, i, j, nthr)
            assert abs(g["epair"][i, j] - ref) <= max(1e-8, tol * abs(ref)), (prec, i, j)
        gscale = np.abs(g["gamma"]).max()
        for _ in range(4):
            i, a, Q = int(rng.integers(100)), int(rng.integers(500)), int(rng.integers(1500))
            ref = oracle.gamma_elem(f.B, f.eo, f.ev, i, a, Q, nthr)
            assert abs(g["gamma"][i, a, Q] - ref) <= tol * max(abs(ref), 1e-3 * gscale), (prec, i, a, Q)
    # the denser sums once, on the split path (the configuration that is timed)
    g = r["bf16"]
    for (a, b) in [(7, 7), (13, 401)]:
        ref = oracle.pab_elem(f.B, f.eo, f.ev, a, b, nthr)
        assert abs(g["pab"][a, b] - ref) <= 1e-9 * max(abs(ref), 1e-3 * np.abs(g["pab"]).max())
    for (i, j) in [(5, 5), (20, 81)]:
        ref = oracle.pij_elem(f.B, f.eo, f.ev, i, j, nthr)
        assert abs(g["pij"][i, j] - ref) <= 1e-9 * max(abs(ref), 1e-3 * np.abs(g["pij"]).max())
