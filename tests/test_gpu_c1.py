"""Full-size parity: the single large fragment (nocc=100, nvir=500, naux=1500, seed 0)
in the configuration bench.py times (BF16 split with the library's default slices, CUDA
graph), the FP8 split mode and the FP64 path, against the oracle's full result for this
fragment (tests/golden/c1_seed0.{json,npz}, written by tests/golden/make_c1_golden.py
from oracle/ alone).

Checked against the oracle: the energy and its opposite-spin part within 1e-8 Eh
(|E| ~ 1e7 Eh, so this is ~1e-15 relative); every pair energy and every element of P_ij
and P_ab within 1e-9 relative to max(|ref|, 1e-3 max|ref|) (near-zero elements are held
to 1e-12 of the largest); Gamma by the relative Frobenius error, the accuracy target of
the path, over 512 seeded elements and per occupied index (its row norms), each within
1e-9.  Gamma's sampled elements are also checked one by one: for the FP64 path and for
the BF16 split with 6 Gamma slices at the per-element bound above; for the default split
paths (BF16: 5 Gamma slices, 43 bits against one Tt scale per fragment) at 1e-9 of the
largest element, since an element 1e3 times below the largest keeps fewer significant
bits of the fragment-wide scale.  Identities that hold at any size check the rest of Gamma:
<B, Gamma> = E (homogeneity), plus Tr P_ij = -Tr P_ab, the Euler relation
-E = 2 (sum_i e_i P_ii + sum_a e_a P_aa), symmetry and signs.
"""
import json
import os

import numpy as np
import pytest
import torch

from paper_2410_21888_gb300 import rimp2, synth

pytestmark = pytest.mark.gpu

DIMS = (100, 500, 1500)
HERE = os.path.dirname(os.path.abspath(__file__))
TOL_E = 1e-8
TOL_A = 1e-9


@pytest.fixture(scope="module")
def golden():
    meta = json.load(open(os.path.join(HERE, "golden", "c1_seed0.json")))
    arr = dict(np.load(os.path.join(HERE, "golden", "c1_seed0.npz")))
    assert tuple(meta["inputs"][k] for k in ("nocc", "nvir", "naux")) == DIMS
    return meta, arr


@pytest.fixture(scope="module")
def c1():
    f = synth.fragment_inputs(*DIMS, seed=0)
    res = {}
    for name, prec, opts in (("bf16", "bf16", {}), ("fp8", "fp8", {}), ("fp64", "fp64", {}),
                             ("bf16_g6", "bf16", {"slices_g": 6})):
        eng = rimp2.Engine([DIMS], precision=prec, **opts)
        eng.set_inputs([f])
        eng.run()
        torch.cuda.synchronize()
        eng.check_status()
        v = eng.views(0)
        res[name] = {k: (float(t.item()) if k.startswith("energy") else t.cpu().numpy())
                     for k, t in v.items()}
        del eng, v
        torch.cuda.empty_cache()
    return f, res


def _elementwise(got, ref, tol):
    floor = 1e-3 * np.abs(ref).max()
    err = np.abs(got - ref) / np.maximum(np.abs(ref), floor)
    return float(err.max())


@pytest.mark.parametrize("prec", ["bf16", "fp8", "fp64"])
def test_c1_energy_vs_oracle(c1, golden, prec):
    _, r = c1
    meta, _ = golden
    assert abs(r[prec]["energy"] - meta["energy"]) <= TOL_E, r[prec]["energy"] - meta["energy"]
    assert abs(r[prec]["energy_os"] - meta["energy_os"]) <= TOL_E, \
        r[prec]["energy_os"] - meta["energy_os"]


@pytest.mark.parametrize("prec", ["bf16", "fp8", "fp64"])
def test_c1_pair_energies_and_densities_vs_oracle(c1, golden, prec):
    _, r = c1
    _, arr = golden
    for k in ("epair", "pij", "pab"):
        assert _elementwise(r[prec][k], arr[k], TOL_A) <= TOL_A, (k, _elementwise(r[prec][k], arr[k], TOL_A))


@pytest.mark.parametrize("prec,strict", [("bf16", False), ("fp8", False), ("fp64", True),
                                         ("bf16_g6", True)])
def test_c1_gamma_vs_oracle(c1, golden, prec, strict):
    _, r = c1
    meta, arr = golden
    g = r[prec]["gamma"]
    idx = arr["gamma_idx"]
    got, ref = g[idx[:, 0], idx[:, 1], idx[:, 2]], arr["gamma_val"]
    assert np.linalg.norm(got - ref) <= TOL_A * np.linalg.norm(ref)
    rn = np.sqrt(np.einsum("iaq,iaq->i", g, g))
    assert np.max(np.abs(rn - arr["gamma_row_norm"]) / arr["gamma_row_norm"]) <= TOL_A
    assert abs(np.linalg.norm(g) - meta["gamma_frobenius"]) <= TOL_A * meta["gamma_frobenius"]
    gmax = np.abs(g).max()
    floor = 1e-3 * gmax if strict else gmax
    err = np.abs(got - ref) / np.maximum(np.abs(ref), floor)
    assert err.max() <= TOL_A, float(err.max())


@pytest.mark.parametrize("prec,tol", [("bf16", 1e-9), ("fp8", 1e-9), ("fp64", 1e-11)])
def test_c1_identities(c1, prec, tol):
    f, res = c1
    r = res[prec]
    E = r["energy"]
    assert E < 0 and r["energy_os"] < 0 and E - r["energy_os"] < 0
    assert np.sum(r["epair"]) == pytest.approx(E, rel=tol)
    assert float(np.sum(f.B * r["gamma"])) == pytest.approx(E, rel=tol)
    assert np.trace(r["pij"]) == pytest.approx(-np.trace(r["pab"]), rel=tol)
    euler = 2.0 * (f.eo @ np.diag(r["pij"]) + f.ev @ np.diag(r["pab"]))
    assert euler == pytest.approx(-E, rel=tol)
    for k in ("pij", "pab", "epair"):
        a = r[k]
        assert np.linalg.norm(a - a.T) <= tol * np.linalg.norm(a)
    assert np.all(np.diag(r["pij"]) <= 0) and np.all(np.diag(r["pab"]) >= 0)
