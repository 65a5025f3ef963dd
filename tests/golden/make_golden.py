"""Writes the exact-arithmetic golden fixtures in this folder.

Calls only oracle/exact.py (rational arithmetic over the Appendix definitions: the
RI integrals of Eq. MP2_ints, amplitudes X^ab_ij, Gamma, D^MP2_ij, D^MP2_ab).  Inputs
are small dyadic numbers, so every stored value is the exact result rounded once to
FP64.  Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import exact  # noqa: E402

CASES = {
    # o = v = 1 reduces to E = (sum_Q B_Q^2)^2 / (2 (e_i - e_a))
    "o1v1x3": {
        "B": [[[0.25, -0.5, 0.125]]],
        "eo": [-0.5], "ev": [1.25],
    },
    # two occupied, two virtual, three auxiliary functions, dyadic entries
    "o2v2x3": {
        "B": [[[0.25, -0.125, 0.5], [0.0625, 0.375, -0.25]],
              [[-0.5, 0.25, 0.125], [0.1875, -0.0625, 0.3125]]],
        "eo": [-1.25, -0.5], "ev": [0.75, 2.0],
    },
    # ragged: three occupied, two virtual, one auxiliary function (rank-1 V)
    "o3v2x1": {
        "B": [[[0.5], [-0.25]], [[0.125], [0.75]], [[-0.375], [0.0625]]],
        "eo": [-1.5, -0.75, -0.375], "ev": [0.25, 1.5],
    },
}


def _f(x):
    return float(x)


def main():
    for name, c in CASES.items():
        r = exact.everything(c["B"], c["eo"], c["ev"])
        out = {
            "citation": "Appendix: RI integrals (Eq. MP2_ints), amplitudes X^ab_ij, "
                        "Gamma^P_ia (MO-B basis), D^MP2_ij, D^MP2_ab; closed-shell energy "
                        "E = sum X^ab_ij [2(ia|jb) - (ib|ja)]",
            "generator": "tests/golden/make_golden.py via oracle/exact.py (Fraction arithmetic)",
            "inputs": c,
            "energy": _f(r["energy"]),
            "energy_exact": str(r["energy"]),
            "gamma": [[[_f(x) for x in row] for row in blk] for blk in r["gamma"]],
            "pij": [[_f(x) for x in row] for row in r["pij"]],
            "pab": [[_f(x) for x in row] for row in r["pab"]],
            "epair": [[_f(x) for x in row] for row in r["epair"]],
        }
        with open(os.path.join(HERE, f"exact_{name}.json"), "w") as fh:
            json.dump(out, fh, indent=1)
            fh.write("\n")


if __name__ == "__main__":
    main()
