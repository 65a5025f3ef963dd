"""Exact rational evaluation of the RI-MP2 energy and intermediates.

TEST INFRASTRUCTURE ONLY.  Pure-Python ``fractions.Fraction`` loops over the
definitions in the Appendix (same formulas as rimp2_oracle.c), for very small
fragments whose B and orbital energies are exact binary fractions.  The results carry
no rounding at all, which pins the FP64 oracle's rounding and also yields golden
fixtures (tests/golden/make_golden.py writes them).
"""
from __future__ import annotations

from fractions import Fraction


def everything(B, eo, ev):
    """B as nested lists [o][v][X] of Fractions (or ints/floats convertible exactly)."""
    o, v, X = len(B), len(B[0]), len(B[0][0])
    B = [[[Fraction(B[i][a][q]) for q in range(X)] for a in range(v)] for i in range(o)]
    eo = [Fraction(x) for x in eo]
    ev = [Fraction(x) for x in ev]

    def V(i, a, j, b):
        return sum((B[i][a][q] * B[j][b][q] for q in range(X)), Fraction(0))

    T = {}
    for i in range(o):
        for j in range(o):
            for a in range(v):
                for b in range(v):
                    T[i, j, a, b] = V(i, a, j, b) / (eo[i] + eo[j] - ev[a] - ev[b])

    def Tt(i, j, a, b):
        return 2 * T[i, j, a, b] - T[i, j, b, a]

    epair = [[sum((Tt(i, j, a, b) * V(i, a, j, b) for a in range(v) for b in range(v)),
                  Fraction(0)) for j in range(o)] for i in range(o)]
    energy = sum((epair[i][j] for i in range(o) for j in range(o)), Fraction(0))
    gamma = [[[sum((Tt(i, j, a, b) * B[j][b][q] for j in range(o) for b in range(v)),
                   Fraction(0)) for q in range(X)] for a in range(v)] for i in range(o)]
    pij = [[-sum((Tt(i, k, a, b) * T[j, k, a, b] for k in range(o) for a in range(v)
                  for b in range(v)), Fraction(0)) for j in range(o)] for i in range(o)]
    pab = [[sum((Tt(i, j, a, c) * T[i, j, b, c] for i in range(o) for j in range(o)
                 for c in range(v)), Fraction(0)) for b in range(v)] for a in range(v)]
    return {"energy": energy, "gamma": gamma, "pij": pij, "pab": pab, "epair": epair}
