"""ctypes front end of the plain FP64 C oracle (rimp2_oracle.c).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU
baseline may import this module.  It builds ``liboracle.so`` with gcc on first use
(``build()``), independently of the GPU library, and never touches a GPU.

Functions follow the appendix definitions; see the header of rimp2_oracle.c.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "rimp2_oracle.c")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile liboracle.so (plain C, OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-std=c11", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i, d = ctypes.c_int, ctypes.c_double
            lib.rimp2_oracle_fragment_range.argtypes = [i, i, i, _dp, _dp, _dp, i, i, i,
                                                        _dp, _dp, _dp, _dp, _dp]
            lib.rimp2_oracle_fragment_range.restype = i
            for name in ("rimp2_oracle_pair_energy", "rimp2_oracle_pab_elem",
                         "rimp2_oracle_pij_elem"):
                f = getattr(lib, name)
                f.argtypes = [i, i, i, _dp, _dp, _dp, i, i, i]
                f.restype = d
            lib.rimp2_oracle_gamma_elem.argtypes = [i, i, i, _dp, _dp, _dp, i, i, i, i]
            lib.rimp2_oracle_gamma_elem.restype = d
            lib.rimp2_oracle_threads.argtypes = []
            lib.rimp2_oracle_threads.restype = i
            lib.rimp2_oracle_spin_components.argtypes = [i, i, i, _dp, _dp, _dp, i, _dp, _dp]
            lib.rimp2_oracle_spin_components.restype = i
            lib.rimp2_oracle_pair_spin.argtypes = [i, i, i, _dp, _dp, _dp, i, i, _dp]
            lib.rimp2_oracle_pair_spin.restype = i
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _inputs(B, eo, ev):
    B = np.ascontiguousarray(B, dtype=np.float64)
    eo = np.ascontiguousarray(eo, dtype=np.float64)
    ev = np.ascontiguousarray(ev, dtype=np.float64)
    o, v, X = B.shape
    assert eo.shape == (o,) and ev.shape == (v,)
    return B, eo, ev, o, v, X


def threads() -> int:
    return int(_load().rimp2_oracle_threads())


def fragment(B, eo, ev, nthreads: int = 0, k_range=None, want=("gamma", "pij", "pab", "epair")):
    """Energy, Gamma[o][v][X], P_ij[o][o], P_ab[v][v] and pair energies of one fragment.

    ``k_range=(k0, k1)`` restricts the second pair index (a bounded sample used only to
    time the oracle); the default is the whole fragment.
    """
    B, eo, ev, o, v, X = _inputs(B, eo, ev)
    k0, k1 = (0, o) if k_range is None else k_range
    out = {"energy": np.zeros(1)}
    out["gamma"] = np.zeros((o, v, X)) if "gamma" in want else None
    out["pij"] = np.zeros((o, o)) if "pij" in want else None
    out["pab"] = np.zeros((v, v)) if "pab" in want else None
    out["epair"] = np.zeros((o, o)) if "epair" in want else None
    rc = _load().rimp2_oracle_fragment_range(
        o, v, X, _ptr(B), _ptr(eo), _ptr(ev), int(k0), int(k1), int(nthreads),
        _ptr(out["energy"]), _ptr(out["gamma"]), _ptr(out["pij"]), _ptr(out["pab"]),
        _ptr(out["epair"]))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    out["energy"] = float(out["energy"][0])
    return out


def pair_energy(B, eo, ev, i, j, nthreads=0) -> float:
    B, eo, ev, o, v, X = _inputs(B, eo, ev)
    return _load().rimp2_oracle_pair_energy(o, v, X, _ptr(B), _ptr(eo), _ptr(ev), i, j, nthreads)


def gamma_elem(B, eo, ev, i, a, Q, nthreads=0) -> float:
    B, eo, ev, o, v, X = _inputs(B, eo, ev)
    return _load().rimp2_oracle_gamma_elem(o, v, X, _ptr(B), _ptr(eo), _ptr(ev), i, a, Q,
                                           nthreads)


def pab_elem(B, eo, ev, a, b, nthreads=0) -> float:
    B, eo, ev, o, v, X = _inputs(B, eo, ev)
    return _load().rimp2_oracle_pab_elem(o, v, X, _ptr(B), _ptr(eo), _ptr(ev), a, b, nthreads)


def pij_elem(B, eo, ev, i, j, nthreads=0) -> float:
    B, eo, ev, o, v, X = _inputs(B, eo, ev)
    return _load().rimp2_oracle_pij_elem(o, v, X, _ptr(B), _ptr(eo), _ptr(ev), i, j, nthreads)


def spin_components(B, eo, ev, nthreads=0):
    """(E_OS, E_SS): opposite-spin sum T V and same-spin sum (T - T^T) V of one fragment
    (E = E_OS + E_SS; SCS-MP2 is named in the paper's Introduction)."""
    B, eo, ev, o, v, X = _inputs(B, eo, ev)
    out = np.zeros(2)
    rc = _load().rimp2_oracle_spin_components(o, v, X, _ptr(B), _ptr(eo), _ptr(ev), int(nthreads),
                                               _ptr(out[0:1]), _ptr(out[1:2]))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return float(out[0]), float(out[1])


def pair_spin(B, eo, ev, i, j):
    """(opposite-spin, same-spin) energy of the pair (i, j)."""
    B, eo, ev, o, v, X = _inputs(B, eo, ev)
    out = np.zeros(2)
    if _load().rimp2_oracle_pair_spin(o, v, X, _ptr(B), _ptr(eo), _ptr(ev), i, j, _ptr(out)) != 0:
        raise ValueError("pair index out of range or allocation failed")
    return float(out[0]), float(out[1])


def algorithmic_flops(o: int, v: int, X: int) -> float:
    """2mnk FLOP count of one fragment (the paper's counting convention, Sec. "Measurement
    methodology"): V over pairs i<=j, Gamma, P_ab and P_ij as GEMMs."""
    return float(o * (o + 1) * v * v * X + 2 * o * o * v * v * X + 2 * o * o * v ** 3
                 + 2 * o ** 3 * v * v)
