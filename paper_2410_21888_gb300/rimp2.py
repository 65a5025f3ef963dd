"""Python binding of librimp2 (ctypes).  Argument marshalling only: every step of the
RI-MP2 hot path runs in the library's CUDA kernels; PyTorch provides device memory and
streams.  There is no CPU fallback: without the built library on a CUDA machine the
calls raise.

Names follow include/rimp2.h: ``Plan`` wraps rimp2_plan_create / rimp2_energy_grad,
``Engine`` owns device pools for a fixed batch of fragments, and ``energy_grad`` is the
one-call convenience for a single fragment (host or device inputs).
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "librimp2.so")

RIMP2_FP64 = 0
RIMP2_BF16_SPLIT = 1
RIMP2_FP8_SPLIT = 2
PRECISIONS = {"fp64": RIMP2_FP64, "bf16": RIMP2_BF16_SPLIT, "bf16_split": RIMP2_BF16_SPLIT,
              "fp8": RIMP2_FP8_SPLIT, "fp8_split": RIMP2_FP8_SPLIT}

ERRORS = {
    -1: "BAD_ARG", -2: "SHAPE", -3: "DENOM", -4: "NONFINITE", -5: "WORKSPACE", -6: "CUDA",
    -7: "TIMEOUT", -8: "UNSUPPORTED", -9: "NOMEM",
}

EXPORTED = ("rimp2_default_options", "rimp2_plan_create", "rimp2_workspace_size",
            "rimp2_energy_grad", "rimp2_get_status", "rimp2_get_stats", "rimp2_plan_destroy",
            "rimp2_status_string", "rimp2_version")


class Rimp2Error(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: rimp2 status {code} ({ERRORS.get(code, '?')}: "
                         f"{status_string(code) if _lib is not None else ''})")


class Frag(ctypes.Structure):
    _fields_ = [("nocc", ctypes.c_int32), ("nvir", ctypes.c_int32), ("naux", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("b_off", ctypes.c_int64), ("eo_off", ctypes.c_int64),
                ("ev_off", ctypes.c_int64), ("gamma_off", ctypes.c_int64),
                ("pij_off", ctypes.c_int64), ("pab_off", ctypes.c_int64),
                ("epair_off", ctypes.c_int64)]


class Batch(ctypes.Structure):
    _fields_ = [("nfrag", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("frags", ctypes.POINTER(Frag)), ("B", ctypes.c_void_p), ("eps", ctypes.c_void_p),
                ("gamma", ctypes.c_void_p), ("pij", ctypes.c_void_p), ("pab", ctypes.c_void_p),
                ("epair", ctypes.c_void_p), ("energy", ctypes.c_void_p),
                ("energy_os", ctypes.c_void_p), ("energy_scs", ctypes.c_void_p)]


class Options(ctypes.Structure):
    _fields_ = [("slices_v", ctypes.c_int32), ("slices_t", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("check_inputs", ctypes.c_int32),
                ("autotune", ctypes.c_int32), ("profile_stages", ctypes.c_int32),
                ("max_workspace_bytes", ctypes.c_size_t), ("stage_k", ctypes.c_int32),
                ("n_tile", ctypes.c_int32), ("autotune_cache", ctypes.c_char_p),
                ("slices_g", ctypes.c_int32), ("scs_os", ctypes.c_double),
                ("scs_ss", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("flops_per_call", ctypes.c_double), ("last_ms", ctypes.c_double),
                ("calls", ctypes.c_int64), ("tiles_per_call", ctypes.c_int64),
                ("launches_per_call", ctypes.c_int32), ("waves", ctypes.c_int32),
                ("graph_captures", ctypes.c_int32), ("status", ctypes.c_int32),
                ("tune_variant", ctypes.c_int32), ("tune_done", ctypes.c_int32),
                ("tune_ms", ctypes.c_double * 4), ("stage_ms", ctypes.c_double * 4),
                ("slices", ctypes.c_int32 * 3), ("pad", ctypes.c_int32),
                ("launch_ms", ctypes.c_double * 2), ("tc_flops", ctypes.c_double * 4),
                ("n_tile", ctypes.c_int32 * 3), ("stage_k", ctypes.c_int32 * 3),
                ("tune_trials", ctypes.c_int32), ("pad2", ctypes.c_int32)]


_lib = None


def load(path: str = LIB_PATH):
    """Load librimp2.so (built in-tree by __graft_entry__.build()); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"librimp2.so not found at {path}: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    vp, i32 = ctypes.c_void_p, ctypes.c_int32
    lib.rimp2_default_options.argtypes = [ctypes.POINTER(Options)]
    lib.rimp2_default_options.restype = None
    lib.rimp2_plan_create.argtypes = [ctypes.POINTER(Frag), i32, i32, ctypes.POINTER(Options),
                                      ctypes.POINTER(vp)]
    lib.rimp2_plan_create.restype = ctypes.c_int
    lib.rimp2_workspace_size.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    lib.rimp2_workspace_size.restype = ctypes.c_int
    lib.rimp2_energy_grad.argtypes = [vp, ctypes.POINTER(Batch), vp, ctypes.c_size_t, vp]
    lib.rimp2_energy_grad.restype = ctypes.c_int
    lib.rimp2_get_status.argtypes = [vp]
    lib.rimp2_get_status.restype = ctypes.c_int
    lib.rimp2_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    lib.rimp2_get_stats.restype = ctypes.c_int
    lib.rimp2_plan_destroy.argtypes = [vp]
    lib.rimp2_plan_destroy.restype = None
    lib.rimp2_status_string.argtypes = [ctypes.c_int]
    lib.rimp2_status_string.restype = ctypes.c_char_p
    lib.rimp2_version.argtypes = []
    lib.rimp2_version.restype = ctypes.c_char_p
    _lib = lib
    return lib


def status_string(code: int) -> str:
    return load().rimp2_status_string(int(code)).decode()


def version() -> str:
    return load().rimp2_version().decode()


def _check(code: int, what: str):
    if code != 0:
        raise Rimp2Error(code, what)


def default_options() -> Options:
    o = Options()
    load().rimp2_default_options(ctypes.byref(o))
    return o


def _require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("rimp2 needs a CUDA device (sm_103a); no CPU fallback exists")


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Plan:
    """rimp2_plan for a fixed list of fragment shapes (nocc, nvir, naux).

    Options map one to one onto rimp2_options (include/rimp2.h): ``slices_v`` / ``slices_t``
    / ``slices_g`` are the digit slices of V's operands, of P_ab / P_ij's and of Gamma's
    (0: the precision's default; ``slices_g`` defaults to ``slices_t``); ``n_tile`` (48, 64,
    80, 96) and ``stage_k`` (16, 32) shape the tensor-core tiles; ``profile_stages``
    records per-stage device times (``stats().stage_ms``); ``autotune`` times the
    contraction-stage variants in situ, optionally cached in ``autotune_cache``;
    ``max_workspace_bytes`` splits a large batch into waves; ``scs_os`` / ``scs_ss`` are
    the spin-component weights of the ``energy_scs`` output (None: the library default,
    Grimme's SCS-MP2).
    """

    def __init__(self, dims: Sequence[tuple], precision: str = "fp64", slices_v: int = 0,
                 slices_t: int = 0, use_graph: bool = True, check_inputs: bool = True,
                 max_workspace_bytes: int = 0, profile_stages: bool = False,
                 want_gamma: bool = True, want_p: bool = True, autotune: bool = False,
                 autotune_cache: str | None = None, stage_k: int = 0, n_tile: int = 0,
                 slices_g: int = 0, scs_os: float | None = None, scs_ss: float | None = None):
        _require_cuda()
        lib = load()
        self.dims = [tuple(int(x) for x in d) for d in dims]
        self.precision = precision
        frags = (Frag * max(1, len(self.dims)))()
        for k, (o, v, X) in enumerate(self.dims):
            frags[k].nocc, frags[k].nvir, frags[k].naux = o, v, X
            frags[k].gamma_off = 0 if want_gamma else -1
            frags[k].pij_off = frags[k].pab_off = 0 if want_p else -1
        opt = default_options()
        opt.slices_v, opt.slices_t, opt.slices_g = int(slices_v), int(slices_t), int(slices_g)
        opt.use_graph, opt.check_inputs = int(use_graph), int(check_inputs)
        opt.max_workspace_bytes = int(max_workspace_bytes)
        opt.profile_stages = int(profile_stages)
        opt.autotune = int(autotune)
        opt.stage_k = int(stage_k)
        opt.n_tile = int(n_tile)
        if scs_os is not None:
            opt.scs_os = float(scs_os)
        if scs_ss is not None:
            opt.scs_ss = float(scs_ss)
        self._cache = autotune_cache.encode() if autotune_cache else None
        opt.autotune_cache = self._cache
        h = ctypes.c_void_p()
        _check(lib.rimp2_plan_create(frags, len(self.dims), PRECISIONS[precision],
                                     ctypes.byref(opt), ctypes.byref(h)), "rimp2_plan_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def workspace_size(self) -> int:
        n = ctypes.c_size_t()
        _check(load().rimp2_workspace_size(self._h, ctypes.byref(n)), "rimp2_workspace_size")
        return int(n.value)

    def energy_grad(self, batch: Batch, workspace: torch.Tensor, stream=None):
        ws_ptr = workspace.data_ptr() if workspace is not None and workspace.numel() else None
        ws_bytes = workspace.numel() * workspace.element_size() if ws_ptr else 0
        _check(load().rimp2_energy_grad(self._h, ctypes.byref(batch), ws_ptr, ws_bytes,
                                        _stream_handle(stream)), "rimp2_energy_grad")

    def status(self) -> int:
        return int(load().rimp2_get_status(self._h))

    def stats(self) -> Stats:
        s = Stats()
        _check(load().rimp2_get_stats(self._h, ctypes.byref(s)), "rimp2_get_stats")
        return s

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().rimp2_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Engine:
    """Device pools + plan for a fixed batch of fragments.

    ``set_inputs`` copies B / orbital energies (numpy or torch, host or device) into the
    device pools; ``run`` launches the hot path; results stay in the device tensors
    ``energy``, ``gamma``, ``pij``, ``pab``, ``epair`` (pools, see ``views``).
    """

    def __init__(self, dims: Sequence[tuple], precision: str = "fp64", want_gamma=True,
                 want_p=True, want_epair=True, device="cuda", **plan_opts):
        _require_cuda()
        self.dims = [tuple(int(x) for x in d) for d in dims]
        self.device = torch.device(device)
        self.plan = Plan(self.dims, precision=precision, want_gamma=want_gamma, want_p=want_p,
                         **plan_opts)
        nb = sum(o * v * X for o, v, X in self.dims)
        ne = sum(o + v for o, v, X in self.dims)
        npij = sum(o * o for o, v, X in self.dims)
        npab = sum(v * v for o, v, X in self.dims)
        f64 = dict(dtype=torch.float64, device=self.device)
        self.B = torch.zeros(max(nb, 1), **f64)
        self.eps = torch.zeros(max(ne, 1), **f64)
        self.gamma = torch.zeros(max(nb, 1), **f64) if want_gamma else None
        self.pij = torch.zeros(max(npij, 1), **f64) if want_p else None
        self.pab = torch.zeros(max(npab, 1), **f64) if want_p else None
        self.epair = torch.zeros(max(npij, 1), **f64) if want_epair else None
        self.energy = torch.zeros(max(len(self.dims), 1), **f64)
        self.energy_os = torch.zeros(max(len(self.dims), 1), **f64)   # opposite-spin part
        self.energy_scs = torch.zeros(max(len(self.dims), 1), **f64)  # spin-component scaled
        ws = self.plan.workspace_size()
        self.workspace = torch.empty(max(ws, 256), dtype=torch.uint8, device=self.device)
        self._frags = (Frag * max(1, len(self.dims)))()
        self.offsets = []
        b = e = pij = pab = 0
        for k, (o, v, X) in enumerate(self.dims):
            fr = self._frags[k]
            fr.nocc, fr.nvir, fr.naux, fr.flags = o, v, X, 0
            fr.b_off, fr.eo_off, fr.ev_off = b, e, e + o
            fr.gamma_off = b if want_gamma else -1
            fr.pij_off = pij if want_p else -1
            fr.pab_off = pab if want_p else -1
            fr.epair_off = pij if want_epair else -1
            self.offsets.append((b, e, pij, pab))
            b += o * v * X
            e += o + v
            pij += o * o
            pab += v * v
        self._batch = Batch()
        self._batch.nfrag = len(self.dims)
        self._batch.frags = self._frags
        self._batch.B = self.B.data_ptr()
        self._batch.eps = self.eps.data_ptr()
        self._batch.gamma = self.gamma.data_ptr() if want_gamma else None
        self._batch.pij = self.pij.data_ptr() if want_p else None
        self._batch.pab = self.pab.data_ptr() if want_p else None
        self._batch.epair = self.epair.data_ptr() if want_epair else None
        self._batch.energy = self.energy.data_ptr()
        self._batch.energy_os = self.energy_os.data_ptr()
        self._batch.energy_scs = self.energy_scs.data_ptr()

    def set_inputs(self, frags, non_blocking=False):
        """frags: sequence of objects with .B [o][v][X], .eo, .ev (numpy or torch)."""
        for k, fr in enumerate(frags):
            o, v, X = self.dims[k]
            b, e, _, _ = self.offsets[k]
            self.B[b:b + o * v * X].copy_(torch.as_tensor(fr.B).reshape(-1), non_blocking=non_blocking)
            self.eps[e:e + o].copy_(torch.as_tensor(fr.eo), non_blocking=non_blocking)
            self.eps[e + o:e + o + v].copy_(torch.as_tensor(fr.ev), non_blocking=non_blocking)

    def run(self, stream=None):
        self.plan.energy_grad(self._batch, self.workspace, stream=stream)

    def check_status(self):
        st = self.plan.status()
        if st != 0:
            raise Rimp2Error(st, "device status")

    def views(self, k: int) -> dict:
        """Per-fragment views of the output pools (device tensors)."""
        o, v, X = self.dims[k]
        b, e, pij, pab = self.offsets[k]
        out = {"energy": self.energy[k], "energy_os": self.energy_os[k],
               "energy_scs": self.energy_scs[k]}
        if self.gamma is not None:
            out["gamma"] = self.gamma[b:b + o * v * X].view(o, v, X)
        if self.pij is not None:
            out["pij"] = self.pij[pij:pij + o * o].view(o, o)
            out["pab"] = self.pab[pab:pab + v * v].view(v, v)
        if self.epair is not None:
            out["epair"] = self.epair[pij:pij + o * o].view(o, o)
        return out


def energy_grad(B, eo, ev, precision: str = "fp64", want_gamma=True, want_p=True, sync=True,
                **plan_opts) -> dict:
    """One fragment through the library: B[o][v][X], eps_occ[o], eps_vir[v] as numpy
    arrays or torch tensors (host or device).  Returns device tensors."""
    B_t = torch.as_tensor(B)
    o, v, X = (int(x) for x in B_t.shape)
    eng = Engine([(o, v, X)], precision=precision, want_gamma=want_gamma, want_p=want_p,
                 **plan_opts)

    class _F:
        pass

    f = _F()
    f.B, f.eo, f.ev = B_t, torch.as_tensor(eo), torch.as_tensor(ev)
    eng.set_inputs([f])
    eng.run()
    out = eng.views(0)
    if sync:
        torch.cuda.synchronize()
        eng.check_status()
    out["engine"] = eng
    return out


def scs_energy(B, eo, ev, precision: str = "fp64", c_os: float | None = None,
               c_ss: float | None = None, **plan_opts):
    """Spin-component-scaled MP2 energy c_os E_OS + c_ss E_SS of one fragment, formed by
    the library (batch.energy_scs; default weights: Grimme's SCS-MP2).  Returns the
    device scalar."""
    out = energy_grad(B, eo, ev, precision=precision, want_gamma=False, want_p=False,
                      scs_os=c_os, scs_ss=c_ss, **plan_opts)
    return out["energy_scs"]


# ---------------------------------------------------------------- MBE3 (include/rimp2_mbe.h)

TRIMER_RULES = {"max": 0, "two_pairs": 1}


def _mbe_lib():
    lib = load()
    if not getattr(lib, "_mbe_ready", False):
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.rimp2_mbe_polymers.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_int32,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                           i32p, ctypes.c_int64, i64p, i32p, ctypes.c_int64, i64p]
        lib.rimp2_mbe_polymers.restype = ctypes.c_int
        lib.rimp2_mbe_coefficients.argtypes = [ctypes.c_int32, i32p, ctypes.c_int64, i32p,
                                               ctypes.c_int64, i32p, i32p, ctypes.c_int64, i64p]
        lib.rimp2_mbe_coefficients.restype = ctypes.c_int
        lib.rimp2_mbe_combine.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                          ctypes.c_void_p, ctypes.c_void_p]
        lib.rimp2_mbe_combine.restype = ctypes.c_int
        vp = ctypes.c_void_p
        lib.rimp2_assembly_create.argtypes = [ctypes.c_int32, i32p, i32p, i32p, ctypes.c_int64,
                                              i32p, i32p, i64p, i64p, i64p, ctypes.POINTER(vp)]
        lib.rimp2_assembly_create.restype = ctypes.c_int
        lib.rimp2_assembly_sizes.argtypes = [vp, i64p, i64p, i64p]
        lib.rimp2_assembly_sizes.restype = ctypes.c_int
        lib.rimp2_assembly_block_index.argtypes = [vp, i64p]
        lib.rimp2_assembly_block_index.restype = ctypes.c_int
        lib.rimp2_assembly_run.argtypes = [vp, vp, vp, vp, vp, vp, vp, ctypes.c_int32, vp]
        lib.rimp2_assembly_run.restype = ctypes.c_int
        lib.rimp2_assembly_destroy.argtypes = [vp]
        lib.rimp2_assembly_destroy.restype = None
        lib._mbe_ready = True
    return lib


def _i32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def mbe_polymers(centroids, r_dimer: float, r_trimer: float, rule: str = "max"):
    """Dimers (n_d x 2) and trimers (n_t x 3) within the cutoffs (host, C++)."""
    lib = _mbe_lib()
    c = np.ascontiguousarray(centroids, dtype=np.float64)
    n = c.shape[0]
    nd, nt = ctypes.c_int64(), ctypes.c_int64()
    cp = c.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    _check(lib.rimp2_mbe_polymers(cp, n, r_dimer, r_trimer, TRIMER_RULES[rule], None, 0,
                                  ctypes.byref(nd), None, 0, ctypes.byref(nt)),
           "rimp2_mbe_polymers")
    d = np.zeros((max(nd.value, 1), 2), dtype=np.int32)
    t = np.zeros((max(nt.value, 1), 3), dtype=np.int32)
    _check(lib.rimp2_mbe_polymers(cp, n, r_dimer, r_trimer, TRIMER_RULES[rule], _i32(d),
                                  nd.value, ctypes.byref(nd), _i32(t), nt.value, ctypes.byref(nt)),
           "rimp2_mbe_polymers")
    return d[:nd.value], t[:nt.value]


def mbe_coefficients(n: int, dimers, trimers):
    """Fragments ([k] tuples of monomer ids) and integer coefficients c with
    E_MBE3 = sum c_f E_f (host, C++)."""
    lib = _mbe_lib()
    d = np.ascontiguousarray(np.asarray(dimers, dtype=np.int32).reshape(-1, 2))
    t = np.ascontiguousarray(np.asarray(trimers, dtype=np.int32).reshape(-1, 3))
    nf = ctypes.c_int64()
    _check(lib.rimp2_mbe_coefficients(n, _i32(d), len(d), _i32(t), len(t), None, None, 0,
                                      ctypes.byref(nf)), "rimp2_mbe_coefficients")
    fr = np.zeros((max(nf.value, 1), 3), dtype=np.int32)
    co = np.zeros(max(nf.value, 1), dtype=np.int32)
    _check(lib.rimp2_mbe_coefficients(n, _i32(d), len(d), _i32(t), len(t), _i32(fr), _i32(co),
                                      nf.value, ctypes.byref(nf)), "rimp2_mbe_coefficients")
    frags = [tuple(int(x) for x in row if x >= 0) for row in fr[:nf.value]]
    return frags, co[:nf.value].copy()


class MBEAssembly:
    """MBE3 assembly of the fragments' Gamma, P_ij, P_ab over the system's index spaces
    (include/rimp2_mbe.h).  `fragments`: monomer tuples in the order the fragments
    concatenate their orbitals; offsets of each fragment's outputs in the batch pools
    (e.g. Engine.offsets: Gamma at the B offset); -1 for no contribution."""

    def __init__(self, nocc, nvir, naux, fragments, coeff, gamma_off, pij_off, pab_off):
        lib = _mbe_lib()
        self._lib = lib
        self.n = len(nocc)
        sz = [np.ascontiguousarray(np.asarray(x, dtype=np.int32)) for x in (nocc, nvir, naux)]
        fm = np.full((len(fragments), 3), -1, dtype=np.int32)
        for k, f in enumerate(fragments):
            fm[k, :len(f)] = f
        co = np.ascontiguousarray(np.asarray(coeff, dtype=np.int32))
        offs = [np.ascontiguousarray(np.asarray(x, dtype=np.int64)) for x in (gamma_off, pij_off, pab_off)]
        i64 = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        h = ctypes.c_void_p()
        _check(lib.rimp2_assembly_create(self.n, _i32(sz[0]), _i32(sz[1]), _i32(sz[2]), len(fragments),
                                         _i32(fm), _i32(co), i64(offs[0]), i64(offs[1]), i64(offs[2]),
                                         ctypes.byref(h)), "rimp2_assembly_create")
        self._h = h
        G, O, V = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib.rimp2_assembly_sizes(h, ctypes.byref(G), ctypes.byref(O), ctypes.byref(V)),
               "rimp2_assembly_sizes")
        self.gamma_elems, self.o_total, self.v_total = G.value, O.value, V.value
        idx = np.zeros(self.n ** 3, dtype=np.int64)
        _check(lib.rimp2_assembly_block_index(h, i64(idx)), "rimp2_assembly_block_index")
        self.block_index = idx.reshape(self.n, self.n, self.n)

    def outputs(self, device="cuda"):
        f64 = dict(dtype=torch.float64, device=device)
        return (torch.zeros(max(self.gamma_elems, 1), **f64),
                torch.zeros((self.o_total, self.o_total), **f64),
                torch.zeros((self.v_total, self.v_total), **f64))

    def run(self, gamma, pij, pab, gamma_sys, pij_sys, pab_sys, accumulate=False, stream=None):
        ptr = lambda t: None if t is None else t.data_ptr()
        _check(self._lib.rimp2_assembly_run(self._h, ptr(gamma), ptr(pij), ptr(pab), ptr(gamma_sys),
                                            ptr(pij_sys), ptr(pab_sys), int(bool(accumulate)),
                                            _stream_handle(stream)), "rimp2_assembly_run")

    def block(self, gamma_sys, I, J, K, nocc, nvir, naux):
        off = int(self.block_index[I, J, K])
        if off < 0:
            return None
        n = nocc[I] * nvir[J] * naux[K]
        return gamma_sys[off:off + n].view(nocc[I], nvir[J], naux[K])

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.rimp2_assembly_destroy(h)
            self._h = None


def mbe_combine(energy: torch.Tensor, coeff: torch.Tensor, stream=None) -> torch.Tensor:
    """Device FP64 sum_f coeff[f] * energy[f] (compensated); returns a 1-element tensor."""
    _require_cuda()
    assert energy.dtype == torch.float64 and coeff.dtype == torch.int32
    out = torch.empty(1, dtype=torch.float64, device=energy.device)
    _check(_mbe_lib().rimp2_mbe_combine(energy.data_ptr(), coeff.data_ptr(), energy.numel(),
                                        out.data_ptr(), _stream_handle(stream)),
           "rimp2_mbe_combine")
    return out


def mbe_corrections(energy: torch.Tensor, terms: torch.Tensor, sign, want_log=False,
                    stream=None):
    """Device per-polymer corrections sum_q sign[q] E[terms[t, q]] (FP64) and optionally
    log10(|.| + 1e-16) (FP32)."""
    lib = _mbe_lib()
    if not getattr(lib, "_corr_ready", False):
        lib.rimp2_mbe_corrections.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int64,
                                              ctypes.c_int32] + [ctypes.c_void_p] * 3
        lib.rimp2_mbe_corrections.restype = ctypes.c_int
        lib._corr_ready = True
    terms = terms.to(device="cuda", dtype=torch.int32).contiguous()
    n, k = terms.shape
    sg = torch.as_tensor(sign, dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    lg = torch.empty(n, dtype=torch.float32, device="cuda") if want_log else None
    _check(lib.rimp2_mbe_corrections(energy.data_ptr(), terms.data_ptr(), sg.data_ptr(), n, k,
                                     out.data_ptr(), lg.data_ptr() if want_log else None,
                                     _stream_handle(stream)), "rimp2_mbe_corrections")
    return (out, lg) if want_log else out


# ---------------------------------------------------------------- MLP screen (include/rimp2_mlp.h)

MLP_PARAMS = 64 * 9 + 64 + 64 * 64 + 64 + 64 * 64 + 64 + 64 + 1


def _mlp_lib():
    lib = load()
    if not getattr(lib, "_mlp_ready", False):
        vp = ctypes.c_void_p
        lib.rimp2_screen_features.argtypes = [vp, vp, ctypes.c_int32, vp, ctypes.c_int64, vp, vp, vp]
        lib.rimp2_screen_features.restype = ctypes.c_int
        lib.rimp2_mlp_grad.argtypes = [vp, vp, vp, vp, ctypes.c_int32, vp, vp, vp, vp, vp]
        lib.rimp2_mlp_grad.restype = ctypes.c_int
        lib.rimp2_mlp_adam.argtypes = [vp, vp, vp, vp, ctypes.c_int32, ctypes.c_float, vp]
        lib.rimp2_mlp_adam.restype = ctypes.c_int
        lib.rimp2_mlp_predict.argtypes = [vp, vp, ctypes.c_int64, vp, vp, vp, vp]
        lib.rimp2_mlp_predict.restype = ctypes.c_int
        lib._mlp_ready = True
    return lib


def _p(t):
    return None if t is None else t.data_ptr()


def screen_features(centroids, nocc, trimers, dimer_de, stream=None) -> torch.Tensor:
    """[nt, 9] FP32 features (device) from device tensors: centroids [n,3] f64, nocc [n]
    i32, trimers [nt,3] i32, dimer_de [n,n] f64."""
    nt = trimers.shape[0]
    out = torch.empty((nt, 9), dtype=torch.float32, device="cuda")
    _check(_mlp_lib().rimp2_screen_features(_p(centroids), _p(nocc), centroids.shape[0],
                                            _p(trimers), nt, _p(dimer_de), _p(out),
                                            _stream_handle(stream)), "rimp2_screen_features")
    return out


def mlp_grad(master, feats, y, idx, n, mean, std, want_loss=True, stream=None):
    grad = torch.empty(MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda") if want_loss else None
    _check(_mlp_lib().rimp2_mlp_grad(_p(master), _p(feats), _p(y), _p(idx), int(n), _p(mean),
                                     _p(std), _p(grad), _p(loss), _stream_handle(stream)),
           "rimp2_mlp_grad")
    return grad, loss


def mlp_adam(master, grad, m, v, t, lr, stream=None):
    _check(_mlp_lib().rimp2_mlp_adam(_p(master), _p(grad), _p(m), _p(v), int(t), float(lr),
                                     _stream_handle(stream)), "rimp2_mlp_adam")


def mlp_predict(master, feats, mean, std, stream=None) -> torch.Tensor:
    out = torch.empty(feats.shape[0], dtype=torch.float32, device="cuda")
    _check(_mlp_lib().rimp2_mlp_predict(_p(master), _p(feats), feats.shape[0], _p(mean), _p(std),
                                        _p(out), _stream_handle(stream)), "rimp2_mlp_predict")
    return out


# ---------------------------------------------------------------------------------------
# gradient step after the densities (include/rimp2_grad.h)

class ZvecArgs(ctypes.Structure):
    _fields_ = [("nocc", ctypes.c_int32), ("nvir", ctypes.c_int32), ("naux", ctypes.c_int32),
                ("max_iter", ctypes.c_int32), ("tol", ctypes.c_double),
                ("Bf", ctypes.c_void_p), ("eps", ctypes.c_void_p), ("jmh", ctypes.c_void_p),
                ("gamma", ctypes.c_void_p), ("pij", ctypes.c_void_p), ("pab", ctypes.c_void_p),
                ("gamma_p", ctypes.c_void_p), ("lp", ctypes.c_void_p), ("lpp", ctypes.c_void_p),
                ("dai", ctypes.c_void_p), ("info", ctypes.c_void_p)]


def _grad_lib():
    lib = load()
    if not getattr(lib, "_grad_ready", False):
        lib.rimp2_zvec_workspace_size.argtypes = [ctypes.c_int32] * 4 + [ctypes.POINTER(ctypes.c_size_t)]
        lib.rimp2_zvec_workspace_size.restype = ctypes.c_int
        lib.rimp2_zvec_solve.argtypes = [ctypes.POINTER(ZvecArgs), ctypes.c_void_p, ctypes.c_size_t,
                                         ctypes.c_void_p]
        lib.rimp2_zvec_solve.restype = ctypes.c_int
        lib._grad_ready = True
    return lib


def _dev64(x):
    return torch.as_tensor(x, dtype=torch.float64).to("cuda").contiguous()


def zvector_workspace_size(nocc: int, nvir: int, naux: int, max_iter: int = 0) -> int:
    n = ctypes.c_size_t()
    _check(_grad_lib().rimp2_zvec_workspace_size(nocc, nvir, naux, max_iter, ctypes.byref(n)),
           "rimp2_zvec_workspace_size")
    return n.value


def zvector(Bf, eps, gamma, pij, pab, jmh=None, max_iter: int = 0, tol: float = 0.0,
            workspace: torch.Tensor | None = None, stream=None, sync: bool = True) -> dict:
    """Gamma^P, L', L'' and the Z-vector solution D_ai ([nocc][nvir]) of one fragment
    through rimp2_zvec_solve.  Bf[n][n][naux], eps[n], gamma[nocc][nvir][naux],
    pij[nocc][nocc], pab[nvir][nvir], jmh[naux][naux] (or None): numpy or torch, host or
    device (copied to the device as FP64).  Returns device tensors; info = (iterations,
    ||r|| / ||rhs||, ||rhs||)."""
    _require_cuda()
    lib = _grad_lib()
    Bf_t, eps_t = _dev64(Bf), _dev64(eps)
    g_t, pij_t, pab_t = _dev64(gamma), _dev64(pij), _dev64(pab)
    o, v, X = (int(s) for s in g_t.shape)
    n = o + v
    if tuple(Bf_t.shape) != (n, n, X):
        raise ValueError(f"Bf has shape {tuple(Bf_t.shape)}, expected {(n, n, X)}")
    jmh_t = _dev64(jmh) if jmh is not None else None
    f64 = dict(dtype=torch.float64, device="cuda")
    out = {"lp": torch.empty((o, n), **f64), "lpp": torch.empty((v, n), **f64),
           "dai": torch.empty((o, v), **f64), "info": torch.empty(3, **f64)}
    if jmh_t is not None:
        out["gamma_p"] = torch.empty((o, v, X), **f64)
    need = zvector_workspace_size(o, v, X, max_iter)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device="cuda")
    a = ZvecArgs()
    a.nocc, a.nvir, a.naux, a.max_iter, a.tol = o, v, X, int(max_iter), float(tol)
    a.Bf, a.eps, a.jmh = _p(Bf_t), _p(eps_t), _p(jmh_t)
    a.gamma, a.pij, a.pab = _p(g_t), _p(pij_t), _p(pab_t)
    a.gamma_p = _p(out.get("gamma_p"))
    a.lp, a.lpp, a.dai, a.info = _p(out["lp"]), _p(out["lpp"]), _p(out["dai"]), _p(out["info"])
    _check(lib.rimp2_zvec_solve(ctypes.byref(a), _p(workspace), workspace.numel(),
                                _stream_handle(stream)), "rimp2_zvec_solve")
    out["_keep"] = (Bf_t, eps_t, g_t, pij_t, pab_t, jmh_t, workspace)
    if sync:
        torch.cuda.synchronize()
    return out
