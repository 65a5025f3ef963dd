"""The C-ABI library loads and exports every symbol include/*.h declares (CPU only:
no compute call is made without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_2410_21888_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(rimp2_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    path = libbuild.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = declared_symbols()
    for n in ("rimp2_plan_create", "rimp2_energy_grad", "rimp2_workspace_size",
              "rimp2_plan_destroy", "rimp2_get_status", "rimp2_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu(lib):
    lib.rimp2_status_string.restype = ctypes.c_char_p
    lib.rimp2_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.rimp2_version()
    for code in range(0, -10, -1):
        assert lib.rimp2_status_string(code)


def test_plan_create_rejects_bad_args_without_gpu(lib):
    """Host-side validation returns before touching the device."""
    from paper_2410_21888_gb300 import rimp2
    lib.rimp2_plan_create.argtypes = [ctypes.POINTER(rimp2.Frag), ctypes.c_int32, ctypes.c_int32,
                                      ctypes.POINTER(rimp2.Options), ctypes.POINTER(ctypes.c_void_p)]
    h = ctypes.c_void_p()
    assert lib.rimp2_plan_create(None, 1, 0, None, ctypes.byref(h)) == -1   # frags NULL
    fr = (rimp2.Frag * 1)()
    fr[0].nocc, fr[0].nvir, fr[0].naux = -1, 4, 4
    assert lib.rimp2_plan_create(fr, 1, 0, None, ctypes.byref(h)) == -1     # negative size
    fr[0].nocc = 2
    assert lib.rimp2_plan_create(fr, 1, 7, None, ctypes.byref(h)) == -8     # bad precision
    assert lib.rimp2_plan_create(fr, 1, 0, None, None) == -1                # out NULL


def test_binding_fails_loudly_without_gpu():
    import torch

    from paper_2410_21888_gb300 import rimp2
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(RuntimeError):
        rimp2.Plan([(2, 3, 4)])


def test_zvec_host_validation_without_gpu(lib):
    """rimp2_zvec_workspace_size and rimp2_zvec_solve check sizes, pointers and the
    workspace before any device call."""
    from paper_2410_21888_gb300 import rimp2
    lib.rimp2_zvec_workspace_size.argtypes = [ctypes.c_int32] * 4 + [ctypes.POINTER(ctypes.c_size_t)]
    lib.rimp2_zvec_solve.argtypes = [ctypes.POINTER(rimp2.ZvecArgs), ctypes.c_void_p,
                                     ctypes.c_size_t, ctypes.c_void_p]
    n = ctypes.c_size_t()
    assert lib.rimp2_zvec_workspace_size(100, 500, 1500, 0, ctypes.byref(n)) == 0
    small = n.value
    assert small > 100 * 100 * 1500 * 8            # holds the o*o*X exchange intermediate
    assert lib.rimp2_zvec_workspace_size(100, 500, 1500, 200, ctypes.byref(n)) == 0
    assert n.value > small                           # one work-queue counter per launch
    assert lib.rimp2_zvec_workspace_size(-1, 5, 5, 0, ctypes.byref(n)) == -1
    assert lib.rimp2_zvec_workspace_size(3, 5, 5, 0, None) == -1
    a = rimp2.ZvecArgs()
    a.nocc, a.nvir, a.naux = 3, 4, 5
    assert lib.rimp2_zvec_solve(None, None, 0, None) == -1
    assert lib.rimp2_zvec_solve(ctypes.byref(a), None, 0, None) == -1   # outputs missing
    fake = ctypes.c_void_p(256)                      # never dereferenced: rejected first
    a.Bf = a.eps = a.gamma = a.pij = a.pab = fake
    a.lp = a.lpp = a.dai = a.info = fake
    assert lib.rimp2_zvec_solve(ctypes.byref(a), None, 1 << 20, None) == -5   # no workspace
    assert lib.rimp2_zvec_solve(ctypes.byref(a), ctypes.c_void_p(4096), 16, None) == -5
    a.tol = -1.0
    assert lib.rimp2_zvec_solve(ctypes.byref(a), ctypes.c_void_p(4096), 1 << 30, None) == -1


def test_default_options_without_gpu(lib):
    """rimp2_default_options fills the struct the binding mirrors field by field: the
    SCS-MP2 weights (Grimme's 6/5 and 1/3) sit after the last integer option."""
    from paper_2410_21888_gb300 import rimp2
    lib.rimp2_default_options.argtypes = [ctypes.POINTER(rimp2.Options)]
    lib.rimp2_default_options.restype = None
    o = rimp2.Options()
    o.slices_g = 77
    lib.rimp2_default_options(ctypes.byref(o))
    assert o.use_graph == 1 and o.check_inputs == 1 and o.slices_g == 0
    assert o.scs_os == 6.0 / 5.0 and o.scs_ss == 1.0 / 3.0
