"""GPU tests of the split-precision (BF16 integer-slice, tcgen05) path.

1. The tensor-core slice GEMM alone against exact integer arithmetic: BF16 digits in
   [-64, 64] for the leading slice and [-256, 256] for the others, level sums
   2^(-9(p+q)) sum_k A_p B_q for p + q < s.  Levels 0 and 1 of each 512-long K chunk are
   exact integers in FP32 (|S_1| <= 512 * 2 * 2^6 * 2^8 = 2^24; higher levels too unless
   a partial sum passes 2^24); levels 0..2 are folded into a double-float accumulator
   exactly, levels >= 3 in FP32, so the result matches the exact value to ~2^-46 of the
   absolute digit products.
2. Fragments through rimp2_energy_grad(precision=BF16_SPLIT) against the FP64 oracle.
   Tolerances: energy within 1e-8 Eh per fragment; Gamma, P_ij, P_ab, pair energies
   within 1e-9 relative Frobenius (the accuracy target of the split path).
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import oracle
from paper_2410_21888_gb300 import rimp2, synth

pytestmark = pytest.mark.gpu

TOL_E_ABS = 1e-8
TOL_A = 1e-9


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def _hook():
    lib = rimp2.load()
    f = lib.rimp2_testing_slice_gemm_k
    f.argtypes = [ctypes.c_int32] * 7 + [ctypes.c_void_p] * 4
    f.restype = ctypes.c_int
    return f


def _exact_levels(A, B, s, chunk=512, bits=9):
    """sum_{p+q<s} 2^(-bits (p+q)) A_p B_q^T with exact int64 level sums, and the
    magnitude the kernel's rounding is relative to: sum over K chunks and levels of
    2^(-bits l) sum_k |A_p||B_q| (the usual dot-product error model)."""
    M, N, K = A.shape[1], B.shape[1], A.shape[2]
    out = np.zeros((M, N))
    mag = np.zeros((M, N))
    for k0 in range(0, max(K, 1), chunk):
        for l in range(s):
            lev = np.zeros((M, N), dtype=np.int64)
            lab = np.zeros((M, N), dtype=np.int64)
            for p in range(l + 1):
                a = A[p, :, k0:k0 + chunk].astype(np.int64)
                b = B[l - p, :, k0:k0 + chunk].astype(np.int64)
                lev += a @ b.T
                lab += np.abs(a) @ np.abs(b).T
            out += lev.astype(np.float64) * 2.0 ** (-bits * l)
            mag += lab.astype(np.float64) * 2.0 ** (-bits * l)
    return out, mag


@pytest.mark.parametrize("stage_k", [16, 32])
@pytest.mark.parametrize("M,N,K,s,seed", [
    (128, 96, 64, 2, 0),
    (128, 96, 32, 5, 1),
    (200, 150, 300, 5, 2),       # ragged M/N, one chunk with a partial K block
    (256, 192, 1500, 5, 7),      # three chunks, 1500 = the large-fragment naux
    (130, 97, 1000, 3, 3),       # two chunks in two accumulator sets (3 x 64 columns each)
    (64, 40, 33, 4, 4),          # partial tiles and a partial K block
    (300, 260, 700, 6, 5),       # six slices: one accumulator set (64-column tiles)
    (129, 70, 257, 8, 6),        # n_tile 64, eight slices
])
def test_slice_gemm_matches_exact_integer_products(M, N, K, s, seed, stage_k):
    rng = np.random.default_rng(seed)
    kpad = (K + 7) // 8 * 8
    A = rng.integers(-256, 257, size=(s, M, K))
    B = rng.integers(-256, 257, size=(s, N, K))
    A[0] = rng.integers(-64, 65, size=(M, K))   # the leading digit is two bits narrower
    B[0] = rng.integers(-64, 65, size=(N, K))
    if seed == 0:     # worst case for exactness: level 1 reaches 2^24 in each chunk
        A[:] = 256
        B[:] = -256
        A[0] = 64
        B[0] = -64
    Ap = np.zeros((s, M, kpad)); Ap[:, :, :K] = A
    Bp = np.zeros((s, N, kpad)); Bp[:, :, :K] = B
    Ad = torch.tensor(Ap, dtype=torch.bfloat16, device="cuda")
    Bd = torch.tensor(Bp, dtype=torch.bfloat16, device="cuda")
    assert torch.equal(Ad.float().cpu(), torch.tensor(Ap, dtype=torch.float32))
    C = torch.full((M, N), np.nan, dtype=torch.float64, device="cuda")
    rc = _hook()(M, N, K, kpad, s, stage_k, 0, Ad.data_ptr(), Bd.data_ptr(), C.data_ptr(),
                 torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    ref, mag = _exact_levels(A, B, s)
    got = C.cpu().numpy()
    assert np.all(np.isfinite(got))
    # an FP32 accumulator alone would err by ~2^-24 of mag and one wrong integer in
    # levels 0..2 by >= 2^-18 (absolute); demand 2^-44 of the absolute products
    bound = 2.0 ** -44 * (mag + 1.0)
    assert np.all(np.abs(got - ref) <= bound), float(np.max(np.abs(got - ref) - bound))


@pytest.mark.parametrize("M,N,K,s,seed", [
    (128, 64, 64, 8, 0),         # worst case magnitudes, one stage
    (200, 150, 1100, 8, 1),      # one 8192-long chunk, ragged
    (130, 64, 9000, 10, 4),      # two chunks, the first 8192 long: levels 0..4 near 2^23
    (130, 48, 700, 10, 2),       # ten slices, 48-column tiles
    (140, 40, 600, 16, 3),       # sixteen slices, 32-column tiles, one pipeline stage
])
def test_fp8_slice_gemm_matches_exact_integer_products(M, N, K, s, seed):
    """FP8 e4m3 digits in [-16, 16], 5-bit levels, K chunks of 8192: levels 0..4 of a chunk
    are exact sums (below 5 * 8192 * 2^8 < 2^24), higher ones within 2^-24 of the level."""
    rng = np.random.default_rng(seed)
    kpad = (K + 15) // 16 * 16
    A = rng.integers(-16, 17, size=(s, M, K))
    B = rng.integers(-16, 17, size=(s, N, K))
    if seed in (0, 4):
        A[:] = 16
        B[:] = -16
    Ap = np.zeros((s, M, kpad)); Ap[:, :, :K] = A
    Bp = np.zeros((s, N, kpad)); Bp[:, :, :K] = B
    Ad = torch.tensor(Ap, dtype=torch.float32).to(torch.float8_e4m3fn).cuda()
    Bd = torch.tensor(Bp, dtype=torch.float32).to(torch.float8_e4m3fn).cuda()
    assert torch.equal(Ad.float().cpu(), torch.tensor(Ap, dtype=torch.float32))
    C = torch.full((M, N), np.nan, dtype=torch.float64, device="cuda")
    rc = _hook()(M, N, K, kpad, s, 64, 1, Ad.data_ptr(), Bd.data_ptr(), C.data_ptr(),
                 torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    ref, mag = _exact_levels(A, B, s, chunk=8192, bits=5)
    got = C.cpu().numpy()
    bound = 2.0 ** -44 * (mag + 1.0)
    assert np.all(np.abs(got - ref) <= bound), float(np.max(np.abs(got - ref) - bound))


def check_split(out, ref, tol_e=TOL_E_ABS, tol_a=TOL_A):
    E = float(out["energy"].item())
    assert abs(E - ref["energy"]) <= tol_e, (E, ref["energy"], E - ref["energy"])
    for k in ("gamma", "pij", "pab", "epair"):
        g = out[k].detach().cpu().numpy()
        assert rel(g, ref[k]) <= tol_a, (k, rel(g, ref[k]))


@pytest.mark.parametrize("dims,seed", [
    ((10, 40, 150), 0),
    ((3, 5, 7), 2),
    ((2, 70, 33), 3),
    ((7, 13, 129), 4),
    ((13, 37, 17), 6),
    ((1, 1, 1), 1),
    ((5, 31, 1), 5),
    ((4, 130, 300), 7),      # nvir > 128: several M tiles in P_ab, ragged
    ((13, 333, 150), 8),     # Gamma's K (j,b) with a partial last K block
])
@pytest.mark.parametrize("mode", ["bf16-32", "bf16-16", "fp8", "fp8-16"])
def test_split_fragment_parity(dims, seed, mode):
    f = synth.fragment_inputs(*dims, seed=seed)
    ref = oracle.fragment(f.B, f.eo, f.ev)
    if mode == "fp8":
        out = rimp2.energy_grad(f.B, f.eo, f.ev, precision="fp8")
    elif mode == "fp8-16":
        out = rimp2.energy_grad(f.B, f.eo, f.ev, precision="fp8", slices_v=16, slices_t=16,
                                slices_g=16)
    else:
        out = rimp2.energy_grad(f.B, f.eo, f.ev, precision="bf16", stage_k=int(mode[5:]))
    check_split(out, ref)


@pytest.mark.parametrize("dims,seed", [((10, 40, 150), 0), ((13, 333, 150), 8)])
def test_split_fragment_parity_48_column_tiles(dims, seed):
    """n_tile 48: V and Gamma (5 slices) keep two accumulator sets in TMEM (2 x 240
    columns) and alternate between them chunk by chunk; P (6 slices) uses one set."""
    f = synth.fragment_inputs(*dims, seed=seed)
    check_split(rimp2.energy_grad(f.B, f.eo, f.ev, precision="bf16", n_tile=48),
                oracle.fragment(f.B, f.eo, f.ev))


def test_split_gamma_in_two_slabs():
    """nocc=100, nvir=250: Gamma's K = (j,b) = 100 x 256 padded elements is cut into two
    slabs that meet in Gamma by FP64 atomics."""
    f = synth.fragment_inputs(100, 250, 64, seed=12)
    check_split(rimp2.energy_grad(f.B, f.eo, f.ev, precision="bf16"),
                oracle.fragment(f.B, f.eo, f.ev))


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_split_padded_row_segments_in_a_dirty_workspace(precision):
    """nvir = 1120: the digit planes pad each (j, b) row segment to 1152 elements (the
    widest alignment under 3 % of padding), 32 more than the 32-wide amplitude tiles reach.
    Those padding columns enter the contractions of P_ab, P_ij and Gamma, so they must be
    written as zero on every call: the workspace is filled with NaN bytes first."""
    f = synth.fragment_inputs(2, 1120, 48, seed=13)
    ref = oracle.fragment(f.B, f.eo, f.ev)
    eng = rimp2.Engine([f.B.shape], precision=precision)
    eng.set_inputs([f])
    eng.workspace.fill_(0xFF)
    eng.run()
    torch.cuda.synchronize()
    eng.check_status()
    check_split(eng.views(0), ref)


def test_split_degenerate_sizes():
    for dims in [(3, 0, 5), (0, 4, 5), (3, 4, 0)]:
        f = synth.fragment_inputs(*dims, seed=0)
        out = rimp2.energy_grad(f.B, f.eo, f.ev, precision="bf16")
        assert float(out["energy"].item()) == 0.0
        for k in ("gamma", "pij", "pab"):
            assert torch.count_nonzero(out[k]).item() == 0


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_split_uneven_batch_matches_oracle(precision):
    s = synth.MonomerSystem(n_monomers=6, box=14.0, seed=0, nocc_range=(2, 5))
    polys = [(0,), (3,), (0, 1), (2, 4), (1, 3, 5), (0, 2, 4), (5,)]
    frags = [s.fragment(p) for p in polys]
    eng = rimp2.Engine([f.B.shape for f in frags], precision=precision)
    eng.set_inputs(frags)
    eng.run()
    torch.cuda.synchronize()
    eng.check_status()
    for k, f in enumerate(frags):
        check_split(eng.views(k), oracle.fragment(f.B, f.eo, f.ev))


def test_split_error_decreases_with_slices():
    f = synth.fragment_inputs(6, 30, 90, seed=11)
    ref = oracle.fragment(f.B, f.eo, f.ev)
    errs = []
    for s in (3, 4, 6):
        out = rimp2.energy_grad(f.B, f.eo, f.ev, precision="bf16", slices_v=s, slices_t=s,
                                slices_g=s)
        errs.append(rel(out["gamma"].cpu().numpy(), ref["gamma"]))
    assert errs[0] > errs[1] > errs[2] or errs[2] < 1e-12, errs


@pytest.mark.parametrize("precision,sgs", [("bf16", (2, 3, 4, 5)), ("fp8", (5, 6, 7, 8))])
def test_gamma_slices_change_gamma_only(precision, sgs):
    """Gamma contracts the leading s_g digit planes of Tt against its own B digits (one
    scale per aux index): its slice count moves Gamma's error alone.  The energy does not
    read digit planes (bit-identical); P_ab and P_ij read all s_t planes (equal up to the
    order of their FP64 atomic sums)."""
    f = synth.fragment_inputs(9, 70, 200, seed=13)
    ref = oracle.fragment(f.B, f.eo, f.ev)
    outs = [rimp2.energy_grad(f.B, f.eo, f.ev, precision=precision, slices_g=s) for s in sgs]
    errs = [rel(o["gamma"].cpu().numpy(), ref["gamma"]) for o in outs]
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] <= TOL_A, errs
    e0 = float(outs[0]["energy"].item())
    for o in outs[1:]:
        assert float(o["energy"].item()) == e0
        for k in ("pij", "pab"):
            a, b = o[k].cpu().numpy(), outs[0][k].cpu().numpy()
            assert rel(a, b) <= 1e-14, k


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_gamma_zero_rows_and_aux_columns(precision):
    """Zero rows (i,a) and a zero occupied block of B leave zero rows of V and T while Tt
    keeps its transposed terms; a zero aux column Q takes the exponent floor as its scale
    and gives an exactly zero Gamma column."""
    f = synth.fragment_inputs(6, 45, 120, seed=17)
    B = f.B.copy()
    B[2, 7, :] = 0.0
    B[:, :, 11] = 0.0
    B[4, :, :] = 0.0
    ref = oracle.fragment(B, f.eo, f.ev)
    out = rimp2.energy_grad(B, f.eo, f.ev, precision=precision)
    check_split(out, ref)
    g = out["gamma"].cpu().numpy().reshape(B.shape)
    assert np.all(g[:, :, 11] == 0.0)


def test_gamma_rows_of_very_different_size():
    """Virtual energies spread over three decades: rows (i,a) of T and Tt for high
    virtuals are orders of magnitude below the fragment's largest element, whose exponent
    sets the digit scale; the relative Frobenius errors, carried by the large rows, stay
    within the target."""
    rng = np.random.default_rng(23)
    o, v, X = 8, 96, 260
    eo = rng.uniform(-1.5, -0.3, o)
    ev = np.sort(np.exp(rng.uniform(np.log(0.05), np.log(80.0), v)))
    B = rng.normal(0.0, 0.05, (o, v, X))
    ref = oracle.fragment(B, eo, ev)
    check_split(rimp2.energy_grad(B, eo, ev, precision="bf16"), ref)


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_split_inputs_spanning_the_double_range(precision):
    """The slicing kernels split FP64 inputs into double-floats with integer instructions
    for |x| in [2^-74, 2^127) and fall back to FP64 conversions outside: B here mixes
    ordinary entries with entries near 1e-30 and exact zeros (some aux columns and rows
    tiny throughout, others mixed), and the results still match the oracle."""
    rng = np.random.default_rng(29)
    o, v, X = 6, 40, 90
    eo = rng.uniform(-1.5, -0.3, o)
    ev = rng.uniform(0.2, 3.0, v)
    B = rng.normal(0.0, 0.05, (o, v, X))
    B[:, :, 7] *= 1e-28            # an aux column far below 2^-74
    B[2, 5, :] *= 1e-29            # a row far below it
    B[1, 3, ::3] = 0.0             # exact zeros
    B[4, :, 11] = rng.normal(0.0, 1e-24, v)
    ref = oracle.fragment(B, eo, ev)
    check_split(rimp2.energy_grad(B, eo, ev, precision=precision), ref)


@pytest.mark.parametrize("dims", [(4, 60, 4000), (8, 40, 2000)])
@pytest.mark.parametrize("precision,sv,tol", [("bf16", 4, 2e-11), ("fp8", 8, 1e-12)])
def test_diagonal_dominated_energy_has_no_one_signed_error(dims, precision, sv, tol):
    """With naux >> nocc*nvir most of E comes from the diagonal V_ii(a,a) = sum_Q B^2,
    whose two operands have identical digits.  Were it taken from the truncated product
    triangle, the squared middle digit of the first dropped even level (BF16 4 slices:
    level 4, 2^-36; FP8 8 slices: level 8, 2^-40) would shift E by ~1e-10 and ~1e-11
    relative; from the FP64 row sum it stays at the random truncation level."""
    f = synth.fragment_inputs(*dims, seed=5)
    ref = oracle.fragment(f.B, f.eo, f.ev, want=())["energy"]
    out = rimp2.energy_grad(f.B, f.eo, f.ev, precision=precision, slices_v=sv,
                            want_gamma=False, want_p=False)
    assert abs(float(out["energy"].item()) - ref) <= tol * abs(ref)
