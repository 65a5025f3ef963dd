// Split-precision path of the RI-MP2 hot path (precision RIMP2_BF16_SPLIT).
//
// Per wave of fragments:
//   1. k_split_reset   per-fragment exponent slots
//   2. k_slice_b1      B -> balanced base-512 digits with one scale per row (i,a): the
//                      operands of V (Eq. MP2_ints); also d_m = e_i - e_a per row
//   3. k_bcol_max      max over (j,b) of |B^Q_jb| for every aux index Q
//   4. k_slice_b2      B -> digits with one scale per aux index Q, transposed to
//                      [Q][(j,b)]: the B operand of Gamma
//   5. split GEMM      V on the tensor cores, epilogue T = V / D kept as a double-float
//                      pair of planes, max |T| exponent
//   6. k_amp_split     Tt = 2T - T^T, pair energies e_ij (FP64 per pair), digits of Tt and
//                      T with one scale per fragment
//   7. energy reduce   FP64 compensated cross-pair sum (shared with the FP64 path)
//   8. zero P, split GEMMs for P_ab and P_ij, then for Gamma (Appendix Gamma, D^MP2_ab,
//      D^MP2_ij); Gamma contracts the leading s_g digit planes of Tt
#include <climits>
#include <cstring>
#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "split_path.cuh"

namespace rimp2 {

namespace {

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

// V tiles are walked in groups of this many rows (tile order, see decode_tile)
constexpr int kVGroupRows = 16;
// smallest K extent of a split-K piece of P_ab / P_ij
constexpr long long kMinPieceK = 4096;
// K extent of one Gamma slab (elements of the contracted (j,b) index).  Measured at
// nocc=100 nvir=500 naux=1500 (K = 51200): the Gamma/P launch takes 144.7 ms with slabs
// of 2048, 140.5 with 4096, 138.0 with 8192, 136.5 with 16384 and 138.5 without slabs.
constexpr long long kGammaSlabK = 16384;
int rup(int x, int m) { return (x + m - 1) / m * m; }

}  // namespace

// ------------------------------------------------------------------ device helpers

struct dfl { float h, l; };

__device__ __forceinline__ dfl d_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dfl d_fast(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ dfl d_add(dfl a, dfl b) {
  dfl s = d_two_sum(a.h, b.h);
  s.l += a.l + b.l;
  return d_fast(s.h, s.l);
}
__device__ __forceinline__ dfl d_neg(dfl a) { return {-a.h, -a.l}; }
// (__fmul_rn: the rounded product must not be contracted into d_fast's addition)
__device__ __forceinline__ dfl d_mul(dfl a, dfl b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
  return d_fast(p, e);
}
__device__ __forceinline__ dfl d_from(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}

__device__ __forceinline__ int find_sfd(const SplitFragDev* __restrict__ f, int n, long long t,
                                        int which) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const long long k = which == 0 ? f[mid].row_begin : which == 1 ? f[mid].b2_tile_begin
                        : which == 2 ? f[mid].pair_begin : f[mid].qblk_begin;
    if (k <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// One digit (an integer in [-2^(LB-1), 2^(LB-1)]) in the slice format: BF16 (LB = 9:
// its 8-bit significand holds every integer up to 256) or FP8 e4m3 (LB = 5); both
// represent these integers exactly.  The leading digit is HEAD bits narrower: a value x
// is sliced relative to 2^E with |x| <= 2^(E-1-HEAD) (BF16: d_0 in [-64, 64], which keeps
// the level-1 sums of a 512-long chunk within 2^24).
template <bool F8> struct Digit;
template <> struct Digit<false> {
  using T = __nv_bfloat16;
  static constexpr int LB = SG_LB_BF16;
  static constexpr int HEAD = SG_HEAD_BF16;
  __device__ static T enc(float d) { return __float2bfloat16_rn(d); }
};
template <> struct Digit<true> {
  using T = unsigned char;
  static constexpr int LB = SG_LB_FP8;
  static constexpr int HEAD = SG_HEAD_FP8;
  __device__ static T enc(float d) {
    return (T)__nv_cvt_float_to_fp8(d, __NV_SATFINITE, __NV_E4M3);
  }
};

// Four digits of one slice, packed for one store: BF16 digits are exact integers, so their
// bit patterns are the upper halves of the FP32 values; FP8 digits go through the e4m3
// conversion.
template <bool F8> struct Pack4;
template <> struct Pack4<false> {
  using T = uint2;
  __device__ static T pack(float d0, float d1, float d2, float d3) {
    return make_uint2(__byte_perm(__float_as_uint(d0), __float_as_uint(d1), 0x7632),
                      __byte_perm(__float_as_uint(d2), __float_as_uint(d3), 0x7632));
  }
};
template <> struct Pack4<true> {
  using T = uint32_t;
  __device__ static T pack(float d0, float d1, float d2, float d3) {
    return (uint32_t)Digit<true>::enc(d0) | ((uint32_t)Digit<true>::enc(d1) << 8) |
           ((uint32_t)Digit<true>::enc(d2) << 16) | ((uint32_t)Digit<true>::enc(d3) << 24);
  }
};

// One digit step of a normalised double-float (|xl| <= ulp(xh)/2) relative to the current
// scale: d = rint(xh) by the 1.5 * 2^23 shift (round to nearest even, |xh| <= 2^22);
// xh - d is exact and, when non-zero, a multiple of ulp(xh) >= 2|xl|, so Fast2Sum re-joins
// it with xl exactly; the remainder is scaled by 2^LB for the next digit.
template <int LB>
__device__ __forceinline__ float digit_step(float& xh, float& xl) {
  const float kShift = 12582912.f;
  const float d = __fsub_rn(__fadd_rn(xh, kShift), kShift);
  const float a = __fsub_rn(xh, d);
  const float s = __fadd_rn(a, xl);
  const float e = __fsub_rn(xl, __fsub_rn(s, a));
  xh = s * (float)(1 << LB);
  xl = e * (float)(1 << LB);
  return d;
}

// Two FP32 lanes in one 64-bit register for the packed f32x2 arithmetic of sm_100+
// (add/sub/mul.rn.f32x2: each lane rounds exactly like the scalar instruction).
typedef unsigned long long f2x;
__device__ __forceinline__ f2x f2_pack(float a, float b) {
  f2x r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(f2x r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ f2x f2_add(f2x a, f2x b) {
  f2x d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x f2_sub(f2x a, f2x b) {
  f2x d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x f2_mul(f2x a, f2x b) {
  f2x d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

__device__ __forceinline__ f2x f2_fma(f2x a, f2x b, f2x c) {
  f2x d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// digit_step on two elements at once, with the scaling by 2^LB folded into the Fast2Sum
// (seven packed operations instead of eight, bit-identical): with a = xh - d and
// s = a + xl as in digit_step, 2^LB s = RN(2^LB a + 2^LB xl) is one FMA; 2^LB (s - a) is
// exact, so the FMA 2^LB s - 2^LB a returns it unrounded, and 2^LB xl minus it is the
// exact error term 2^LB e
template <int LB>
__device__ __forceinline__ f2x digit_step2(f2x& xh, f2x& xl) {
  const f2x kShift = f2_pack(12582912.f, 12582912.f);
  const f2x kScale = f2_pack((float)(1 << LB), (float)(1 << LB));
  const f2x kNegScale = f2_pack(-(float)(1 << LB), -(float)(1 << LB));
  const f2x d = f2_sub(f2_add(xh, kShift), kShift);
  const f2x a = f2_sub(xh, d);
  const f2x l = f2_mul(xl, kScale);
  xh = f2_fma(a, kScale, l);
  xl = f2_sub(l, f2_fma(a, kNegScale, xh));
  return d;
}

// Digits of four consecutive elements (double-floats x[k] already scaled to the slice
// frame), one packed store per slice plane; the digit steps run on element pairs.  NS > 0:
// the plane count is NS, known at compile time (the loop unrolls; st is not read).
// STREAM: the stores carry the evict-first hint (the amplitude kernel's digit planes are
// far larger than L2 and are read back by later launches only).
template <bool F8, int NS = 0, bool STREAM = false>
__device__ __forceinline__ void put4(dfl x[4], int st, typename Digit<F8>::T* out,
                                     long long plane) {
  constexpr int LB = Digit<F8>::LB;
  using PT = typename Pack4<F8>::T;
  f2x h01 = f2_pack(x[0].h, x[1].h), l01 = f2_pack(x[0].l, x[1].l);
  f2x h23 = f2_pack(x[2].h, x[3].h), l23 = f2_pack(x[2].l, x[3].l);
  auto one = [&](int p) {
    float d0, d1, d2, d3;
    f2_unpack(digit_step2<LB>(h01, l01), d0, d1);
    f2_unpack(digit_step2<LB>(h23, l23), d2, d3);
    if constexpr (STREAM) __stcs((PT*)(out + p * plane), Pack4<F8>::pack(d0, d1, d2, d3));
    else *(PT*)(out + p * plane) = Pack4<F8>::pack(d0, d1, d2, d3);
  };
  if constexpr (NS > 0) {
#pragma unroll
    for (int p = 0; p < NS; ++p) one(p);
  } else {
    for (int p = 0; p < st; ++p) one(p);
  }
}

// 2^e as two normal powers of two (e clamped to [-252, 254])
__device__ __forceinline__ void pow2_factors(int e, float& s1, float& s2) {
  e = max(-252, min(254, e));
  s1 = __int_as_float(((e / 2) + 127) << 23);
  s2 = __int_as_float(((e - e / 2) + 127) << 23);
}

// ------------------------------------------------------------------ kernels

// One CTA per fragment: the atomicMax targets (max |T| exponent, column maxima of |B|)
__global__ void k_split_reset(const SplitFragDev* __restrict__ f, int n, Bases bs) {
  const SplitFragDev& F = f[blockIdx.x];
  char* ws = (char*)bs.ws;
  if (threadIdx.x == 0) ((unsigned*)(ws + F.scal))[1] = 0u;
  if (F.sg_out > 0) {
    unsigned long long* cm = (unsigned long long*)(ws + F.ecolm);
    for (int q = threadIdx.x; q < F.X; q += blockDim.x) cm[q] = 0ull;
  }
}

// One warp per row (i,a) of B: row exponent, digits of the V operand, d_m and the diagonal
// V_ii(a,a) = sum_Q (B^Q_ia)^2 in FP64.  The diagonal is the one element of V whose two operands have the same
// digits: there the truncated triangle's first dropped even level holds the square of
// the middle digit, an error of one sign that does not average out; the epilogue takes
// this FP64 value instead.
template <bool F8>
__global__ void __launch_bounds__(256)
k_slice_b1(const SplitFragDev* __restrict__ f, int nf, long long rows, int sv, Bases bs) {
  using DT = typename Digit<F8>::T;
  const long long gr = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (gr >= rows) return;
  const SplitFragDev& F = f[find_sfd(f, nf, gr, 0)];
  const int r = (int)(gr - F.row_begin);
  const double* x = bs.B + F.b_off + (long long)r * F.X;
  unsigned long long mx = 0;   // max |x| as bits
  double ss = 0.0;
  for (int q = lane; q < F.X; q += 32) {
    const double xq = x[q];
    mx = max(mx, abs_bits(xq));
    ss = fma(xq, xq, ss);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    ss += __shfl_xor_sync(0xffffffffu, ss, off);
  }
  const int E = mx > 0 ? ilogb_bits(mx) + 2 + Digit<F8>::HEAD : -1000;
  char* ws = (char*)bs.ws;
  const long long plane = (long long)F.o * F.v * F.xpad;
  DT* out = (DT*)(ws + F.bs1) + (long long)r * F.xpad;
  float s1, s2;
  pow2_factors(Digit<F8>::LB - E, s1, s2);
  // four consecutive elements a lane, one packed store per plane (elements in [X, xpad)
  // get zero digits; the V operand's tensor map ends at X)
  for (int q0 = 4 * lane; q0 < F.X; q0 += 128) {
    dfl xs[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float h, l;
      split_to_df(q0 + k < F.X ? x[q0 + k] : 0.0, h, l);
      xs[k] = {(h * s1) * s2, (l * s1) * s2};
    }
    put4<F8>(xs, sv, out + q0, plane);
  }
  if (lane == 0) {
    ((int*)(ws + F.erow))[r] = E;
    const int i = r / F.v, a = r - i * F.v;
    const dfl d = d_from(bs.eps[F.eo_off + i] - bs.eps[F.ev_off + a]);
    ((float2*)(ws + F.drow))[r] = make_float2(d.h, d.l);
    const dfl vd = d_from(ss);
    ((float2*)(ws + F.vdrow))[r] = make_float2(vd.h, vd.l);
  }
}

// Column maxima of B for Gamma's B operand: max over rows (j,b) of |B^Q_jb| for every aux
// index Q.  One CTA per 32 aux indices x 256 rows (lane: Q, warp: every 8th row), FP64
// bits combined by atomicMax (non-negative doubles order like their bit patterns).
__global__ void __launch_bounds__(256)
k_bcol_max(const SplitFragDev* __restrict__ f, int nf, Bases bs) {
  __shared__ unsigned long long red[8][32];   // |B| maxima as bits
  const long long gb = blockIdx.x;
  const SplitFragDev& F = f[find_sfd(f, nf, gb, 3)];
  const long long lb = gb - F.qblk_begin;
  const int nqb = (F.X + 31) / 32;
  const int qb = (int)(lb % nqb), rc = (int)(lb / nqb);
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int Q = qb * 32 + lane;
  const int r0 = rc * 256, r1 = min(F.o * F.v, r0 + 256);
  unsigned long long mx = 0;
  if (Q < F.X) {
    const double* x = bs.B + F.b_off + Q;
#pragma unroll 8
    for (int r = r0 + g; r < r1; r += 8) mx = max(mx, abs_bits(x[(long long)r * F.X]));
  }
  red[g][lane] = mx;
  __syncthreads();
  if (g == 0) {
    for (int k = 1; k < 8; ++k) mx = max(mx, red[k][lane]);
    if (Q < F.X && mx > 0) atomicMax((unsigned long long*)((char*)bs.ws + F.ecolm) + Q, mx);
  }
}

// Gamma's B operand: Bs2[p][Q][c], c = j*vpad + b (zero for b >= nvir), one scale
// 2^E_Q per aux index, E_Q = ilogb(max_(j,b) |B^Q_jb|) + 2 + HEAD (also stored for the GEMM
// epilogue).  Tiles of 32 aux indices x 128 columns c transposed through shared memory;
// each thread then writes four consecutive c of one Q, one packed store per plane.
template <bool F8>
__global__ void __launch_bounds__(256)
k_slice_b2(const SplitFragDev* __restrict__ f, int nf, int st, Bases bs) {
  using DT = typename Digit<F8>::T;
  __shared__ double tile[128][33];
  const long long gt = blockIdx.x;
  const SplitFragDev& F = f[find_sfd(f, nf, gt, 1)];
  const long long lt = gt - F.b2_tile_begin;
  const int RL = F.o * F.vpad;
  const int ntc = (RL + 127) / 128;
  const int tq = (int)(lt / ntc), tc = (int)(lt % ntc);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const double* B = bs.B + F.b_off;
  for (int r = ty; r < 128; r += 8) {
    const int c = tc * 128 + r, Q = tq * 32 + tx;
    double val = 0.0;
    if (c < RL && Q < F.X) {
      const int j = c / F.vpad, b = c - j * F.vpad;
      if (b < F.v) val = B[((long long)j * F.v + b) * F.X + Q];
    }
    tile[r][tx] = val;
  }
  __syncthreads();
  char* ws = (char*)bs.ws;
  const unsigned long long* cm = (const unsigned long long*)(ws + F.ecolm);
  int* ec = (int*)(ws + F.ecol);
  const long long plane = (long long)F.X * F.ldd;
  DT* out = (DT*)(ws + F.bs2);
  const int qi = threadIdx.x >> 3, cg = threadIdx.x & 7;
  const int Q = tq * 32 + qi;
  if (Q >= F.X) return;
  const int E = cm[Q] > 0 ? ilogb_bits(cm[Q]) + 2 + Digit<F8>::HEAD : -1000;
  if (tc == 0 && cg == 0) ec[Q] = E;
  float s1, s2;
  pow2_factors(Digit<F8>::LB - E, s1, s2);
#pragma unroll
  for (int k4 = 0; k4 < 4; ++k4) {
    const int cl = k4 * 32 + cg * 4, c = tc * 128 + cl;   // RL is a multiple of 4
    if (c >= RL) break;
    dfl xs[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float h, l;
      split_to_df(tile[cl + k][qi], h, l);
      xs[k] = {(h * s1) * s2, (l * s1) * s2};
    }
    put4<F8>(xs, st, out + (long long)Q * F.ldd + c, plane);
  }
}

// One CTA per ordered pair (i, j), i-major, so that the CTAs in flight fill the same rows
// of the digit planes.  The CTA writes the (i,j) block only; it reads the stored block
// (min(i,j), max(i,j)) of the double-float T planes (rows (i,a), columns j*vpadt + b;
// T_ij(a,b) = T_ji(b,a)) in pairs of 32 x 32 tiles (ta <= tb): X = tile (ta, tb) and
// Y = tile (tb, ta), 16-byte loads prefetched into registers while the previous pair is
// processed.  Every thread forms, for one row and four consecutive columns of the output
// tiles (ta, tb) and (tb, ta), Tt = 2T - T^T and the digits of T and Tt (one scale per
// fragment each; one packed store per slice; columns in [nvir, vpad) get zero digits).
// CTAs with i <= j also accumulate
// the pair energy e_ij = sum_ab Tt_ij(a,b) V_ij(a,b) (V = T D) and its opposite-spin
// part sum_ab T_ij(a,b) V_ij(a,b) in double-float (D from the double-float row terms
// d_m = e_i - e_a).
template <bool F8>
__global__ void __launch_bounds__(256, 3)
k_amp_split(const SplitFragDev* __restrict__ f, int nf, int st, Bases bs) {
  using DT = typename Digit<F8>::T;
  constexpr int LB = Digit<F8>::LB;
  // hi and lo parts of the tile pair in separate planes: with rows of 33 floats both the
  // row-wise and the transposed reads of a warp (4 rows x 8 column groups) hit 32 banks
  __shared__ float Xh[32][33], Xl[32][33], Yh[32][33], Yl[32][33];
  __shared__ float red_h[8], red_l[8], ros_h[8], ros_l[8];
  const int tid = threadIdx.x, r = tid >> 3, c0 = (tid & 7) * 4;
  const long long gp = blockIdx.x;
  const SplitFragDev& F = f[find_sfd(f, nf, gp, 2)];
  const int v = F.v, o = F.o, vpad = F.vpad;
  const int i = (int)((gp - F.pair_begin) / o), j = (int)((gp - F.pair_begin) % o);
  const bool tr = i > j;                  // the stored block is (j, i)
  const int i0 = tr ? j : i, j0 = tr ? i : j;
  const long long ldd = F.ldd, ldt = F.ldt;
  st = F.st_out;              // Tt digit planes (0: energy only)
  const int stt = F.st_t;     // T digit planes (0: no P)
  // BF16: the usual plane count (6) unrolled; FP8's ten planes stay a loop (unrolled,
  // they cost more registers than the loop saves: 33.4 against 32.3 ms at nocc=100 nvir=500 naux=1500)
  constexpr int NS = F8 ? 0 : 6;
  const bool ns = NS > 0 && st == NS && stt == NS;
  char* ws = (char*)bs.ws;
  const float* Th = (const float*)(ws + F.thi);
  const float* Tl = (const float*)(ws + F.tlo);
  const float2* __restrict__ dr = (const float2*)(ws + F.drow);
  const unsigned emax = *(const unsigned*)(ws + F.scal + 4);
  float s1t, s2t, s1tt, s2tt;   // 2^(LB - E) as two normal factors, for T and Tt
  // |T| < 2^(emax - 126) and |Tt| <= 3 max |T| < 2^(emax - 124): the scales keep both
  // within 2^(E - 2 - HEAD) and 2^(E - 1 - HEAD)
  constexpr int HEAD = Digit<F8>::HEAD;
  pow2_factors(LB - ((int)emax - 124 + HEAD), s1t, s2t);
  pow2_factors(LB - ((int)emax - 123 + HEAD), s1tt, s2tt);
  DT* tts = (DT*)(ws + F.tts);
  DT* ts = (DT*)(ws + F.ts);
  const long long plane = (long long)o * v * ldd;
  const long long rowI = (long long)i * v, rowJ = (long long)j * v;      // output rows, D terms
  const long long colJ = (long long)j * vpad;                            // output columns
  const long long rowS = (long long)i0 * v, colS = (long long)j0 * F.vpadt; // stored T block
  const int nt = (v + 31) / 32;
  dfl e_acc = {0.f, 0.f}, e_os = {0.f, 0.f};   // pair energy and its opposite-spin part

  float4 xh, xl, yh, yl;
  auto load = [&](int ta, int tb) {
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    xh = xl = yh = yl = z;
    const int ax = ta * 32 + r, bx = tb * 32 + c0;
    if (ax < v && bx < F.vpadt) {
      const long long ix = (rowS + ax) * ldt + colS + bx;
      xh = __ldg((const float4*)(Th + ix));
      xl = __ldg((const float4*)(Tl + ix));
    }
    const int ay = tb * 32 + r, by = ta * 32 + c0;
    if (ay < v && by < F.vpadt) {
      const long long iy = (rowS + ay) * ldt + colS + by;
      yh = __ldg((const float4*)(Th + iy));
      yl = __ldg((const float4*)(Tl + iy));
    }
  };

  // one output tile row segment: t_k and its transposed partner y_k for the four columns
  // col0 + k (local column index lc0 + k of the output block), written at global row orow
  auto emit = [&](const dfl t_in[4], const dfl y_in[4], long long orow, long long ocol0, int lc0,
                  bool energy, long long drow_r, long long drow_c0) {
    dfl t[4], tt[4];
    float2 dm = make_float2(0.f, 0.f), dn[4];
    if (energy) {   // the D terms of the row and the four columns, issued together
      dm = dr[drow_r];
#pragma unroll
      for (int k = 0; k < 4; ++k) dn[k] = lc0 + k < v ? dr[drow_c0 + k] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const bool ok = lc0 + k < v;
      t[k] = ok ? t_in[k] : dfl{0.f, 0.f};
      tt[k] = ok ? d_add({2.f * t_in[k].h, 2.f * t_in[k].l}, d_neg(y_in[k])) : dfl{0.f, 0.f};
      if (energy && ok) {
        const dfl D = d_add({dm.x, dm.y}, {dn[k].x, dn[k].y});
        const dfl V = d_mul(t[k], D);
        e_acc = d_add(e_acc, d_mul(tt[k], V));
        e_os = d_add(e_os, d_mul(t[k], V));
      }
    }
    if (st == 0) return;
    const long long o_ = orow * ldd + ocol0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      t[k] = {(t[k].h * s1t) * s2t, (t[k].l * s1t) * s2t};
      tt[k] = {(tt[k].h * s1tt) * s2tt, (tt[k].l * s1tt) * s2tt};
    }
    if (ns) {
      put4<F8, NS, true>(t, stt, ts + o_, plane);
      put4<F8, NS, true>(tt, st, tts + o_, plane);
    } else {
      put4<F8, 0, true>(t, stt, ts + o_, plane);
      put4<F8, 0, true>(tt, st, tts + o_, plane);
    }
  };

  int ta = 0, tb = 0;
  if (nt > 0) load(0, 0);
  while (ta < nt) {
    __syncthreads();   // the previous pair is no longer read from shared memory
    Xh[r][c0 + 0] = xh.x; Xh[r][c0 + 1] = xh.y; Xh[r][c0 + 2] = xh.z; Xh[r][c0 + 3] = xh.w;
    Xl[r][c0 + 0] = xl.x; Xl[r][c0 + 1] = xl.y; Xl[r][c0 + 2] = xl.z; Xl[r][c0 + 3] = xl.w;
    Yh[r][c0 + 0] = yh.x; Yh[r][c0 + 1] = yh.y; Yh[r][c0 + 2] = yh.z; Yh[r][c0 + 3] = yh.w;
    Yl[r][c0 + 0] = yl.x; Yl[r][c0 + 1] = yl.y; Yl[r][c0 + 2] = yl.z; Yl[r][c0 + 3] = yl.w;
    __syncthreads();
    const int cta = ta, ctb = tb;
    if (++tb == nt) { ++ta; tb = ta; }
    if (ta < nt) load(ta, tb);   // next pair in flight while this one is processed

    dfl t4[4], y4[4];
    // output tile (cta, ctb): T_ij(a,b) = X[r][c] (stored (i,j)) or Y[c][r] (stored (j,i));
    // the partner T_ij(b,a) is the other one of the two
    {
      const int la = cta * 32 + r, lb = ctb * 32 + c0;
      if (la < v && lb < vpad) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const dfl x = {Xh[r][c0 + k], Xl[r][c0 + k]}, y = {Yh[c0 + k][r], Yl[c0 + k][r]};
          t4[k] = tr ? y : x;
          y4[k] = tr ? x : y;
        }
        emit(t4, y4, rowI + la, colJ + lb, lb, !tr, rowI + la, rowJ + lb);
      }
    }
    if (cta != ctb) {   // output tile (ctb, cta): Y[r][c] (stored (i,j)) or X[c][r]
      const int la = ctb * 32 + r, lb = cta * 32 + c0;
      if (la < v && lb < vpad) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const dfl x = {Yh[r][c0 + k], Yl[r][c0 + k]}, y = {Xh[c0 + k][r], Xl[c0 + k][r]};
          t4[k] = tr ? y : x;
          y4[k] = tr ? x : y;
        }
        emit(t4, y4, rowI + la, colJ + lb, lb, !tr, rowI + la, rowJ + lb);
      }
    }
  }
  // digit columns [32 nt, vpad) that no tile reaches (the padded row segment is longer
  // than the tiles, e.g. nvir = 1500 with 1536-element segments): zero in every row
  if (st > 0 && vpad > nt * 32) {
    using U4 = uint4;
    const int w16 = (vpad - nt * 32) * (int)sizeof(DT) / 16;   // 16-byte units per row
    const long long units = (long long)(st + stt) * v * w16;
    for (long long u = tid; u < units; u += blockDim.x) {
      long long x = u;
      const int c = (int)(x % w16); x /= w16;
      const int a = (int)(x % v);
      const int p = (int)(x / v);
      DT* base = p < stt ? ts + p * plane : tts + (p - stt) * plane;
      DT* row = base + (rowI + a) * ldd + colJ + nt * 32;
      ((U4*)row)[c] = make_uint4(0u, 0u, 0u, 0u);
    }
  }
  // pair energy: warp, then block, in double-float; one FP64 value per pair
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const dfl o2 = {__shfl_down_sync(0xffffffffu, e_acc.h, off),
                    __shfl_down_sync(0xffffffffu, e_acc.l, off)};
    e_acc = d_add(e_acc, o2);
    const dfl o3 = {__shfl_down_sync(0xffffffffu, e_os.h, off),
                    __shfl_down_sync(0xffffffffu, e_os.l, off)};
    e_os = d_add(e_os, o3);
  }
  if ((tid & 31) == 0) {
    red_h[tid >> 5] = e_acc.h; red_l[tid >> 5] = e_acc.l;
    ros_h[tid >> 5] = e_os.h; ros_l[tid >> 5] = e_os.l;
  }
  __syncthreads();
  if (tid == 0 && !tr) {
    double e = 0.0, eos = 0.0;
    for (int w = 0; w < 8; ++w) {
      e += (double)red_h[w] + (double)red_l[w];
      eos += (double)ros_h[w] + (double)ros_l[w];
    }
    double* ep = (double*)(ws + F.ep);
    ep[(long long)i * o + j] = e;
    ep[(long long)j * o + i] = e;
    ep += (long long)o * o;          // opposite-spin pair energies
    ep[(long long)i * o + j] = eos;
    ep[(long long)j * o + i] = eos;
  }
}

// ------------------------------------------------------------------ host

namespace {

// Tile shapes a launch of `slices` digit planes can take: the default one (n_tile_first,
// 0: the kernel's default width) first, then every other (n_tile, K per stage) the kernel
// is built for whose level accumulators fit the 512 TMEM columns (BF16: 48..96 columns x
// K 32 or 16; FP8: 32..64 columns); non-zero n_tile / stage_k options pin that dimension.
std::vector<SplitLaunch> shape_candidates(int slices, bool fp8, int n_tile_first, int stage_k,
                                          int n_tile) {
  std::vector<SplitLaunch> c;
  c.push_back(split_launch_config(slices, stage_k ? stage_k : 32, n_tile_first, fp8));
  auto add = [&](const SplitLaunch& x) {
    for (const auto& y : c)
      if (y.n_tile_max == x.n_tile_max && y.bk == x.bk) return;
    c.push_back(x);
  };
  if (fp8) {
    for (int nt : {64, 48, 32})
      if ((n_tile == 0 || n_tile == nt) && slices * nt <= 512) {
        const SplitLaunch x = split_launch_config(slices, 64, nt, true);
        if (x.n_tile_max == nt) add(x);
      }
  } else {
    for (int bk : {32, 16})
      for (int nt : {64, 48, 80, 96})
        if ((stage_k == 0 || stage_k == bk) && (n_tile == 0 || n_tile == nt)) {
          const SplitLaunch x = split_launch_config(slices, bk, nt, false);
          if (x.n_tile_max == nt && slices * nt <= 512) add(x);
        }
  }
  return c;
}

}  // namespace

void split_set_shapes(SplitPlan& sp, int iv, int it, int ig) {
  auto pick = [](const std::vector<SplitLaunch>& c, int i) {
    return std::max(0, std::min(i, (int)c.size() - 1));
  };
  sp.shape_v = pick(sp.cand_v, iv);
  sp.shape_t = pick(sp.cand_t, it);
  // Gamma with P's slice count runs in P's launch: it must take that launch's shape
  sp.shape_g = sp.slices_g == sp.slices_t ? sp.shape_t : pick(sp.cand_g, ig);
  sp.cfg_v = sp.cand_v[sp.shape_v];
  sp.cfg_t = sp.cand_t[sp.shape_t];
  sp.cfg_g = sp.cand_g[sp.shape_g];
}

int split_plan_init(SplitPlan& sp, int precision, const rimp2_options& opt) {
  sp.precision = precision;
  sp.slices_v = opt.slices_v;
  sp.slices_t = opt.slices_t;
  sp.slices_g = opt.slices_g;
  sp.fp8 = precision == RIMP2_FP8_SPLIT;
  // Default tile widths per launch (BF16; an n_tile option overrides them): V takes 48
  // columns when two accumulator sets then fit TMEM, so that its heavy epilogue (T = V/D,
  // two stores per element) overlaps the next chunk's MMAs; Gamma, with K = nocc x nvir,
  // takes 80, whose wider B tiles cut its operand traffic; P_ab / P_ij keep 64.  Measured
  // by the autotuner at nocc=100 nvir=500 naux=1500 (5 / 6 / 5 slices): V 44.8 ms against
  // 45.8 at 64 columns, Gamma 74 against 80 ms.
  int nv = opt.n_tile, ng = opt.n_tile;
  if (!sp.fp8 && opt.n_tile == 0) {
    nv = 2 * sp.slices_v * 48 <= 512 ? 48 : 0;
    ng = sp.slices_g * 80 <= 512 && sp.slices_g != sp.slices_t ? 80 : 0;
  }
  sp.cand_v = shape_candidates(sp.slices_v, sp.fp8, nv, opt.stage_k, opt.n_tile);
  sp.cand_t = shape_candidates(sp.slices_t, sp.fp8, opt.n_tile, opt.stage_k, opt.n_tile);
  sp.cand_g = shape_candidates(sp.slices_g, sp.fp8, ng, opt.stage_k, opt.n_tile);
  split_set_shapes(sp, 0, 0, 0);
  sp.grid = split_gemm_grid();
  if (split_gemm_prepare() != cudaSuccess) { cudaGetLastError(); return RIMP2_ERR_CUDA; }
  sp.ready = true;
  return RIMP2_OK;
}

void split_plan_release(SplitPlan&) {}

namespace {

struct Layout {
  size_t bs1, bs2, erow, drow, vdrow, thi, tlo, tts, ts, ecolm, ecol, ep, scal, total;
};

// element size of the digit planes and the padding that keeps every row 16-byte aligned
size_t esz_of(const SplitPlan& sp) { return sp.fp8 ? 1 : 2; }
int padg(const SplitPlan& sp) { return sp.fp8 ? 16 : 8; }

// Padded extent of a digit-row segment of n elements: the widest alignment up to 128 bytes
// of digits that costs under 3 % of padding (so that row segments start on L2 line or
// sector boundaries), at least the 16-byte TMA stride rule.
int pad_extent(const SplitPlan& sp, int n) {
  const int esz = (int)esz_of(sp);
  for (int a = 128 / esz; a > padg(sp); a /= 2) {
    const int r = rup(n, a);
    if ((long long)(r - n) * 100 < 3LL * n) return r;
  }
  return rup(n, padg(sp));
}

// Row stride of a plane whose rows hold n elements of esz bytes: the smallest odd multiple of
// 128 bytes that holds them.  Tiles that run side by side read rows a fixed number of rows
// apart; with strides that are multiples of large powers of two their addresses coincide
// modulo 4 KB and crowd the same L2 slices.
long long row_stride(long long n, long long esz) {
  long long lines = (n * esz + 127) / 128;
  if ((lines & 1) == 0) ++lines;
  return lines * 128 / esz;
}

Layout frag_layout(const SplitPlan& sp, const rimp2_frag& f) {
  const size_t o = f.nocc, v = f.nvir, X = f.naux;
  const size_t esz = esz_of(sp);
  const size_t ov = o * v, vpad = pad_extent(sp, (int)v), xpad = pad_extent(sp, (int)X), RL = o * vpad;
  // digit planes exist only when an output needs them: T and Tt for P_ab and P_ij; Tt
  // (its leading s_g planes) and B^T with one scale per aux index for Gamma
  const bool want_p = f.pij_off >= 0 || f.pab_off >= 0;
  const size_t st_g = f.gamma_off >= 0 ? (size_t)sp.slices_g : 0;
  const size_t st_t = want_p ? (size_t)sp.slices_t : 0;
  const size_t st_tt = std::max(st_t, st_g);
  Layout L{};
  size_t off = 0;
  L.bs1 = off; off += al256((size_t)sp.slices_v * ov * xpad * esz);
  const size_t ldd = (size_t)row_stride((long long)RL, (long long)esz);
  const size_t ldt = (size_t)row_stride((long long)o * rup((int)v, 32), 4);
  L.bs2 = off; off += al256(st_g * X * ldd * esz);
  L.erow = off; off += al256(ov * 4);
  L.drow = off; off += al256(ov * 8);
  L.vdrow = off; off += al256(ov * 8);
  L.thi = off; off += al256(ov * ldt * 4);   // T planes: rows (i,a), columns j*vpadt + b
  L.tlo = off; off += al256(ov * ldt * 4);
  L.tts = off; off += al256(st_tt * ov * ldd * esz);
  L.ts = off; off += al256(st_t * ov * ldd * esz);
  L.ecolm = off; off += al256(X * 8);
  L.ecol = off; off += al256(X * 4);
  L.ep = off; off += al256(2 * o * o * 8);   // pair energies, opposite-spin pair energies
  L.scal = off; off += 256;
  L.total = off;
  return L;
}

void choose_split_k(SplitProb& P, int grid, int mul) {
  const long long tiles = (long long)P.tiles_m * P.tiles_n;
  long long want = std::max(1LL, ((long long)mul * grid + tiles - 1) / tiles);
  want = std::min<long long>(want, std::max(1, P.k1_count));
  int chunk = (int)((P.k1_count + want - 1) / want);
  if (chunk < 1) chunk = 1;
  P.k1_chunk = chunk;
  P.ksplit = std::max(1, (P.k1_count + chunk - 1) / chunk);
}

// Tensor-core FLOPs one problem issues: 2 x 128 x n_tile x K per computed tile (the
// skip rules of the kernel's tile decoder: V keeps tiles with some row >= some column,
// symmetric accumulations tiles with some row <= some column) x the digit products.
double prob_mma_flops(const SplitProb& P, int slices, int bk) {
  long long tiles = 0;
  for (int tm = 0; tm < P.tiles_m; ++tm)
    for (int tn = 0; tn < P.tiles_n; ++tn) {
      bool skip = P.kind == PK_V && tm * SG_BM + SG_BM - 1 < tn * P.n_tile;
      if (P.sym) skip = tm * SG_BM > tn * P.n_tile + P.n_tile - 1;
      tiles += !skip;
    }
  const double K = (double)P.k1_count * P.k0_blocks * bk;
  return (double)tiles * 2.0 * SG_BM * P.n_tile * K * (slices * (slices + 1) / 2);
}

void finish(std::vector<SplitProb>& v, long long& total) {
  std::stable_sort(v.begin(), v.end(), [](const SplitProb& a, const SplitProb& b) {
    return (double)a.k0_blocks * a.k1_chunk > (double)b.k0_blocks * b.k1_chunk;
  });
  total = 0;
  for (auto& P : v) {
    P.tile_begin = total;
    total += P.ntiles;
  }
}

}  // namespace

size_t split_frag_ws_bytes(const SplitPlan& sp, const rimp2_frag& f) {
  return frag_layout(sp, f).total;
}

int split_build_wave(SplitPlan& sp, const rimp2_frag* frags, const std::vector<int>& members,
                     const double* B, void* ws, std::vector<FragDev>& fdev, SplitWave& w,
                     long long& total_pairs, long long& max_b) {
  (void)B;
  char* wsb = (char*)ws;
  size_t off = 0;
  long long pairs = 0, rows = 0, b2t = 0, qbl = 0;
  const int sv = sp.slices_v, st = sp.slices_t, sgl = sp.slices_g;
  // Gamma with P's slice count joins P's launch and so takes its tile shape
  const SplitLaunch& cg = sgl == st ? sp.cfg_t : sp.cfg_g;
  const int NTv = sp.cfg_v.n_tile_max, NTt = sp.cfg_t.n_tile_max, NTg = cg.n_tile_max;
  const int BKv = sp.cfg_v.bk, BKt = sp.cfg_t.bk, BKg = cg.bk;
  // split-K target of P_ab / P_ij in multiples of the grid: finer pieces keep the tiles of
  // one occupied-index range closer together in time (their operand rows stay in L2);
  // measured at nocc=100 nvir=500 naux=1500: the P launch 33.3 ms at 2x, 32.2 at 8x, 31.6
  // at 16x; at nocc=42 nvir=168 naux=630: 0.73, 0.65, 0.68 ms
  const int split_mul = sp.variant == 2 ? 16 : 8;
  const bool pij_direct = sp.variant == 1;
  // exponents of the Tt and T digit planes: the stored max |T| exponent plus these (the
  // amplitude kernel's scales)
  const int head = sp.fp8 ? SG_HEAD_FP8 : SG_HEAD_BF16;
  const int kTtAdd = -123 + head, kTAdd = -124 + head;
  w.want_gamma = false;
  for (int idx : members) {
    const rimp2_frag& f = frags[idx];
    const Layout L = frag_layout(sp, f);
    const int o = f.nocc, v = f.nvir, X = f.naux;
    const int ov = o * v, vpad = pad_extent(sp, v), xpad = pad_extent(sp, X), RL = o * vpad;
    const uint64_t E2 = esz_of(sp);
    const int vpadt = rup(v, 32);
    const long long ldd = row_stride(RL, (long long)E2), ldt = row_stride((long long)o * vpadt, 4);
    SplitFragDev s{};
    s.o = o; s.v = v; s.X = X; s.idx = idx; s.vpad = vpad; s.xpad = xpad;
    s.ldd = ldd; s.ldt = ldt; s.vpadt = vpadt;
    const bool g = f.gamma_off >= 0 && X > 0 && ov > 0;
    const bool want_p = f.pij_off >= 0 || f.pab_off >= 0;
    s.st_t = want_p ? st : 0;
    s.sg_out = g ? sgl : 0;
    s.st_out = std::max(s.st_t, s.sg_out);
    s.b_off = f.b_off; s.eo_off = f.eo_off; s.ev_off = f.ev_off;
    s.bs1 = off + L.bs1; s.bs2 = off + L.bs2; s.erow = off + L.erow; s.drow = off + L.drow;
    s.vdrow = off + L.vdrow;
    s.thi = off + L.thi; s.tlo = off + L.tlo; s.tts = off + L.tts; s.ts = off + L.ts;
    s.ecolm = off + L.ecolm; s.ecol = off + L.ecol;
    s.ep = off + L.ep; s.scal = off + L.scal;
    s.pair_begin = pairs; s.row_begin = rows; s.b2_tile_begin = b2t; s.qblk_begin = qbl;
    pairs += (long long)o * o;   // amplitude stage: one CTA per ordered pair
    rows += ov;
    if (g) {
      b2t += (long long)((X + 31) / 32) * ((RL + 127) / 128);
      qbl += (long long)((X + 31) / 32) * ((ov + 255) / 256);
      w.want_gamma = true;
    }
    w.sfd.push_back(s);
    // the shared FP64 kernels (checks, energy reduce, zeroing) use FragDev
    FragDev d{};
    d.o = o; d.v = v; d.X = X; d.idx = idx;
    d.b_off = f.b_off; d.eo_off = f.eo_off; d.ev_off = f.ev_off;
    d.t_off = d.tt_off = -1;
    d.ep_off = (long long)(s.ep / 8);
    d.epos_off = d.ep_off + (long long)o * o;
    d.gamma_off = f.gamma_off; d.pij_off = f.pij_off; d.pab_off = f.pab_off;
    d.epair_off = f.epair_off; d.pair_begin = s.pair_begin;
    fdev.push_back(d);
    max_b = std::max<long long>(max_b, (long long)ov * X);
    off += L.total;
    if (ov == 0) continue;

    // V over rows (i,a) x (j,b), K = Q
    {
      SplitProb P{};
      P.kind = PK_V; P.frag = idx;
      P.M = P.N = ov; P.n_tile = NTv;
      P.tiles_m = (ov + SG_BM - 1) / SG_BM; P.tiles_n = (ov + NTv - 1) / NTv;
      P.ksplit = 1; P.k0_blocks = (X + BKv - 1) / BKv; P.k1_count = 1; P.k1_chunk = 1;
      P.a_mode = P.b_mode = TM_3D; P.div5 = 1;
      P.ea_rows = P.eb_rows = 1; P.ea_off = P.eb_off = s.erow;
      P.c_off = s.thi; P.c2_off = s.tlo; P.ldc = ldt; P.alpha = 1.0; P.vpad = vpadt;
      P.d_off = s.drow; P.vd_off = s.vdrow; P.et_off = s.scal + 4; P.v = v;
      P.group_m = kVGroupRows;
      P.ntiles = (long long)P.tiles_m * P.tiles_n;
      const uint64_t dims[3] = {(uint64_t)std::max(X, 1), (uint64_t)ov, (uint64_t)sv};
      const uint64_t str[2] = {(uint64_t)xpad * E2, (uint64_t)ov * xpad * E2};
      const uint32_t boxA[3] = {(uint32_t)BKv, SG_BM, (uint32_t)sv}, boxB[3] = {(uint32_t)BKv, (uint32_t)NTv, (uint32_t)sv};
      if (encode_tmap(&P.tmA, wsb + s.bs1, 3, dims, str, boxA, (int)E2) != RIMP2_OK ||
          encode_tmap(&P.tmB, wsb + s.bs1, 3, dims, str, boxB, (int)E2) != RIMP2_OK)
        return RIMP2_ERR_UNSUPPORTED;
      w.probs_v.push_back(P);
    }
    const uint64_t plane_b = (uint64_t)ov * ldd * E2;
    if (g) {  // Gamma[(i,a)][Q] = sum_(j,b) Tt[(i,a)][(j,b)] B[(j,b)][Q]
      SplitProb P{};
      P.kind = PK_GAMMA; P.frag = idx;
      P.M = ov; P.N = X; P.n_tile = NTg;
      P.tiles_m = (ov + SG_BM - 1) / SG_BM; P.tiles_n = (X + NTg - 1) / NTg;
      P.ksplit = 1; P.k0_blocks = (RL + BKg - 1) / BKg; P.k1_count = 1; P.k1_chunk = 1;
      P.a_mode = P.b_mode = TM_3D; P.div5 = 1;
      // K = (j,b) cut into slabs of about kGammaSlabK elements (split-K for large
      // fragments), slab index outermost: the tiles in flight share one slab, and the
      // tiles of a row start close together, which keeps their Tt rows in L2; the slabs
      // meet in Gamma by FP64 atomics.  Fewer, longer slabs mean fewer atomics and tile
      // switches, which measured faster down to two or three slabs.
      const int kb = P.k0_blocks;
      int slabs = sp.variant == 3 ? 1 : (int)(((long long)kb * BKg + kGammaSlabK / 2) / kGammaSlabK);
      if (slabs > 1) {
        const int per = (kb + slabs - 1) / slabs;
        slabs = (kb + per - 1) / per;
        P.k0_blocks = per; P.k1_count = slabs; P.ksplit = slabs;
        P.a_mode = P.b_mode = TM_3DK; P.div5 = per * BKg; P.ks_outer = 1;
        fdev.back().zero_gamma = 1;
      }
      // the leading s_g planes of Tt (one scale per fragment) and B with one scale per aux
      // index Q
      P.ea_rows = 0; P.ea_off = s.scal + 4; P.ea_add = kTtAdd;
      P.eb_rows = 1; P.eb_off = s.ecol; P.eb_add = 0;
      P.c_off = f.gamma_off; P.ldc = X; P.alpha = 1.0;
      P.ntiles = (long long)P.tiles_m * P.tiles_n * P.ksplit;
      const uint64_t dA[3] = {(uint64_t)RL, (uint64_t)ov, (uint64_t)s.st_out};
      const uint64_t sA[2] = {(uint64_t)ldd * E2, plane_b};
      const uint64_t dB[3] = {(uint64_t)RL, (uint64_t)X, (uint64_t)sgl};
      const uint64_t sB[2] = {(uint64_t)ldd * E2, (uint64_t)X * ldd * E2};
      const uint32_t boxA[3] = {(uint32_t)BKg, SG_BM, (uint32_t)sgl}, boxB[3] = {(uint32_t)BKg, (uint32_t)NTg, (uint32_t)sgl};
      if (encode_tmap(&P.tmA, wsb + s.tts, 3, dA, sA, boxA, (int)E2) != RIMP2_OK ||
          encode_tmap(&P.tmB, wsb + s.bs2, 3, dB, sB, boxB, (int)E2) != RIMP2_OK)
        return RIMP2_ERR_UNSUPPORTED;
      // with the slice count of P, Gamma joins P's launch
      (sgl == st ? w.probs_c : w.probs_g).push_back(P);
    }
    if (f.pab_off >= 0) {  // P_ab = sum_i sum_(j,c) Tt[(i,a)][(j,c)] T[(i,b)][(j,c)]
      SplitProb P{};
      P.kind = PK_PAB; P.frag = idx;
      P.M = P.N = v; P.n_tile = NTt;
      P.tiles_m = (v + SG_BM - 1) / SG_BM; P.tiles_n = (v + NTt - 1) / NTt;
      P.k0_blocks = (RL + BKt - 1) / BKt; P.k1_count = o;
      P.a_mode = P.b_mode = TM_4D; P.div5 = 1;
      P.ea_rows = P.eb_rows = 0; P.ea_off = P.eb_off = s.scal + 4;
      P.ea_add = kTtAdd; P.eb_add = kTAdd;
      P.c_off = f.pab_off; P.ldc = v; P.alpha = 1.0; P.sym = 1;
      choose_split_k(P, sp.grid, split_mul);
      // split index outermost: the tiles in flight share one range of i and so read the
      // same Tt_i / T_i rows; with it innermost, neighbours worked on different i and the
      // launch re-read its operands from DRAM (226 GB at nocc=100 nvir=500, 0.92 of HBM)
      P.ks_outer = 1;
      P.ntiles = (long long)P.tiles_m * P.tiles_n * P.ksplit;
      const uint64_t d4[4] = {(uint64_t)RL, (uint64_t)v, (uint64_t)o, (uint64_t)st};
      const uint64_t s4[3] = {(uint64_t)ldd * E2, (uint64_t)v * ldd * E2, plane_b};
      const uint32_t boxA[4] = {(uint32_t)BKt, SG_BM, 1, (uint32_t)st}, boxB[4] = {(uint32_t)BKt, (uint32_t)NTt, 1, (uint32_t)st};
      if (encode_tmap(&P.tmA, wsb + s.tts, 4, d4, s4, boxA, (int)E2) != RIMP2_OK ||
          encode_tmap(&P.tmB, wsb + s.ts, 4, d4, s4, boxB, (int)E2) != RIMP2_OK)
        return RIMP2_ERR_UNSUPPORTED;
      w.probs_c.push_back(P);
    }
    if (f.pij_off >= 0 && pij_direct) {  // P_ij = -sum_(k,a) sum_b Tt[(i,a)][(k,b)] T[(j,a)][(k,b)]
      SplitProb P{};
      P.kind = PK_PIJ; P.frag = idx;
      P.M = P.N = o; P.n_tile = NTt;
      P.tiles_m = (o + SG_BM - 1) / SG_BM; P.tiles_n = (o + NTt - 1) / NTt;
      P.k0_blocks = (vpad + BKt - 1) / BKt; P.k1_count = o * v;
      P.a_mode = P.b_mode = TM_5D; P.div5 = v;
      P.ea_rows = P.eb_rows = 0; P.ea_off = P.eb_off = s.scal + 4;
      P.ea_add = kTtAdd; P.eb_add = kTAdd;
      P.c_off = f.pij_off; P.ldc = o; P.alpha = -1.0; P.sym = 1;
      choose_split_k(P, sp.grid, split_mul);
      P.ks_outer = 1;   // as for P_ab: the tiles in flight share one (k,b) range
      P.ntiles = (long long)P.tiles_m * P.tiles_n * P.ksplit;
      const uint64_t d5[5] = {(uint64_t)vpad, (uint64_t)o, (uint64_t)v, (uint64_t)o, (uint64_t)st};
      const uint64_t s5[4] = {(uint64_t)vpad * E2, (uint64_t)ldd * E2, (uint64_t)v * ldd * E2, plane_b};
      const uint32_t boxA[5] = {(uint32_t)BKt, 1, 1, SG_BM, (uint32_t)st}, boxB[5] = {(uint32_t)BKt, 1, 1, (uint32_t)NTt, (uint32_t)st};
      if (encode_tmap(&P.tmA, wsb + s.tts, 5, d5, s5, boxA, (int)E2) != RIMP2_OK ||
          encode_tmap(&P.tmB, wsb + s.ts, 5, d5, s5, boxB, (int)E2) != RIMP2_OK)
        return RIMP2_ERR_UNSUPPORTED;
      w.probs_c.push_back(P);
    } else if (f.pij_off >= 0) {
      // P_ij through the pair symmetry Tt_ik(a,b) = Tt_ki(b,a):
      // P_ij = -sum_(k,b) sum_a Tt[(k,b)][(i,a)] T[(k,b)][(j,a)]; the rows i of one
      // (k,b) row are vpad elements apart, so a 128-row TMA box reads one contiguous span
      SplitProb P{};
      P.kind = PK_PIJ; P.frag = idx;
      P.M = P.N = o; P.n_tile = NTt;
      P.tiles_m = (o + SG_BM - 1) / SG_BM; P.tiles_n = (o + NTt - 1) / NTt;
      P.k0_blocks = (vpad + BKt - 1) / BKt; P.k1_count = o * v;
      P.a_mode = P.b_mode = TM_4D; P.div5 = 1;
      P.ea_rows = P.eb_rows = 0; P.ea_off = P.eb_off = s.scal + 4;
      P.ea_add = kTtAdd; P.eb_add = kTAdd;
      P.c_off = f.pij_off; P.ldc = o; P.alpha = -1.0; P.sym = 1;
      choose_split_k(P, sp.grid, split_mul);
      P.ks_outer = 1;   // as for P_ab: the tiles in flight share one (k,b) range
      P.ntiles = (long long)P.tiles_m * P.tiles_n * P.ksplit;
      const uint64_t d4[4] = {(uint64_t)vpad, (uint64_t)o, (uint64_t)ov, (uint64_t)st};
      const uint64_t s4[3] = {(uint64_t)vpad * E2, (uint64_t)ldd * E2, plane_b};
      const uint32_t boxA[4] = {(uint32_t)BKt, SG_BM, 1, (uint32_t)st}, boxB[4] = {(uint32_t)BKt, (uint32_t)NTt, 1, (uint32_t)st};
      if (encode_tmap(&P.tmA, wsb + s.tts, 4, d4, s4, boxA, (int)E2) != RIMP2_OK ||
          encode_tmap(&P.tmB, wsb + s.ts, 4, d4, s4, boxB, (int)E2) != RIMP2_OK)
        return RIMP2_ERR_UNSUPPORTED;
      w.probs_c.push_back(P);
    }
  }
  // A split-K piece of P_ab / P_ij spans at least kMinPieceK elements of K: the per-problem
  // target (a multiple of the grid, for locality at large sizes) would otherwise cut the
  // P_ij of small fragments, K0 = nvir per outer index, into pieces whose drain, epilogue
  // and atomics cost as much as their MMAs
  for (auto& P : w.probs_c)
    if (P.kind == PK_PAB || P.kind == PK_PIJ) {
      const long long per = (long long)P.k0_blocks * BKt;   // K elements per outer index
      const int chunk = (int)std::min<long long>(P.k1_count, (kMinPieceK + per - 1) / per);
      if (P.k1_chunk < chunk) {
        P.k1_chunk = chunk;
        P.ksplit = std::max(1, (P.k1_count + chunk - 1) / chunk);
        P.ntiles = (long long)P.tiles_m * P.tiles_n * P.ksplit;
      }
    }
  // Sixteen epilogue warps when every fragment's aux dimension is short: V's tiles then
  // have little K for their MMAs to hide the T = V/D epilogue behind, which more warps
  // share (MBE3 stated batch: dimer level 86.1 -> 79.3 ms); with naux ~1500 the extra
  // warps cost V's MMA issuer a little (41.6 -> 42.2 ms at nocc=100 nvir=500).
  {
    int max_x = 0;
    for (const auto& s : w.sfd) max_x = std::max(max_x, s.X);
    w.epi_warps = max_x <= 1024 ? 16 : 8;
  }
  total_pairs = pairs;
  w.rows = rows;
  w.b2_tiles = b2t;
  w.qblks = qbl;
  finish(w.probs_v, w.tiles_v);
  finish(w.probs_c, w.tiles_c);
  finish(w.probs_g, w.tiles_g);
  // every problem's tiles and TMA boxes must match the kernel instance of its launch
  auto same_shape = [](const std::vector<SplitProb>& v, const SplitLaunch& c) {
    for (const auto& P : v)
      if (P.n_tile != c.n_tile_max) return false;
    return true;
  };
  if (!same_shape(w.probs_v, sp.cfg_v) || !same_shape(w.probs_c, sp.cfg_t) ||
      !same_shape(w.probs_g, sp.cfg_g))
    return RIMP2_ERR_UNSUPPORTED;
  w.mma_v = w.mma_c = w.mma_g = 0.0;
  for (const auto& P : w.probs_v) w.mma_v += prob_mma_flops(P, sv, BKv);
  for (const auto& P : w.probs_c) w.mma_c += prob_mma_flops(P, st, BKt);
  for (const auto& P : w.probs_g) w.mma_g += prob_mma_flops(P, sgl, BKg);
  return RIMP2_OK;
}

size_t split_layout_wave(SplitWave& w, size_t off) {
  off = al256(off);
  w.off_sfd = off; off = al256(off + w.sfd.size() * sizeof(SplitFragDev));
  w.off_pv = off; off = al256(off + w.probs_v.size() * sizeof(SplitProb));
  w.off_pc = off; off = al256(off + w.probs_c.size() * sizeof(SplitProb));
  w.off_pg = off; off = al256(off + w.probs_g.size() * sizeof(SplitProb));
  w.off_bv = off; off = al256(off + w.probs_v.size() * sizeof(long long));
  w.off_bc = off; off = al256(off + w.probs_c.size() * sizeof(long long));
  w.off_bg = off; off = al256(off + w.probs_g.size() * sizeof(long long));
  return off;
}

void split_fill_wave(const SplitWave& w, char* host) {
  if (!w.sfd.empty()) memcpy(host + w.off_sfd, w.sfd.data(), w.sfd.size() * sizeof(SplitFragDev));
  if (!w.probs_v.empty()) memcpy(host + w.off_pv, w.probs_v.data(), w.probs_v.size() * sizeof(SplitProb));
  if (!w.probs_c.empty()) memcpy(host + w.off_pc, w.probs_c.data(), w.probs_c.size() * sizeof(SplitProb));
  if (!w.probs_g.empty()) memcpy(host + w.off_pg, w.probs_g.data(), w.probs_g.size() * sizeof(SplitProb));
  auto begins = [&](const std::vector<SplitProb>& v, size_t off) {
    for (size_t k = 0; k < v.size(); ++k) {
      const long long b = v[k].tile_begin;
      memcpy(host + off + k * sizeof(long long), &b, sizeof(b));
    }
  };
  begins(w.probs_v, w.off_bv);
  begins(w.probs_c, w.off_bc);
  begins(w.probs_g, w.off_bg);
}

int split_enqueue_wave(SplitPlan& sp, SplitWave& w, char* dblk, const FragDev* dfd, int nf,
                       long long total_pairs, Bases bs, unsigned* ctr, cudaStream_t s,
                       int* launches, long long* tiles, cudaEvent_t* ev) {
  const SplitFragDev* sfd = (const SplitFragDev*)(dblk + w.off_sfd);
  int nl = 0;
  cudaError_t e = cudaSuccess;
  if (nf > 0) {
    k_split_reset<<<(unsigned)nf, 128, 0, s>>>(sfd, nf, bs);
    ++nl;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && w.rows > 0) {
    if (sp.fp8) k_slice_b1<true><<<(unsigned)((w.rows + 7) / 8), 256, 0, s>>>(sfd, nf, w.rows, sp.slices_v, bs);
    else k_slice_b1<false><<<(unsigned)((w.rows + 7) / 8), 256, 0, s>>>(sfd, nf, w.rows, sp.slices_v, bs);
    ++nl;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && w.qblks > 0) {
    k_bcol_max<<<(unsigned)w.qblks, 256, 0, s>>>(sfd, nf, bs);
    ++nl;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && w.b2_tiles > 0) {
    if (sp.fp8) k_slice_b2<true><<<(unsigned)w.b2_tiles, 256, 0, s>>>(sfd, nf, sp.slices_g, bs);
    else k_slice_b2<false><<<(unsigned)w.b2_tiles, 256, 0, s>>>(sfd, nf, sp.slices_g, bs);
    ++nl;
    e = cudaGetLastError();
  }
  if (ev) cudaEventRecordWithFlags(ev[1], s, cudaEventRecordExternal);
  if (e == cudaSuccess && w.tiles_v > 0) {
    SplitLaunch cfg = sp.cfg_v;
    cfg.epi_warps = w.epi_warps;
    e = launch_split_gemm((const SplitProb*)(dblk + w.off_pv), (const long long*)(dblk + w.off_bv),
                          (int)w.probs_v.size(), w.tiles_v, bs,
                          ctr + 0, cfg, sp.grid, s);
    ++nl;
  }
  if (ev) cudaEventRecordWithFlags(ev[2], s, cudaEventRecordExternal);
  if (e == cudaSuccess && total_pairs > 0) {
    if (sp.fp8) k_amp_split<true><<<(unsigned)total_pairs, 256, 0, s>>>(sfd, nf, sp.slices_t, bs);
    else k_amp_split<false><<<(unsigned)total_pairs, 256, 0, s>>>(sfd, nf, sp.slices_t, bs);
    ++nl;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) { e = launch_energy_reduce(dfd, nf, bs, s); ++nl; }
  if (e == cudaSuccess) { e = launch_zero_p(dfd, nf, bs, s); ++nl; }
  if (ev) cudaEventRecordWithFlags(ev[3], s, cudaEventRecordExternal);
  if (e == cudaSuccess && w.tiles_c > 0) {
    SplitLaunch cfg = sp.cfg_t;
    cfg.epi_warps = w.epi_warps;
    e = launch_split_gemm((const SplitProb*)(dblk + w.off_pc), (const long long*)(dblk + w.off_bc),
                          (int)w.probs_c.size(), w.tiles_c, bs,
                          ctr + 1, cfg, sp.grid, s);
    ++nl;
  }
  if (ev) cudaEventRecordWithFlags(ev[4], s, cudaEventRecordExternal);
  if (e == cudaSuccess && w.tiles_g > 0) {
    SplitLaunch cfg = sp.cfg_g;
    cfg.epi_warps = w.epi_warps;
    e = launch_split_gemm((const SplitProb*)(dblk + w.off_pg), (const long long*)(dblk + w.off_bg),
                          (int)w.probs_g.size(), w.tiles_g, bs,
                          ctr + 2, cfg, sp.grid, s);
    ++nl;
  }
  if (ev) cudaEventRecordWithFlags(ev[5], s, cudaEventRecordExternal);
  *launches = nl;
  *tiles = w.tiles_v + w.tiles_c + w.tiles_g;
  return e == cudaSuccess ? RIMP2_OK : RIMP2_ERR_CUDA;
}

}  // namespace rimp2
