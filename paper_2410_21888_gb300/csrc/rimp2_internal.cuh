// Internal declarations shared by the librimp2 translation units (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rimp2.h"

namespace rimp2 {

// Device status word bits (plan-owned, read by rimp2_get_status).
enum : unsigned {
  ST_DENOM = 1u,      // some e_a <= e_i
  ST_NONFINITE = 2u,  // NaN/Inf in B or eps
  ST_TIMEOUT = 4u,    // a bounded mbarrier wait expired
  ST_INTERNAL = 8u,   // a device-side index check failed (access skipped)
};

// FP64 inputs read on the integer pipes: this GPU's FP64 unit runs at a small fraction of
// its FP32 and integer rates, and its conversions and comparisons would bound the
// element-wise kernels that read B.
#ifdef __CUDACC__
// |x| as an integer key: non-negative doubles order like their bit patterns
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
// x is neither Inf nor NaN
__device__ __forceinline__ bool finite_bits(double x) {
  return (((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FFu) != 0x7FFu;
}
// ilogb of a positive double given by its bits (exponent field; FP64 subnormals, far below
// any input this library sees, take the FP64 route)
__device__ __forceinline__ int ilogb_bits(unsigned long long b) {
  const int e = (int)((b >> 52) & 0x7FFu);
  return e != 0 ? e - 1023 : ilogb(__longlong_as_double((long long)b));
}
// h = (float)x and l = (float)(x - (double)h), both correctly rounded, from the bits of x:
// the 53-bit significand rounded to 24 bits (to nearest, ties to even) gives h, and the
// exact remainder, an integer below 2^29 in units of x's last bit, converted with
// rounding and scaled by a power of two gives l.  Bit-identical to the two conversions
// wherever h and any non-zero l are normal floats (|x| in [2^-74, 2^127)); other inputs,
// far from anything this library sees, take the FP64 conversions.
__device__ __forceinline__ void split_to_df(double x, float& h, float& l) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((u >> 52) & 0x7FFu);
  if (e < 949 || e > 1149) {
    h = (float)x;
    l = (float)(x - (double)h);
    return;
  }
  const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
  const unsigned long long m = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const unsigned long long r = m & ((1ull << 29) - 1);
  unsigned long long mh = m >> 29;
  if (r > (1ull << 28) || (r == (1ull << 28) && (mh & 1ull))) ++mh;
  // fraction field mh - 2^23 added to the exponent field: a carry (mh = 2^24) raises it
  h = __uint_as_float(sign + ((unsigned)(e - 1023 + 127) << 23) + (unsigned)(mh - (1ull << 23)));
  const int d = (int)((long long)m - (long long)(mh << 29));   // |d| <= 2^28
  // 2^(e - 1075) as two normal factors; x - h = 0 rounds to +0 whatever the sign of x
  const int k = e - 1075, k1 = k / 2, k2 = k - k1;
  const float s1 = __int_as_float((k1 + 127) << 23), s2 = __int_as_float((k2 + 127) << 23);
  const float lv = (__int2float_rn(d) * s1) * s2;
  l = d == 0 ? 0.0f : (sign ? -lv : lv);
}
#endif

// Kinds of contraction problems handled by the grouped GEMM kernels.
enum ProbKind : int {
  PK_V = 0,      // V_ij(a,b) = sum_Q B B over (i,a)x(j,b), upper triangle of tiles,
                 // epilogue T = V / D, written to both triangles of the workspace T
  PK_GAMMA = 1,  // Gamma[(i,a)][Q] = sum_(j,b) Tt[(i,a)][(j,b)] B[(j,b)][Q]
  PK_PAB = 2,    // P_ab += sum_i sum_(j,c) Tt[i][a][(j,c)] T[i][b][(j,c)]
  PK_PIJ = 3,    // P_ij += -sum_(k,b) sum_a Tt[k][b][i][a] T[k][b][j][a]
  PK_GEN = 4,    // C = alpha A Bop^T on caller pointers pa / pb / pc (gradient step)
};

// Base pointers of one call.  Problem descriptors hold element offsets only, so a
// plan's descriptors stay valid when a caller reuses the same pools.
struct Bases {
  const double* B;
  const double* eps;
  double* ws;
  double* gamma;
  double* pij;
  double* pab;
  double* epair;
  double* energy;
  double* energy_os;   // may be null
  double* energy_scs;  // may be null: scs_os * E_OS + scs_ss * (E - E_OS)
  double scs_os, scs_ss;
  unsigned* status;
};

// One GEMM-shaped problem C(m,n) = alpha * sum_{k1,k0} A(m,k0,k1) Bop(n,k0,k1).
// A(m,k0,k1) = A[a_off + m*sAm + k0*sAk + k1*sA1]; Bop likewise with n.
struct GemmProb {
  int kind, frag;
  int M, N, K0, K1;
  int tiles_m, tiles_n, ksplit, k1_chunk;
  long long tile_begin, ntiles;  // position in the flattened work queue
  long long a_off, b_off, c_off; // a from B (PK_V) or ws; b from B (PK_V, PK_GAMMA) or ws
  long long sAm, sAk, sA1, sBn, sBk, sB1, ldc;
  double alpha;
  long long eo_off, ev_off;  // orbital energies (PK_V epilogue)
  int v, b_from_B;           // b_from_B: Bop reads the B pool (else workspace)
  const double* pa;          // PK_GEN: A, Bop and C base pointers (offsets unused)
  const double* pb;
  double* pc;
  int accumulate, pad;       // PK_GEN: 1 adds into C (atomics); 0 stores (needs ksplit 1)
};

// Per-fragment info used by the elementwise / reduction kernels.
struct FragDev {
  int o, v, X, idx;           // idx: position in the batch (energy[idx])
  int zero_gamma, pad0;       // 1: Gamma is accumulated by atomics, zero it first
  long long b_off, eo_off, ev_off;
  long long t_off, tt_off, ep_off;   // workspace offsets (elements)
  long long epos_off;         // opposite-spin pair energies [o][o] (elements), or -1
  long long gamma_off, pij_off, pab_off, epair_off;  // -1: not requested
  long long pair_begin;       // prefix of o(o+1)/2 pair blocks in the wave
};

// ---- launchers (fp64_kernels.cu) ----
cudaError_t launch_check_inputs(const FragDev* d_frags, int nfrag, long long max_bx,
                                Bases bs, cudaStream_t s);
// skip (device, may be null): when *skip != 0 at launch time every CTA returns at once
cudaError_t launch_gemm_f64(const GemmProb* d_probs, int nprobs, long long total_tiles,
                            Bases bs, unsigned* counter, int grid, cudaStream_t s,
                            const int* skip = nullptr);
int gemm_f64_occupancy_grid();
cudaError_t launch_amplitude_f64(const FragDev* d_frags, int nfrag, long long total_pairs,
                                 Bases bs, cudaStream_t s);
cudaError_t launch_energy_reduce(const FragDev* d_frags, int nfrag, Bases bs, cudaStream_t s);
cudaError_t launch_zero_p(const FragDev* d_frags, int nfrag, Bases bs, cudaStream_t s);

// tile sizes of the FP64 grouped GEMM
constexpr int F64_BM = 64;
constexpr int F64_BN = 64;
constexpr int F64_BK = 16;

}  // namespace rimp2
