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
