// Split-precision tensor-core GEMM (tcgen05, sm_103a): shared declarations.
//
// Operands are "slices": balanced base-512 integer digits of FP64 values relative to a
// power-of-two scale, stored as BF16 (its 8-bit significand holds every integer up to
// 256 exactly):
//   x ~= sum_p d_p 2^(E - 9(p+1)),   |x| <= 2^(E-3),
// so that the leading digit d_0 lies in [-64, 64] and the others in [-256, 256]; or (FP8
// mode) balanced base-32 digits in [-16, 16] stored as e4m3 (exact), |x| <= 2^(E-1),
// with 5 in place of 9 in every formula below.
// C(m,n) = sum_k A(m,k) B(n,k) is then 2^(EA(m) + EB(n) - 2 LB) sum_l 2^(-LB l) S_l with
// S_l = sum_{p+q=l} sum_k dA_p dB_q, the truncated level sum kept for l < s.  Each S_l
// accumulates in its own FP32 TMEM accumulator over K chunks, where the levels folded
// exactly are exact integers by construction.  BF16, chunks of 512: |S_0| <= 512 * 2^12
// = 2^21 and |S_1| <= 512 * 2 * 2^6 * 2^8 = 2^24 (the narrow leading digit is what allows
// 512).  FP8, chunks of 8192: levels 0..4 stay below 5 * 8192 * 2^8 < 2^24.  A higher
// level rounds only if its partial sum exceeds 2^24 in magnitude, which bounds that error
// by 2^-24 of the level.  Each chunk is then folded into a per-element double-float
// (hi, lo) accumulator in registers.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rimp2_internal.cuh"

namespace rimp2 {

constexpr int SG_BM = 128;          // rows per tile (TMEM lanes)
constexpr int SG_BN_MAX = 96;       // max columns per tile
// bits per digit, K elements per accumulation chunk, and the bits by which the leading
// digit is narrower than the others (the scale of x is 2^E with |x| <= 2^(E-1-HEAD)), of
// each digit format
constexpr int SG_LB_BF16 = 9, SG_CHUNK_K_BF16 = 512, SG_HEAD_BF16 = 2;
constexpr int SG_LB_FP8 = 5, SG_CHUNK_K_FP8 = 8192, SG_HEAD_FP8 = 0;
// K per pipeline stage: 32 (64-byte rows, 64B swizzle) or 16 (32-byte rows, 32B swizzle);
// the smaller stage fits twice as many stages in shared memory
constexpr int SG_MAX_SLICES = 16;   // FP8; BF16 stops at 8
// warp 0 TMA, warp 1 MMA, then the epilogue warps: 8 or 16 per launch (SplitLaunch::
// epi_warps), each of the four TMEM lane quadrants served by 2 or 4 warps that split the
// tile's columns between them

// TMA coordinate modes of one operand
enum : int {
  TM_3D = 0,    // {k0*32, row, slice}
  TM_4D = 1,    // {k0*32, row, k1, slice}
  TM_5D = 2,    // {k0*32, k1 / div, k1 % div, row, slice}
  TM_3DK = 3,   // {k1*div + k0*32, row, slice}: a flat K cut into slabs of div elements
};

// Extra problem kind used only by the testing hook: store sum_l 2^-8l S_l * 2^(EA+EB-16)
constexpr int PK_RAW = 7;

struct SplitProb {  // 64-byte aligned through its CUtensorMap members
  CUtensorMap tmA;        // A slices, box {32, 128, ..., slices}: one copy loads all slices
  CUtensorMap tmB;        // B slices, box {32, n_tile, ..., slices}
  int kind, frag;
  int M, N, n_tile;
  int tiles_m, tiles_n, ksplit;
  int k0_blocks;          // 32-wide blocks of the inner (contiguous) K dimension
  int k1_count, k1_chunk; // outer K index range and its per-split chunk
  int a_mode, b_mode, div5;
  int ea_rows, eb_rows;   // 1: per-row int32 exponent array; 0: one int32 scalar
  int ea_add, eb_add;     // added to the stored exponent
  int ks_outer;           // 1: the split (slab) index is the slowest index of the tile order
  long long tile_begin, ntiles;
  long long ea_off, eb_off;   // byte offsets into the workspace (int32 data)
  long long c_off, c2_off;    // outputs: PK_V: byte offsets of T_hi / T_lo planes in ws;
                              // others: element offsets into gamma / pab / pij
  long long ldc;
  double alpha;
  long long d_off;            // PK_V: byte offset of float2 d_m = e_i - e_a per row
  long long et_off;           // PK_V: byte offset of the unsigned max-exponent slot of |T|
  long long vd_off;           // PK_V: byte offset of float2 V_mm (diagonal, FP64 row sums)
  int v;                      // PK_V: nvir of the fragment
  int group_m;                // > 1: tiles walked in groups of group_m rows, column by column
  int vpad;                   // PK_V: T plane column of (j,b) is j*vpad + b
  int sym;                    // 1: C is symmetric (P_ab, P_ij): tiles below the diagonal are
                              // skipped and every (m < n) result is added at (m,n) and (n,m)
};

struct SplitLaunch {
  int slices;     // s (levels); same for every problem of one launch
  int bk;         // K elements per pipeline stage (BF16: 16 or 32; FP8: 64)
  bool fp8;       // digits as FP8 e4m3 (5 bits, kind::f8f6f4) instead of BF16 (9 bits)
  int n_tile_max; // widest n_tile of the launch (smem layout)
  int stages;     // pipeline depth
  size_t smem;    // dynamic shared memory bytes
  int epi_warps;  // epilogue warps: 8, or 16 (more warps for a tile's drain and epilogue)
};

// n_tile: columns per level accumulator (0: widest that fits 512 TMEM columns; else 64,
// 80 or 96, capped by the TMEM budget)
SplitLaunch split_launch_config(int slices, int bk = 32, int n_tile = 0, bool fp8 = false);
// d_begins (device, may be null): the problems' tile_begin values as a compact array
cudaError_t launch_split_gemm(const SplitProb* d_probs, const long long* d_begins, int nprobs,
                              long long total_tiles, Bases bs, unsigned* counter,
                              const SplitLaunch& cfg, int grid, cudaStream_t s);
int split_gemm_grid();
// Consumer-side wait limit of the contraction kernel on the current device (ns < 0: the
// normal 2 s); synchronous.  Used by a test hook only.
cudaError_t split_gemm_set_consumer_wait(long long ns);
cudaError_t split_gemm_prepare();

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link)
// box[0] x elem_bytes must be 32 (32B swizzle) or 64 (64B swizzle); elem_bytes 2 = BF16,
// 1 = raw bytes (FP8 digits)
int encode_tmap(CUtensorMap* tm, const void* base, int rank, const uint64_t* dims,
                const uint64_t* strides_bytes, const uint32_t* box, int elem_bytes);

}  // namespace rimp2
