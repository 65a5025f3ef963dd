// Split-precision (integer-slice tensor-core) path: plan/wave interface used by the
// host API.  Implemented in split_path.cu.
#pragma once

#include <vector>

#include "rimp2_internal.cuh"
#include "split_gemm.cuh"

namespace rimp2 {

// Per-fragment workspace layout of the split path (byte offsets into the workspace).
struct SplitFragDev {
  int o, v, X, idx;
  int vpad, xpad;
  int st_out, st_t;         // digit slices to write: Tt (P and Gamma), T (P); 0: none
  int vpadt;                // j-block width of the T planes (nvir rounded up to 32: 128 B)
  long long ldd;    // row stride (elements) of the Tt / T / Gamma-B digit planes (>= o*vpad)
  long long ldt;    // row stride (elements) of the double-float T planes (>= o*vpad)
  long long b_off, eo_off, ev_off;  // elements into the B / eps pools
  long long bs1;    // B digits for V: [s_v][o*v][xpad] bf16, per-row scale
  long long bs2;    // B digits for Gamma: [s_g][X][ldd], one scale 2^E_Q per aux index Q
  long long erow;   // int32 [o*v] row exponents of bs1
  long long drow;   // float2 [o*v]: e_i - e_a as a double-float
  long long vdrow;  // float2 [o*v]: V_ii(a,a) = sum_Q (B^Q_ia)^2 (FP64 sum) as a double-float
  long long thi, tlo;  // float [o*v][ldt]: T as a double-float pair of planes, column j*vpadt + b
  long long tts, ts;   // Tt [st_out] and T [st_t] digit planes [s][o*v][ldd], one scale each
                       // (Gamma reads the leading s_g planes of Tt)
  long long ecolm;  // FP64 bits [X]: max_(j,b) |B^Q_jb| for every aux index Q
  long long ecol;   // int32 [X]: exponent of each aux index of B for Gamma
  long long ep;     // double [o][o] pair energies, then [o][o] opposite-spin pair energies
  long long scal;   // uint32 [1]: max |T| exponent ([0] unused)
  long long pair_begin;   // first amplitude CTA of the fragment (o * o ordered pairs each)
  long long row_begin, b2_tile_begin;
  long long qblk_begin;   // first block (32 Q x 256 rows) of the fragment in the column maxima pass
  int sg_out, pad2;       // slices of Gamma's operands (0: no Gamma)
};

struct SplitPlan {
  int precision = 0;
  int slices_v = 0, slices_t = 0, slices_g = 0;
  SplitLaunch cfg_v{}, cfg_t{}, cfg_g{};   // V; P_ab / P_ij; Gamma
  int grid = 0;
  bool ready = false;
  bool fp8 = false;  // RIMP2_FP8_SPLIT: e4m3 digits
  int variant = 0;   // contraction-stage variant (autotuner), see split_variant_desc
  // tile shapes (n_tile, K per stage) the autotuner trials per launch, the configured
  // default first, and the index of each launch's shape in use
  std::vector<SplitLaunch> cand_v, cand_t, cand_g;
  int shape_v = 0, shape_t = 0, shape_g = 0;
};

// Selects the tile shapes of the V, P_ab / P_ij and Gamma launches (indices into the
// candidate lists, clamped to their ends).
void split_set_shapes(SplitPlan& sp, int iv, int it, int ig);

// Variants of the Gamma/P contraction stage the autotuner times:
//   0: P_ij rows read through the local (k,b)-major view, split-K target 8 x grid
//   1: P_ij rows read through the direct (i,a)-major view, split-K target 8 x grid
//   2: local view, split-K target 16 x grid
//   3: as 0, with Gamma's K in one piece (no slabs, no atomics on Gamma)
// Variants 0..2 cut Gamma's K into slabs accumulated with FP64 atomics.
constexpr int kSplitVariants = 4;

struct SplitWave {
  std::vector<SplitFragDev> sfd;
  std::vector<SplitProb> probs_v, probs_c, probs_g;   // V; P_ab / P_ij; Gamma
  long long tiles_v = 0, tiles_c = 0, tiles_g = 0, rows = 0, b2_tiles = 0, qblks = 0;
  bool want_gamma = false;
  int epi_warps = 8;   // epilogue warps of the wave's contraction launches (see build)
  double mma_v = 0, mma_c = 0, mma_g = 0;   // tensor-core FLOPs issued per launch
  size_t off_sfd = 0, off_pv = 0, off_pc = 0, off_pg = 0;  // byte offsets in the device block
  size_t off_bv = 0, off_bc = 0, off_bg = 0;  // the problems' tile_begin values (int64 each)
};

int split_plan_init(SplitPlan& sp, int precision, const rimp2_options& opt);
void split_plan_release(SplitPlan& sp);
size_t split_frag_ws_bytes(const SplitPlan& sp, const rimp2_frag& f);
int split_build_wave(SplitPlan& sp, const rimp2_frag* frags, const std::vector<int>& members,
                     const double* B, void* ws, std::vector<FragDev>& fdev, SplitWave& w,
                     long long& total_pairs, long long& max_b);
size_t split_layout_wave(SplitWave& w, size_t off);
void split_fill_wave(const SplitWave& w, char* host_block);
int split_enqueue_wave(SplitPlan& sp, SplitWave& w, char* dblk, const FragDev* dfd, int nf,
                       long long total_pairs, Bases bs, unsigned* ctr, cudaStream_t s,
                       int* launches, long long* tiles, cudaEvent_t* ev);

}  // namespace rimp2
