/*
 * rimp2.h - C ABI of the GB300 (sm_103a) RI-MP2 energy and gradient-intermediate
 * library (librimp2.so).
 *
 * What it computes, per fragment f of a batch (closed shell, no frozen core; Sec.
 * "Notation" of arXiv 2410.21888 and its Appendix):
 *
 *   V_ij(a,b)  = sum_Q B^Q_ia B^Q_jb            RI integrals (ia|jb), Eq. MP2_ints
 *   T_ij(a,b)  = V_ij(a,b) / (e_i + e_j - e_a - e_b)
 *                                               amplitudes X^ab_ij (Appendix; the printed
 *                                               denominator is garbled, this is the standard
 *                                               sign)
 *   Tt_ij(a,b) = 2 T_ij(a,b) - T_ij(b,a)        the 2X - X^T combination of Gamma
 *   e_pair[i][j] = sum_ab Tt_ij(a,b) V_ij(a,b), E = sum_ij e_pair[i][j]
 *                                               closed-shell MP2 energy
 *   Gamma^Q_ia = sum_jb Tt_ij(a,b) B^Q_jb       Appendix Gamma in the MO-B basis (the
 *                                               J^-1/2 back-transform is not applied)
 *   P_ij = -sum_kab Tt_ik(a,b) T_jk(a,b)        Appendix D^MP2_ij (unrelaxed)
 *   P_ab =  sum_ijc Tt_ij(a,c) T_ij(b,c)        Appendix D^MP2_ab (unrelaxed)
 *
 * Denominators, pair and cross-pair energy sums are FP64 in every precision mode.  In
 * RIMP2_FP64 every contraction is FP64.  In the split modes the four contractions (V,
 * Gamma, P_ab, P_ij) run on the tensor cores as sums of exact products of integer
 * digit slices (BF16: 9-bit digits; FP8 e4m3: 5-bit digits) accumulated in FP32 and
 * recombined at higher precision.
 *
 * Layouts (all row-major, element offsets into caller-owned device pools):
 *   B[nocc][nvir][naux] FP64, naux fastest;  Gamma: same shape and layout as B;
 *   eps: eps_occ[nocc] at eo_off, eps_vir[nvir] at ev_off (FP64);
 *   P_ij[nocc][nocc], P_ab[nvir][nvir], e_pair[nocc][nocc] (FP64);
 *   energy[nfrag] (FP64), one per fragment in batch order.
 *
 * Ownership: the caller owns every device buffer (inputs, outputs, workspace) and the
 * stream.  A plan owns host metadata, a small device block (task queue counters,
 * problem descriptors, status word) and the CUDA graph it captures.  Outputs are
 * overwritten, never accumulated.
 *
 * Errors: every entry point returns RIMP2_OK (0) or a negative RIMP2_ERR_* code and
 * never aborts, throws or traps.  Conditions that only the device can see (a
 * denominator >= 0, non-finite inputs, an expired bounded wait) are recorded in the
 * plan's status word; rimp2_get_status() reads it after synchronising the plan.
 *
 * Threading: a plan is used by one host thread and one stream at a time.
 */
#ifndef RIMP2_H
#define RIMP2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RIMP2_OK 0
#define RIMP2_ERR_BAD_ARG (-1)      /* null pointer, negative size, bad enum */
#define RIMP2_ERR_SHAPE (-2)        /* batch shapes differ from the plan's */
#define RIMP2_ERR_DENOM (-3)        /* some e_a <= e_i: a denominator is not negative */
#define RIMP2_ERR_NONFINITE (-4)    /* NaN or Inf in B or the orbital energies */
#define RIMP2_ERR_WORKSPACE (-5)    /* workspace pointer null/misaligned or too small */
#define RIMP2_ERR_CUDA (-6)         /* a CUDA runtime call failed */
#define RIMP2_ERR_TIMEOUT (-7)      /* a bounded device-side wait expired */
#define RIMP2_ERR_UNSUPPORTED (-8)  /* option or size outside what this build supports */
#define RIMP2_ERR_NOMEM (-9)        /* host or plan-internal device allocation failed */

typedef enum {
  RIMP2_FP64 = 0,        /* FP64 contractions (CUDA-core DFMA) */
  RIMP2_BF16_SPLIT = 1,  /* BF16 integer-slice products on tcgen05, FP32 accumulate */
  RIMP2_FP8_SPLIT = 2    /* FP8 (e4m3) integer-slice products on tcgen05, FP32 accumulate */
} rimp2_precision;

/* One fragment: sizes and element offsets into the batch pools.  An offset of -1
 * means "not requested" for gamma_off, pij_off, pab_off and epair_off. */
typedef struct rimp2_frag {
  int32_t nocc, nvir, naux, flags; /* flags: reserved, pass 0 */
  int64_t b_off;                   /* into batch.B */
  int64_t eo_off, ev_off;          /* into batch.eps */
  int64_t gamma_off;               /* into batch.gamma, or -1 */
  int64_t pij_off;                 /* into batch.pij, or -1 */
  int64_t pab_off;                 /* into batch.pab, or -1 */
  int64_t epair_off;               /* into batch.epair, or -1 */
} rimp2_frag;

/* Device pointers of one call.  frags is a host array of nfrag entries that must
 * describe the same shapes, in the same order, as the plan's. */
typedef struct rimp2_batch {
  int32_t nfrag, reserved;
  const rimp2_frag* frags;
  const double* B;
  const double* eps;
  double* gamma;
  double* pij;
  double* pab;
  double* epair;
  double* energy;    /* [nfrag], required: E = sum_ijab (2 T_ij(a,b) - T_ij(b,a)) V_ij(a,b) */
  double* energy_os; /* [nfrag] or NULL: the opposite-spin component E_OS = sum T V; the
                        same-spin one is E - E_OS (SCS-MP2, named in the paper's
                        Introduction, weights the two components) */
  double* energy_scs; /* [nfrag] or NULL: the spin-component-scaled energy
                         scs_os * E_OS + scs_ss * (E - E_OS), formed in FP64 from the two
                         compensated sums, with the weights of the plan's options */
} rimp2_batch;

typedef struct rimp2_options {
  int32_t slices_v;    /* split modes: digit slices of B for V; 0 = default (BF16: 5
                          slices of 9 bits, range 2..8; FP8: 8 slices of 5 bits, 2..16).
                          The diagonal V_ii(a,a) is taken from an FP64 row sum of
                          squares: there both operands have the same digits and the
                          truncated triangle's error would have one sign */
  int32_t slices_t;    /* split modes: slices of T and Tt for P_ab and P_ij (one scale
                          per fragment); 0 = default (BF16: 6, range 2..8; FP8: 10,
                          range 2..16) */
  int32_t use_graph;   /* 1 (default): capture the launch sequence once, replay it */
  int32_t check_inputs;/* 1 (default): device check of denominators and finiteness */
  int32_t autotune;    /* 1: the first calls of the plan each run one trial, timed in situ
                          with CUDA events between the stages; later calls use the fastest
                          (default 0).  Split modes: first one trial per tile shape (every
                          launch - V, P_ab / P_ij, Gamma - takes its own i-th candidate of
                          n_tile x stage_k that fits TMEM), then the other variants of the
                          Gamma/P contraction stage (operand view of P_ij, split-K factor,
                          Gamma slabs) with each launch's fastest shape; FP64: the split-K
                          factor.  Results are identical up to rounding order. */
  int32_t profile_stages; /* 1: record CUDA events between the stages of each call so that
                             rimp2_get_stats reports stage_ms (default 0) */
  size_t max_workspace_bytes; /* 0: one wave for the whole batch; else waves sized so
                                 the workspace stays below this many bytes */
  int32_t stage_k;     /* split modes: K elements per pipeline stage of the tensor-core
                          GEMM, 16 or 32 (0 = default 32) */
  int32_t n_tile;      /* BF16 split: columns per level accumulator of every launch, 48,
                          64, 80 or 96, at most the widest that fits TMEM for the slice
                          count.  0 = per launch: V 48 when two sets of slices x 48
                          accumulator columns fit the 512 TMEM columns (the MMAs of one
                          512-long K chunk then run while the previous one is drained),
                          a separate Gamma launch 80, P_ab / P_ij 64 */
  const char* autotune_cache; /* NULL, or a text file "<key> <variant>" per line: a plan
                                 whose key (precision, slices, shapes) is listed starts with
                                 that variant and skips the trials; new results are
                                 appended */
  int32_t slices_g;    /* split modes: slices of the Gamma operands: the leading slices_g
                          digit planes of Tt (one scale per fragment) and B with one scale
                          per aux index Q; range 2..8 (BF16), 2..16 (FP8); 0 = default
                          (BF16: 5, i.e. 45 bits against the per-aux-index scale of B;
                          FP8: slices_t).  Equal to slices_t, Gamma runs in P's launch;
                          fewer give a separate, cheaper Gamma launch */
  double scs_os, scs_ss; /* weights of the opposite- and same-spin components in
                            batch.energy_scs (rimp2_default_options: Grimme's SCS-MP2,
                            6/5 and 1/3; SOS-MP2 is 1.3 and 0) */
} rimp2_options;

typedef struct rimp2_stats {
  double flops_per_call;   /* algorithmic 2mnk count, V over pairs i<=j */
  double last_ms;          /* device time of the last call (0 until measured) */
  int64_t calls;
  int64_t tiles_per_call;  /* work-queue entries popped per call */
  int32_t launches_per_call; /* kernels launched per call */
  int32_t waves;
  int32_t graph_captures;
  int32_t status;          /* last status word seen by rimp2_get_status */
  int32_t tune_variant;    /* contraction-stage variant in use (see autotune) */
  int32_t tune_done;       /* 1 once the autotune trials finished (or were cached) */
  double tune_ms[4];       /* autotune: contraction-stage ms measured for each variant */
  double stage_ms[4];      /* with profile_stages: device ms of the last call, summed over
                              waves: [0] input checks and operand slicing, [1] V GEMM with the
                              T = V/D epilogue, [2] amplitudes, pair/total energies, zeroing,
                              [3] Gamma / P_ab / P_ij contractions */
  int32_t slices[3];       /* split modes: digit slices in use for V, P_ab / P_ij, Gamma */
  int32_t pad;
  double launch_ms[2];     /* with profile_stages: stage [3] split by launch: [0] the P_ab /
                              P_ij launch (with Gamma when it has their slice count), [1] the
                              separate Gamma launch (0 when none) */
  double tc_flops[4];      /* split modes: tensor-core FLOPs issued per call (2 x 128 x n_tile
                              x K x digit products, summed over the tiles computed, padding
                              included, skipped symmetric tiles excluded): [0] V, [1] the
                              P_ab / P_ij launch, [2] the separate Gamma launch, [3] unused */
  int32_t n_tile[3];       /* split modes: tile shape in use (accumulator columns, K per
                              pipeline stage) of the V, P_ab / P_ij and Gamma launches */
  int32_t stage_k[3];
  int32_t tune_trials;     /* autotune: calls that run a trial (tile shapes, then variants) */
  int32_t pad2;
} rimp2_stats;

typedef struct rimp2_plan rimp2_plan;

/* Fills *opt with the defaults listed above. */
void rimp2_default_options(rimp2_options* opt);

/* Creates a plan for nfrag fragments with the given shapes and precision.  Offsets are
 * ignored here except for the "not requested" markers: gamma_off, pij_off or pab_off
 * = -1 at plan creation sizes the workspace without that output (an energy-only plan
 * needs no Tt and no digit planes), and later calls may not request it
 * (RIMP2_ERR_SHAPE).  opt may be NULL (defaults).  Allocates the plan's small device block
 * on the current device.  Returns RIMP2_ERR_BAD_ARG for null/negative inputs,
 * RIMP2_ERR_UNSUPPORTED for an unknown precision or slice count. */
int rimp2_plan_create(const rimp2_frag* frags, int32_t nfrag, int32_t precision,
                      const rimp2_options* opt, rimp2_plan** out);

/* Bytes of device workspace rimp2_energy_grad needs (256-byte aligned pointer). */
int rimp2_workspace_size(const rimp2_plan* plan, size_t* bytes);

/* Asynchronous on `stream` (a cudaStream_t; NULL = legacy default stream): computes E
 * for every fragment and Gamma / P_ij / P_ab / e_pair where requested.  workspace must
 * hold rimp2_workspace_size() bytes; its contents are scratch.  Host-side validation
 * errors return before anything is launched. */
int rimp2_energy_grad(rimp2_plan* plan, const rimp2_batch* batch, void* workspace,
                      size_t ws_bytes, void* stream);

/* Synchronises the plan's last call and returns its device status: RIMP2_OK,
 * RIMP2_ERR_DENOM, RIMP2_ERR_NONFINITE or RIMP2_ERR_TIMEOUT (the first one raised),
 * or RIMP2_ERR_CUDA if synchronising failed.  Clears the status word. */
int rimp2_get_status(rimp2_plan* plan);

/* Copies the plan's counters; with profile_stages it first waits for the last call. */
int rimp2_get_stats(rimp2_plan* plan, rimp2_stats* out);

void rimp2_plan_destroy(rimp2_plan* plan);

/* Static description of a status code. */
const char* rimp2_status_string(int status);

/* Library build identification: "rimp2 <version> sm_103a". */
const char* rimp2_version(void);

/* ---- no-allocation entry point (the paper has no counterpart; library plumbing) ----
 *
 * For callers that cannot allocate device memory: an allocator or framework that has
 * reserved the whole device for itself, a latency-bound loop in which cudaMalloc's
 * implicit synchronisation is not acceptable, a plug-in whose host audits or forbids
 * allocations.  It computes the FP64 energy chain of ONE fragment - input checks, V,
 * T = V / D, pair energies and E - with the kernels rimp2_energy_grad uses, but its
 * scratch is a file-scope device array of RIMP2_NOALLOC_SCRATCH_BYTES that every GPU
 * which loads the library holds until the process exits.  It calls no cudaMalloc,
 * cudaFree or other allocating routine, and reads no host buffer after it returns.
 *
 * Arguments: B[nocc][nvir][naux] and eps[nocc + nvir] (occupied then virtual) are
 * device FP64 inputs; energy (1 double) and epair ([nocc][nocc], or NULL) are device
 * outputs, overwritten.  Asynchronous on `stream` (a cudaStream_t, NULL = legacy
 * default stream).
 *
 * Errors: the return code covers host-side checks only.  Negative sizes or NULL required
 * pointers return RIMP2_ERR_BAD_ARG; a fragment whose scratch,
 * 4096 + align256(8 (nocc nvir)^2) + align256(8 nocc^2) bytes, exceeds
 * RIMP2_NOALLOC_SCRATCH_BYTES (about nocc * nvir > 2040) returns RIMP2_ERR_WORKSPACE
 * before anything is launched.  Inputs that the device check rejects (some e_a <= e_i,
 * or a NaN / Inf in B or eps) make *energy NaN; epair is then unspecified.
 *
 * The first call on a device looks up the array's device address (once per device,
 * with that device current) and so should come before any stream capture.  All calls
 * on a device share the one array and it keeps the last call's contents; each call
 * clears what must start at zero.  Calls whose kernels overlap on the GPU (different
 * streams, or different host threads) race on the array: serialise them. */
#define RIMP2_NOALLOC_SCRATCH_BYTES (32u << 20)

int rimp2_energy_fp64_noalloc(int32_t nocc, int32_t nvir, int32_t naux, const double* B,
                              const double* eps, double* energy, double* epair, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RIMP2_H */
