/*
 * rimp2_testing.h - test hooks of librimp2 (not part of the production ABI).
 *
 * rimp2_testing_slice_gemm runs the split-precision tensor-core GEMM kernel alone on
 * caller-supplied digit planes, so tests can compare it with exact integer products:
 *
 *   C[m][n] = sum_{p + q < slices} 2^(-9 (p + q)) sum_{k < K} A[p][m][k] B[q][n][k]
 *
 * A: BF16 [slices][M][kpad], B: BF16 [slices][N][kpad] (device, row stride kpad
 * elements, kpad a multiple of 8 and >= K), integer values in [-256, 256].
 * C: FP64 [M][N] (device), overwritten.  Synchronous (allocates a small descriptor
 * buffer, launches on `stream`, synchronises, frees).  Returns RIMP2_OK, a negative
 * RIMP2_ERR_* code, or RIMP2_ERR_TIMEOUT if a bounded device wait expired.
 */
#ifndef RIMP2_TESTING_H
#define RIMP2_TESTING_H

#include "rimp2.h"

#ifdef __cplusplus
extern "C" {
#endif

int rimp2_testing_slice_gemm(int32_t M, int32_t N, int32_t K, int32_t kpad, int32_t slices,
                             const void* A, const void* B, double* C, void* stream);

/* Same with an explicit pipeline stage depth in K (BF16: stage_k = 16 for 32-byte or 32
 * for 64-byte swizzled rows) and format: fp8 != 0 takes A and B as FP8 e4m3 bytes with
 * integer values in [-16, 16], slices up to 16, kpad a multiple of 16, and
 *   C[m][n] = sum_{p + q < slices} 2^(-5 (p + q)) sum_k A[p][m][k] B[q][n][k]. */
int rimp2_testing_slice_gemm_k(int32_t M, int32_t N, int32_t K, int32_t kpad, int32_t slices,
                               int32_t stage_k, int32_t fp8, const void* A, const void* B,
                               double* C, void* stream);

/* Sets the limit of the consumer-side waits (the MMA issuer's and the epilogue's
 * mbarrier waits) of the tensor-core contraction kernel on the current device, in
 * nanoseconds; ns < 0 restores the normal 2 s.  With a limit of 0 those waits give up
 * unless one non-blocking probe finds their data already there, so a call takes the
 * abort path: the kernel
 * records RIMP2_ERR_TIMEOUT in the plan's status word, lets its own MMAs and TMA loads
 * in flight finish (bounded by the normal limit), frees its TMEM and returns.  The
 * outputs of such a call are unspecified.  Synchronous; affects every plan on the
 * device until it is set again. */
int rimp2_testing_set_wait_limit(int64_t ns);

/* FP64 throughput of the current device in TFLOP/s, measured in place (the denominators
 * of the plain FP64 path's roofline): kind 0 = CUDA-core DFMA (8 independent FMA chains
 * per thread), kind 1 = FP64 tensor path (mma.sync m8n8k4, 8 independent accumulators
 * per warp); 8 CTAs of 256 threads per SM, best of three timed runs after one warm-up.
 * Synchronous; allocates a small output buffer.  Returns RIMP2_OK, RIMP2_ERR_BAD_ARG or
 * RIMP2_ERR_CUDA. */
int rimp2_testing_fp64_peak(int32_t kind, double* tflops);

#ifdef __cplusplus
}
#endif

#endif /* RIMP2_TESTING_H */
