/*
 * rimp2_testing.h - test hooks of librimp2 (not part of the production ABI).
 *
 * rimp2_testing_slice_gemm runs the split-precision tensor-core GEMM kernel alone on
 * caller-supplied digit planes, so tests can compare it with exact integer products:
 *
 *   C[m][n] = sum_{p + q < slices} 2^(-8 (p + q)) sum_{k < K} A[p][m][k] B[q][n][k]
 *
 * A: BF16 [slices][M][kpad], B: BF16 [slices][N][kpad] (device, row stride kpad
 * elements, kpad a multiple of 8 and >= K), integer values in [-128, 128].
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

#ifdef __cplusplus
}
#endif

#endif /* RIMP2_TESTING_H */
