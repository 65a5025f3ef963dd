/*
 * rimp2_mlp.h - learned trimer screen: a small MLP that predicts log10|dE_IJK| of a
 * trimer's many-body correction from its geometry and dimer corrections, trained and
 * run by the library's own kernels.  The paper sets its trimer cutoff by an explicit
 * reference-monomer MBE study (Sec. "Molecular Fragmentation", Sec. "Time step
 * latency": contributions below 0.1 kJ/mol are dropped); this screen replaces that
 * study with a model trained on corrections the method itself computed.
 *
 * Network: 9 -> 64 -> 64 -> 64 -> 1, SiLU after each hidden layer, linear output.
 * Parameters are one FP32 master vector (layout below); the forward pass uses a BF16
 * copy of the weights and biases with FP32 accumulation.
 *   layer l = 1..4 with (in, out) = (9,64), (64,64), (64,64), (64,1):
 *   W_l [out][in] row-major, then b_l [out]; layers consecutive.  RIMP2_MLP_PARAMS total.
 * Features (9 per trimer, FP32): the three centroid distances (ascending), the three
 * monomer nocc (ascending), log10(|dE_IJ| + 1e-16) of the three dimer corrections
 * (ascending).  Kernels standardise them with the caller's mean/std vectors (9 each).
 * Loss: mean squared error of the prediction against the target, over the minibatch.
 *
 * All pointers are device pointers unless stated; calls are asynchronous on `stream`;
 * returns RIMP2_OK or a negative RIMP2_ERR_* code (rimp2.h).
 */
#ifndef RIMP2_MLP_H
#define RIMP2_MLP_H

#include "rimp2.h"

#ifdef __cplusplus
extern "C" {
#endif

#define RIMP2_MLP_IN 9
#define RIMP2_MLP_HIDDEN 64
#define RIMP2_MLP_PARAMS (64 * 9 + 64 + 64 * 64 + 64 + 64 * 64 + 64 + 64 + 1)

/* Trimer features from centroids [n][3] (FP64), monomer nocc [n] (int32), trimers
 * [nt][3] (int32 monomer ids) and a dense [n][n] table of dimer corrections (FP64,
 * symmetric; pairs not computed hold 0).  Output feats [nt][9] (FP32). */
int rimp2_screen_features(const double* centroids, const int32_t* nocc, int32_t n,
                          const int32_t* trimers, int64_t nt, const double* dimer_de,
                          float* feats, void* stream);

/* Gradient of the minibatch loss with respect to the FP32 master parameters (written,
 * not accumulated, to grad[RIMP2_MLP_PARAMS]); loss (1 float, may be NULL).  The
 * minibatch is rows idx[0..n) of feats [*][9] with targets y[*]; idx NULL = rows 0..n. */
int rimp2_mlp_grad(const float* master, const float* feats, const float* y, const int32_t* idx,
                   int32_t n, const float* mean, const float* std, float* grad, float* loss,
                   void* stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected with step t >= 1) on
 * master using grad, state m and v (each RIMP2_MLP_PARAMS floats). */
int rimp2_mlp_adam(float* master, const float* grad, float* m, float* v, int32_t t, float lr,
                   void* stream);

/* Predictions out[n] = MLP(feats[n][9]) with BF16 weights rounded from master. */
int rimp2_mlp_predict(const float* master, const float* feats, int64_t n, const float* mean,
                      const float* std, float* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RIMP2_MLP_H */
