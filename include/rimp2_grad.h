/*
 * rimp2_grad.h - the step of the RI-MP2 gradient after the unrelaxed densities
 * (Appendix of arXiv 2410.21888), for one fragment, FP64 on the device:
 *
 *   Gamma^P_ia = sum_Q Gamma^Q_ia J^{-1/2}_PQ                      (auxiliary quantities)
 *   L'_iq  = sum_aP Gamma^P_ia (P|qa),  L''_aq = sum_iP Gamma^P_ia (P|iq)
 *   (e_a - e_i)/2 D_ai + sum_bj G^{bj}_ai D_bj
 *          = L''_ai - L'_ia - sum_pq G^{pq}_ai Dbar_pq               (Z-vector equation)
 *   G^{rs}_pq = 2 (pq|rs)_RI - (ps|rq)_RI,  (pq|rs)_RI = sum_Q B^Q_pq B^Q_rs,
 *   Dbar = D_ij (+) D_ab, the unrelaxed densities P_ij and P_ab of rimp2_energy_grad.
 *
 * B^Q_pq = sum_P (pq|P) J^{-1/2}_PQ, so (P|pq) = sum_Q B^Q_pq J^{1/2}_QP and
 * L'_iq = sum_aQ Gamma^Q_ia B^Q_qa, L''_aq = sum_iQ Gamma^Q_ia B^Q_iq: L' and L'' need
 * neither J^{1/2} nor the back-transformed Gamma.  The Z-vector equation is solved by
 * conjugate gradients with the diagonal (e_a - e_i)/2 + (ai|ai) as preconditioner; the
 * operator's matrix is symmetric, and positive definite when the orbital gaps dominate
 * the integrals (conjugate gradients then converge).
 *
 * All functions return RIMP2_OK or a negative RIMP2_ERR_* code (see rimp2.h).
 */
#ifndef RIMP2_GRAD_H
#define RIMP2_GRAD_H

#include "rimp2.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rimp2_zvec_args {
  int32_t nocc, nvir, naux;  /* n = nocc + nvir molecular orbitals, occupied first */
  int32_t max_iter;          /* conjugate-gradient iterations at most (0: 100) */
  double tol;                /* stop once ||r|| <= tol ||rhs|| (0: 1e-12) */
  const double* Bf;          /* device [n][n][naux]: B^Q_pq, naux fastest, symmetric in p, q */
  const double* eps;         /* device [n]: orbital energies (occupied first) */
  const double* jmh;         /* device [naux][naux]: J^{-1/2} (symmetric), or NULL */
  const double* gamma;       /* device [nocc][nvir][naux]: Gamma^Q_ia of rimp2_energy_grad */
  const double* pij;         /* device [nocc][nocc]: D^MP2_ij (P_ij) */
  const double* pab;         /* device [nvir][nvir]: D^MP2_ab (P_ab) */
  double* gamma_p;           /* device out [nocc][nvir][naux]: Gamma^P_ia (NULL: skipped;
                                also skipped when jmh is NULL) */
  double* lp;                /* device out [nocc][n]: L'_iq */
  double* lpp;               /* device out [nvir][n]: L''_aq */
  double* dai;               /* device out [nocc][nvir]: D_ai stored at [i][a] */
  double* info;              /* device out [3]: iterations taken, ||r|| / ||rhs||, ||rhs||
                                (iterations = max_iter + 1 when the tolerance was not met) */
} rimp2_zvec_args;

/* Workspace bytes for one fragment of these sizes (device memory the caller owns; 256-byte
 * aligned; contents need not be initialised).  Host only. */
int rimp2_zvec_workspace_size(int32_t nocc, int32_t nvir, int32_t naux, int32_t max_iter,
                              size_t* bytes);

/* Enqueues the step on `stream`.  Outputs are overwritten.  The problem descriptors are
 * staged from host memory into the workspace during the call, which therefore waits for
 * the work already queued on the stream and is not stream-capturable; the step itself
 * runs asynchronously (the conjugate-gradient iterations are all enqueued; those after
 * convergence return at once on the device).  Errors: RIMP2_ERR_BAD_ARG for negative
 * sizes or a NULL required pointer, RIMP2_ERR_WORKSPACE when the workspace is NULL, not
 * 256-byte aligned or below rimp2_zvec_workspace_size, RIMP2_ERR_UNSUPPORTED when the
 * descriptor lists outgrow their 1 MB region (nocc above ~2000), RIMP2_ERR_CUDA for a
 * failed launch or copy. */
int rimp2_zvec_solve(const rimp2_zvec_args* args, void* workspace, size_t ws_bytes,
                     cudaStream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* RIMP2_GRAD_H */
