/*
 * rimp2_mbe.h - many-body expansion (MBE3) around the per-fragment RI-MP2 engine.
 *
 * Eq. mbe3 of arXiv 2410.21888:  E = sum_I E_I + sum_{I<J} dE_IJ + sum_{I<J<K} dE_IJK,
 * dE_IJ = E_IJ - E_I - E_J (Sec. "Molecular Fragmentation"); the trimer correction is
 * the inclusion-exclusion E_IJK - E_IJ - E_IK - E_JK + E_I + E_J + E_K.  Polymers are
 * formed from monomer centroids with distance cutoffs (Sec. "Molecular Fragmentation":
 * polymers within R_cut; centroid distances as in Sec. "Time step latency").
 *
 * All functions return RIMP2_OK or a negative RIMP2_ERR_* code (see rimp2.h).
 */
#ifndef RIMP2_MBE_H
#define RIMP2_MBE_H

#include "rimp2.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Trimer membership rules */
#define RIMP2_TRIMER_MAX_PAIR 0  /* all three centroid distances <= r_trimer */
#define RIMP2_TRIMER_TWO_PAIRS 1 /* at least two of the three distances <= r_trimer */

/* Polymer formation (host).  centroids: host [n][3] (bohr).  Dimers: pairs I<J with
 * |R_I - R_J| <= r_dimer, written as [I, J] to dimers[0 .. min(*n_dimers, cap_d))].
 * Trimers: I<J<K under `trimer_rule` with r_trimer, written as [I, J, K].  The counts
 * are returned in *n_dimers / *n_trimers even when they exceed the capacities (pass a
 * capacity of 0 and NULL arrays to query sizes).  Lists are in lexicographic order. */
int rimp2_mbe_polymers(const double* centroids, int32_t n, double r_dimer, double r_trimer,
                       int32_t trimer_rule, int32_t* dimers, int64_t cap_d, int64_t* n_dimers,
                       int32_t* trimers, int64_t cap_t, int64_t* n_trimers);

/* Inclusion-exclusion bookkeeping (host).  Given n monomers, the dimers kept in the
 * expansion and the trimers kept, returns the list of fragments whose energies are
 * needed (every monomer, every kept dimer, every pair inside a kept trimer, every kept
 * trimer) and integer coefficients c_f with E_MBE3 = sum_f c_f E_f.  Fragments are
 * written as 3 int32 monomer ids each, padded with -1 ([I,-1,-1], [I,J,-1], [I,J,K]),
 * ordered monomers, then pairs, then triples (each lexicographic).  Query the size with
 * cap = 0. */
int rimp2_mbe_coefficients(int32_t n, const int32_t* dimers, int64_t nd, const int32_t* trimers,
                           int64_t nt, int32_t* frags, int32_t* coeff, int64_t cap,
                           int64_t* nfrag);

/* Device: *out = sum_f coeff[f] * energy[f] in FP64 with a compensated (TwoSum) sum in
 * a fixed order (deterministic).  energy, coeff, out are device pointers.  Asynchronous
 * on `stream`. */
int rimp2_mbe_combine(const double* energy, const int32_t* coeff, int64_t nfrag, double* out,
                      void* stream);

/* Device: per-polymer corrections out[t] = sum_q sign[q] * energy[terms[t][q]] for
 * q < k (e.g. k = 3, signs {+1,-1,-1}, terms {IJ, I, J} for dimers; k = 7, signs
 * {+1,-1,-1,-1,+1,+1,+1}, terms {IJK, IJ, IK, JK, I, J, K} for trimers), in FP64.
 * terms [n][k] int32 (device), sign [k] int32 (device).  If out_log10 is not NULL it
 * also receives log10(|out[t]| + 1e-16) as FP32 (the screen's regression target). */
int rimp2_mbe_corrections(const double* energy, const int32_t* terms, const int32_t* sign,
                          int64_t n, int32_t k, double* out, float* out_log10, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RIMP2_MBE_H */
