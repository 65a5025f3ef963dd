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

/* ---- MBE3 assembly of the gradient intermediates over the system's index spaces ----
 *
 * E_MBE3 = sum_f c_f E_f, and every fragment sees a restriction of one global B and one
 * set of orbital energies (occupied, virtual and auxiliary orbitals of all monomers,
 * concatenated monomer by monomer).  The MBE3 derivatives are therefore the
 * coefficient-weighted scatters of the fragments' intermediates:
 *   P_ij_sys[(I,i),(J,j)]       = sum_f c_f P_ij,f[(I,i),(J,j)]    (dE/de_k = 2 P_kk, ...)
 *   P_ab_sys[(I,a),(J,b)]       = sum_f c_f P_ab,f[(I,a),(J,b)]
 *   Gamma_sys[(I,J,K)][i][a][Q] = sum_f c_f Gamma_f[(I,i)][(J,a)][(K,Q)]   (dE/dB = 4 Gamma)
 * over the fragments f holding the monomers involved.  The trimer coefficients are all 1,
 * which is why the paper accumulates trimer gradients directly into the system gradient
 * (Sec. "Asynchronous time steps"); here any level, or any chunk of trimers, can be added
 * to the system arrays as soon as its fragments are done (accumulate = 1), so their
 * per-fragment pools can be reused.
 *
 * Gamma_sys holds every block (I,J,K) of monomers that occur together in a fragment, each
 * [nocc_I][nvir_J][naux_K] (naux fastest), at the element offset given by the block
 * index; P_ij_sys is dense [O][O] (O = sum nocc), P_ab_sys dense [V][V] (V = sum nvir). */
typedef struct rimp2_assembly rimp2_assembly;

/* Host description.  n monomers with nocc[n], nvir[n], naux[n]; nfrag fragments as up to
 * three monomer ids frag_mon[3 f + p] (-1 padded, the monomers in the order the fragment
 * concatenates its orbitals), integer coefficients coeff[f], and the element offsets of
 * each fragment's Gamma, P_ij and P_ab in the batch pools of rimp2_batch (-1: the output
 * takes no contribution from that fragment; then pass NULL or any pointer for that pool).
 * Builds the block list and, per output block, its contributors in fragment order; the
 * device tables are owned by the handle (current device). */
int rimp2_assembly_create(int32_t n, const int32_t* nocc, const int32_t* nvir,
                          const int32_t* naux, int64_t nfrag, const int32_t* frag_mon,
                          const int32_t* coeff, const int64_t* gamma_off, const int64_t* pij_off,
                          const int64_t* pab_off, rimp2_assembly** out);

/* Sizes: elements of the Gamma_sys buffer, O and V. */
int rimp2_assembly_sizes(const rimp2_assembly* a, int64_t* gamma_elems, int64_t* o_total,
                         int64_t* v_total);

/* Host copy of the block index: index[(I n + J) n + K] = element offset of block (I,J,K)
 * in Gamma_sys, or -1 (n^3 entries). */
int rimp2_assembly_block_index(const rimp2_assembly* a, int64_t* index);

/* Device, asynchronous on `stream`: writes (accumulate = 0) or adds (accumulate = 1)
 * Gamma_sys, P_ij_sys and P_ab_sys from the fragments' pools.  Each output element sums
 * its contributors in fragment order (deterministic, no atomics); accumulate = 0 also
 * zeroes the entries of P_sys that no fragment touches.  An output pointer may be NULL
 * to skip it. */
int rimp2_assembly_run(const rimp2_assembly* a, const double* gamma, const double* pij,
                       const double* pab, double* gamma_sys, double* pij_sys, double* pab_sys,
                       int32_t accumulate, void* stream);

void rimp2_assembly_destroy(rimp2_assembly* a);

#ifdef __cplusplus
}
#endif

#endif /* RIMP2_MBE_H */
