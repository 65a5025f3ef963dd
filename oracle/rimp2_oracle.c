/*
 * Plain FP64 CPU oracle for the per-fragment RI-MP2 energy and its gradient
 * intermediates.  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the
 * benchmark's CPU-baseline leg call it; the GPU library never does, and the two
 * share no code.
 *
 * Definitions (closed shell, no frozen core; Sec. "Notation" and the Appendix):
 *   V_ij(a,b)  = sum_Q B^Q_ia B^Q_jb                      RI integrals (ia|jb), Eq. MP2_ints
 *   D_ijab     = e_i + e_j - e_a - e_b                   denominator of the Appendix amplitudes
 *                (the printed denominator is garbled; this is the standard sign)
 *   T_ij(a,b)  = V_ij(a,b) / D_ijab                      amplitudes X^ab_ij of the Appendix
 *   Tt_ij(a,b) = 2 T_ij(a,b) - T_ij(b,a)                 the (2X - X^T) combination of Gamma
 *   E          = sum_ijab Tt_ij(a,b) V_ij(a,b)           closed-shell MP2 energy (not printed;
 *                consistent with Gamma's 2X - X^T and the 4 Gamma factor of Z)
 *   Gamma^Q_ia = sum_jb Tt_ij(a,b) B^Q_jb                Appendix Gamma, in the MO-B basis
 *                (no J^-1/2 back-transform)
 *   P_ij       = -sum_kab Tt_ik(a,b) T_jk(a,b)           Appendix D^MP2_ij
 *   P_ab       =  sum_ijc Tt_ij(a,c) T_ij(b,c)           Appendix D^MP2_ab
 *
 * Layouts: B[o][v][X] and Gamma[o][v][X] (X fastest), P_ij[o][o], P_ab[v][v],
 * e_pair[o][o] with e_pair[i][j] = sum_ab Tt_ij(a,b) V_ij(a,b).
 *
 * Loops follow the definitions directly: an outer loop over the second pair index k,
 * all T_ik for that k formed explicitly, then each sum taken term by term.  Every
 * cross-pair energy sum is Neumaier-compensated; the rest are plain FP64 sums.
 * OpenMP parallelises over independent outputs only, and the cross-pair energy is
 * added serially, so the result does not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { double s, c; } nsum;   /* Neumaier running sum */

static void nadd(nsum* a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
  else a->c += (x - t) + a->s;
  a->s = t;
}
static double nval(const nsum* a) { return a->s + a->c; }

static double dot(const double* x, const double* y, int n) {
  double s = 0.0;
  for (int q = 0; q < n; ++q) s += x[q] * y[q];
  return s;
}

/* V_ij(a,b) for all a, b (v x v, row a) */
static void pair_integrals(int v, int X, const double* Bi, const double* Bj, double* V) {
  for (int a = 0; a < v; ++a)
    for (int b = 0; b < v; ++b)
      V[(size_t)a * v + b] = dot(Bi + (size_t)a * X, Bj + (size_t)b * X, X);
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
}

int rimp2_oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/*
 * Full fragment.  Any of gamma, pij, pab, epair may be NULL.  Outputs are
 * overwritten.  Returns 0, or -1 on an allocation failure / bad size.
 * k_begin..k_end restricts the outer pair index k (for a bounded timing sample);
 * pass 0, o for the whole fragment.
 */
int rimp2_oracle_fragment_range(int o, int v, int X, const double* B, const double* eo,
                                const double* ev, int k_begin, int k_end, int nthreads,
                                double* energy, double* gamma, double* pij, double* pab,
                                double* epair) {
  if (o < 0 || v < 0 || X < 0 || k_begin < 0 || k_end > o || k_begin > k_end) return -1;
  set_threads(nthreads);
  const size_t vv = (size_t)v * v, vX = (size_t)v * X;
  double* V = (double*)malloc(sizeof(double) * ((size_t)o * vv + 1));
  double* T = (double*)malloc(sizeof(double) * ((size_t)o * vv + 1));
  double* Tt = (double*)malloc(sizeof(double) * ((size_t)o * vv + 1));
  double* eik = (double*)malloc(sizeof(double) * ((size_t)o + 1));
  if (!V || !T || !Tt || !eik) { free(V); free(T); free(Tt); free(eik); return -1; }
  if (gamma) memset(gamma, 0, sizeof(double) * (size_t)o * vX);
  if (pij) memset(pij, 0, sizeof(double) * (size_t)o * o);
  if (pab) memset(pab, 0, sizeof(double) * vv);
  if (epair) memset(epair, 0, sizeof(double) * (size_t)o * o);
  nsum E = {0.0, 0.0};

  for (int k = k_begin; k < k_end; ++k) {
    /* V_ik, T_ik, Tt_ik for every i and this k */
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < o; ++i) {
      double* Vi = V + (size_t)i * vv;
      double* Ti = T + (size_t)i * vv;
      double* Tti = Tt + (size_t)i * vv;
      pair_integrals(v, X, B + (size_t)i * vX, B + (size_t)k * vX, Vi);
      for (int a = 0; a < v; ++a)
        for (int b = 0; b < v; ++b)
          Ti[(size_t)a * v + b] = Vi[(size_t)a * v + b] / (eo[i] + eo[k] - ev[a] - ev[b]);
      for (int a = 0; a < v; ++a)
        for (int b = 0; b < v; ++b)
          Tti[(size_t)a * v + b] = 2.0 * Ti[(size_t)a * v + b] - Ti[(size_t)b * v + a];
      nsum e = {0.0, 0.0};
      for (size_t ab = 0; ab < vv; ++ab) nadd(&e, Tti[ab] * Vi[ab]);
      eik[i] = nval(&e);
    }
    for (int i = 0; i < o; ++i) {          /* serial: thread-count independent */
      nadd(&E, eik[i]);
      if (epair) epair[(size_t)i * o + k] = eik[i];
    }
    /* Gamma_i += Tt_ik B_k  (the j = k terms of sum_jb) */
    if (gamma) {
      const double* Bk = B + (size_t)k * vX;
#pragma omp parallel for schedule(static)
      for (int i = 0; i < o; ++i) {
        const double* Tti = Tt + (size_t)i * vv;
        for (int a = 0; a < v; ++a) {
          double* g = gamma + (size_t)i * vX + (size_t)a * X;
          for (int b = 0; b < v; ++b) {
            const double t = Tti[(size_t)a * v + b];
            const double* bb = Bk + (size_t)b * X;
            for (int q = 0; q < X; ++q) g[q] += t * bb[q];
          }
        }
      }
    }
    /* P_ab += sum_i sum_c Tt_ik(a,c) T_ik(b,c) */
    if (pab) {
#pragma omp parallel for schedule(static)
      for (int a = 0; a < v; ++a)
        for (int b = 0; b < v; ++b) {
          double s = 0.0;
          for (int i = 0; i < o; ++i)
            s += dot(Tt + (size_t)i * vv + (size_t)a * v, T + (size_t)i * vv + (size_t)b * v, v);
          pab[(size_t)a * v + b] += s;
        }
    }
    /* P_ij -= sum_ab Tt_ik(a,b) T_jk(a,b) */
    if (pij) {
#pragma omp parallel for schedule(static)
      for (int i = 0; i < o; ++i)
        for (int j = 0; j < o; ++j)
          pij[(size_t)i * o + j] -= dot(Tt + (size_t)i * vv, T + (size_t)j * vv, (int)vv);
    }
  }
  if (energy) *energy = nval(&E);
  free(V); free(T); free(Tt); free(eik);
  return 0;
}

int rimp2_oracle_fragment(int o, int v, int X, const double* B, const double* eo,
                          const double* ev, int nthreads, double* energy, double* gamma,
                          double* pij, double* pab, double* epair) {
  return rimp2_oracle_fragment_range(o, v, X, B, eo, ev, 0, o, nthreads, energy, gamma, pij,
                                     pab, epair);
}

/* ---- single outputs, one at a time, for sampling at sizes where the full
 *      fragment is too slow on a CPU.  Same definitions as above. ---- */

static double Tval(int v, int X, const double* B, const double* eo, const double* ev, int i,
                   int j, int a, int b) {
  const size_t vX = (size_t)v * X;
  return dot(B + i * vX + (size_t)a * X, B + j * vX + (size_t)b * X, X) /
         (eo[i] + eo[j] - ev[a] - ev[b]);
}

/* e_pair[i][j] = sum_ab Tt_ij(a,b) V_ij(a,b) */
double rimp2_oracle_pair_energy(int o, int v, int X, const double* B, const double* eo,
                                const double* ev, int i, int j, int nthreads) {
  (void)o;
  set_threads(nthreads);
  const size_t vv = (size_t)v * v, vX = (size_t)v * X;
  double* V = (double*)malloc(sizeof(double) * (vv + 1));
  if (!V) return NAN;
#pragma omp parallel for schedule(static)
  for (int a = 0; a < v; ++a)
    for (int b = 0; b < v; ++b)
      V[(size_t)a * v + b] = dot(B + i * vX + (size_t)a * X, B + j * vX + (size_t)b * X, X);
  nsum e = {0.0, 0.0};
  for (int a = 0; a < v; ++a)
    for (int b = 0; b < v; ++b) {
      double tab = V[(size_t)a * v + b] / (eo[i] + eo[j] - ev[a] - ev[b]);
      double tba = V[(size_t)b * v + a] / (eo[i] + eo[j] - ev[b] - ev[a]);
      nadd(&e, (2.0 * tab - tba) * V[(size_t)a * v + b]);
    }
  free(V);
  return nval(&e);
}

/* Gamma^Q_ia = sum_j sum_b Tt_ij(a,b) B^Q_jb */
double rimp2_oracle_gamma_elem(int o, int v, int X, const double* B, const double* eo,
                               const double* ev, int i, int a, int Q, int nthreads) {
  set_threads(nthreads);
  const size_t vX = (size_t)v * X;
  double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (int j = 0; j < o; ++j)
    for (int b = 0; b < v; ++b) {
      double tt = 2.0 * Tval(v, X, B, eo, ev, i, j, a, b) - Tval(v, X, B, eo, ev, i, j, b, a);
      s += tt * B[j * vX + (size_t)b * X + Q];
    }
  return s;
}

/* P_ab = sum_i sum_j sum_c Tt_ij(a,c) T_ij(b,c) */
double rimp2_oracle_pab_elem(int o, int v, int X, const double* B, const double* eo,
                             const double* ev, int a, int b, int nthreads) {
  set_threads(nthreads);
  double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(dynamic)
  for (int ij = 0; ij < o * o; ++ij) {
    int i = ij / o, j = ij % o;
    for (int c = 0; c < v; ++c) {
      double tt = 2.0 * Tval(v, X, B, eo, ev, i, j, a, c) - Tval(v, X, B, eo, ev, i, j, c, a);
      s += tt * Tval(v, X, B, eo, ev, i, j, b, c);
    }
  }
  return s;
}

/* P_ij = -sum_k sum_a sum_b Tt_ik(a,b) T_jk(a,b) */
double rimp2_oracle_pij_elem(int o, int v, int X, const double* B, const double* eo,
                             const double* ev, int i, int j, int nthreads) {
  set_threads(nthreads);
  const size_t vv = (size_t)v * v, vX = (size_t)v * X;
  double s = 0.0;
  int fail = 0;
#pragma omp parallel for reduction(+ : s) reduction(| : fail) schedule(dynamic)
  for (int k = 0; k < o; ++k) {
    double* Vik = (double*)malloc(sizeof(double) * (2 * vv + 1));
    if (!Vik) { fail = 1; continue; }
    double* Vjk = Vik + vv;
    pair_integrals(v, X, B + i * vX, B + k * vX, Vik);
    pair_integrals(v, X, B + j * vX, B + k * vX, Vjk);
    double acc = 0.0;
    for (int a = 0; a < v; ++a)
      for (int b = 0; b < v; ++b) {
        double tab = Vik[(size_t)a * v + b] / (eo[i] + eo[k] - ev[a] - ev[b]);
        double tba = Vik[(size_t)b * v + a] / (eo[i] + eo[k] - ev[b] - ev[a]);
        double tj = Vjk[(size_t)a * v + b] / (eo[j] + eo[k] - ev[a] - ev[b]);
        acc += (2.0 * tab - tba) * tj;
      }
    s += acc;
    free(Vik);
  }
  return fail ? NAN : -s;
}

/* ---- spin components of the closed-shell energy (SCS-MP2 is named in the Introduction;
 *      the paper prints no formula).  In spatial orbitals:
 *        E_OS = sum_ijab T_ij(a,b) V_ij(a,b)                  opposite spin (alpha-beta)
 *        E_SS = sum_ijab (T_ij(a,b) - T_ij(b,a)) V_ij(a,b)    same spin (alpha-alpha + beta-beta)
 *      so that E = E_OS + E_SS.  Pair by pair, each term as defined. ---- */

static void pair_spin(int v, int X, const double* B, const double* eo, const double* ev, int i,
                      int j, double* V, nsum* os, nsum* ss) {
  const size_t vX = (size_t)v * X;
  pair_integrals(v, X, B + (size_t)i * vX, B + (size_t)j * vX, V);
  for (int a = 0; a < v; ++a)
    for (int b = 0; b < v; ++b) {
      const double vab = V[(size_t)a * v + b];
      const double tab = vab / (eo[i] + eo[j] - ev[a] - ev[b]);
      const double tba = V[(size_t)b * v + a] / (eo[i] + eo[j] - ev[b] - ev[a]);
      nadd(os, tab * vab);
      nadd(ss, (tab - tba) * vab);
    }
}

/* E_OS and E_SS of a fragment (either pointer may be NULL).  Returns 0 or -1. */
int rimp2_oracle_spin_components(int o, int v, int X, const double* B, const double* eo,
                                 const double* ev, int nthreads, double* e_os, double* e_ss) {
  if (o < 0 || v < 0 || X < 0) return -1;
  set_threads(nthreads);
  const size_t vv = (size_t)v * v, np = (size_t)o * o;
  double* pos = (double*)malloc(sizeof(double) * (np + 1));
  double* pss = (double*)malloc(sizeof(double) * (np + 1));
  if (!pos || !pss) { free(pos); free(pss); return -1; }
  int bad = 0;
#pragma omp parallel
  {
    double* V = (double*)malloc(sizeof(double) * (vv + 1));
    if (!V) {
#pragma omp atomic write
      bad = 1;
    }
#pragma omp for schedule(dynamic)
    for (long long ij = 0; ij < (long long)np; ++ij) {
      if (!V) continue;
      nsum os = {0.0, 0.0}, ss = {0.0, 0.0};
      pair_spin(v, X, B, eo, ev, (int)(ij / o), (int)(ij % o), V, &os, &ss);
      pos[ij] = nval(&os);
      pss[ij] = nval(&ss);
    }
    free(V);
  }
  nsum os = {0.0, 0.0}, ss = {0.0, 0.0};
  for (size_t ij = 0; ij < np; ++ij) {   /* serial: thread-count independent */
    nadd(&os, pos[ij]);
    nadd(&ss, pss[ij]);
  }
  free(pos); free(pss);
  if (bad) return -1;
  if (e_os) *e_os = nval(&os);
  if (e_ss) *e_ss = nval(&ss);
  return 0;
}

/* Spin components of one pair (i, j): out[0] = opposite spin, out[1] = same spin. */
int rimp2_oracle_pair_spin(int o, int v, int X, const double* B, const double* eo,
                           const double* ev, int i, int j, double* out) {
  if (i < 0 || j < 0 || i >= o || j >= o) return -1;
  double* V = (double*)malloc(sizeof(double) * ((size_t)v * v + 1));
  if (!V) return -1;
  nsum os = {0.0, 0.0}, ss = {0.0, 0.0};
  pair_spin(v, X, B, eo, ev, i, j, V, &os, &ss);
  free(V);
  out[0] = nval(&os);
  out[1] = nval(&ss);
  return 0;
}
