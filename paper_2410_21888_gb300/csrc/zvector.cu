// The step of the RI-MP2 gradient after the unrelaxed densities (Appendix), one fragment,
// FP64 (include/rimp2_grad.h):
//   Gamma^P = Gamma^Q J^{-1/2};  L'_iq = sum_aQ Gamma^Q_ia B^Q_qa;  L''_aq = sum_iQ Gamma^Q_ia B^Q_iq
//   and the Z-vector equation for D_ai by preconditioned conjugate gradients.
//
// With x[i][a] = D_ai, the operator of the Z-vector equation is
//   (A x)_ia = (e_a - e_i)/2 x_ia + 2 sum_Q B^Q_ia c^Q - sum_jQ B^Q_ja W^Q_ij,
//   c^Q = sum_jb B^Q_jb x_jb,  W^Q_ij = sum_b B^Q_ib x_jb,
// the Coulomb part 2 (ai|bj) and the exchange part (aj|bi) of G^{bj}_ai.  The right-hand
// side L''_ai - L'_ia - sum_pq G^{pq}_ai Dbar_pq expands the same way:
//   sum_kl G^{kl}_ai D_kl = 2 sum_Q B^Q_ia d^Q - sum_lQ B^Q_la U^Q_il,
//   sum_bc G^{bc}_ai D_bc = 2 sum_Q B^Q_ia e^Q - sum_cQ B^Q_ac V^Q_ic,
//   d^Q = sum_kl B^Q_kl D_kl, e^Q = sum_bc B^Q_bc D_bc, U^Q_il = sum_k B^Q_ik D_kl,
//   V^Q_ic = sum_b B^Q_ib D_bc.
// The contractions with a K of naux or more run on the grouped FP64 GEMM (PK_GEN problems
// on caller pointers); the sums over one index run as column or row sums; the
// conjugate-gradient scalars live on the device and every iteration's kernels return at
// once after convergence, so the host enqueues all iterations without waiting.
#include <algorithm>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "rimp2_grad.h"
#include "rimp2_internal.cuh"

namespace rimp2 {
namespace {

constexpr int kColRows = 64;      // rows per CTA of the column sums (at least)
constexpr int kCgThreads = 1024;  // the single CTA of the conjugate-gradient updates

// device scalars of the solve
struct CgState {
  double rz, bnorm, rnorm, pad;
  int done, iters, pad2, pad3;
};

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

// out[Q] += sum_r w[r] M[r][Q] for rows r = (r1, r0) at base + r1 s1 + r0 s0, w[r1 * R0 + r0]
__global__ void __launch_bounds__(256)
k_colsum(const double* __restrict__ base, long long s1, long long s0, int R1, int R0,
         const double* __restrict__ w, int X, int rows_per, double* __restrict__ out,
         const int* __restrict__ skip) {
  if (skip && *(volatile const int*)skip) return;
  const int Q = blockIdx.x * blockDim.x + threadIdx.x;
  if (Q >= X) return;
  const long long R = (long long)R1 * R0;
  const long long r0 = (long long)blockIdx.y * rows_per;
  const long long r1 = min(R, r0 + rows_per);
  double s = 0.0;
  for (long long r = r0; r < r1; ++r) {
    const int a = (int)(r / R0), b = (int)(r - (long long)a * R0);
    s = fma(w[r], base[a * s1 + b * s0 + Q], s);
  }
  atomicAdd(out + Q, s);
}

// One warp per row (i,a) of the ov block of B: s1 = sum_Q B^Q_ia vec[Q], s2 = sum_Q (B^Q_ia)^2.
//   mode 0: rhs[r] = L''_ai - L'_ia - 2 s1 (vec = d + e); diag[r] = (e_a - e_i)/2 + s2
//   mode 1: y[r] = (e_a - e_i)/2 x[r] + 2 s1 (vec = c)
__global__ void __launch_bounds__(256)
k_rows(const double* __restrict__ Bf, const double* __restrict__ eps, int o, int v, int X,
       const double* __restrict__ vec, int mode, const double* __restrict__ lp,
       const double* __restrict__ lpp, double* __restrict__ rhs, double* __restrict__ diag,
       const double* __restrict__ x, double* __restrict__ y, const int* __restrict__ skip) {
  if (skip && *(volatile const int*)skip) return;
  const long long r = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= (long long)o * v) return;
  const int i = (int)(r / v), a = (int)(r - (long long)i * v);
  const int n = o + v;
  const double* row = Bf + ((long long)i * n + o + a) * X;
  double s1 = 0.0, s2 = 0.0;
  for (int Q = lane; Q < X; Q += 32) {
    const double b = row[Q];
    s1 = fma(b, vec[Q], s1);
    s2 = fma(b, b, s2);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, off);
    s2 += __shfl_xor_sync(0xffffffffu, s2, off);
  }
  if (lane != 0) return;
  const double hg = 0.5 * (eps[o + a] - eps[i]);
  if (mode == 0) {
    rhs[r] = lpp[(long long)a * n + i] - lp[(long long)i * n + o + a] - 2.0 * s1;
    diag[r] = hg + s2;
  } else {
    y[r] = hg * x[r] + 2.0 * s1;
  }
}

// deterministic block sum over kCgThreads threads (every thread gets the result)
__device__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    if (lane == 0) sh[32] = t;
  }
  __syncthreads();
  return sh[32];
}

// start: x = 0, r = rhs, z = r / diag, p = z, rz = r.z, bnorm = ||rhs||, c = 0
__global__ void __launch_bounds__(kCgThreads)
k_cg_init(long long N, const double* __restrict__ rhs, const double* __restrict__ diag,
          double* __restrict__ x, double* __restrict__ r, double* __restrict__ z,
          double* __restrict__ p, double* __restrict__ c, int X, CgState* st, double* info) {
  __shared__ double sh[33];
  double rz = 0.0, bb = 0.0;
  for (long long k = threadIdx.x; k < N; k += blockDim.x) {
    const double b = rhs[k], zk = b / diag[k];
    x[k] = 0.0; r[k] = b; z[k] = zk; p[k] = zk;
    rz = fma(b, zk, rz);
    bb = fma(b, b, bb);
  }
  for (int q = threadIdx.x; q < X; q += blockDim.x) c[q] = 0.0;
  rz = block_sum(rz, sh);
  bb = block_sum(bb, sh);
  if (threadIdx.x == 0) {
    st->rz = rz;
    st->bnorm = sqrt(bb);
    st->rnorm = st->bnorm;
    st->done = bb == 0.0;
    st->iters = 0;
    info[0] = 0.0; info[1] = 0.0; info[2] = st->bnorm;
  }
}

// one conjugate-gradient step after Ap = A p:
//   alpha = rz / p.Ap; x += alpha p; r -= alpha Ap; stop if ||r|| <= tol ||b||;
//   z = r / diag; beta = r.z / rz; p = z + beta p; c = 0 for the next product
__global__ void __launch_bounds__(kCgThreads)
k_cg_step(long long N, const double* __restrict__ diag, double* __restrict__ x,
          double* __restrict__ r, double* __restrict__ z, double* __restrict__ p,
          const double* __restrict__ Ap, double* __restrict__ c, int X, double tol, int it,
          CgState* st, double* info) {
  __shared__ double sh[33];
  if (*(volatile int*)&st->done) return;
  double pap = 0.0;
  for (long long k = threadIdx.x; k < N; k += blockDim.x) pap = fma(p[k], Ap[k], pap);
  pap = block_sum(pap, sh);
  const double alpha = pap != 0.0 ? st->rz / pap : 0.0;
  double rr = 0.0;
  for (long long k = threadIdx.x; k < N; k += blockDim.x) {
    x[k] = fma(alpha, p[k], x[k]);
    const double rk = fma(-alpha, Ap[k], r[k]);
    r[k] = rk;
    rr = fma(rk, rk, rr);
  }
  rr = block_sum(rr, sh);
  const double rnorm = sqrt(rr);
  const bool conv = rnorm <= tol * st->bnorm || pap == 0.0;
  if (!conv) {
    double rz = 0.0;
    for (long long k = threadIdx.x; k < N; k += blockDim.x) {
      const double zk = r[k] / diag[k];
      z[k] = zk;
      rz = fma(r[k], zk, rz);
    }
    rz = block_sum(rz, sh);
    const double beta = rz / st->rz;
    for (long long k = threadIdx.x; k < N; k += blockDim.x) p[k] = fma(beta, p[k], z[k]);
    for (int q = threadIdx.x; q < X; q += blockDim.x) c[q] = 0.0;
    __syncthreads();
    if (threadIdx.x == 0) st->rz = rz;
  }
  if (threadIdx.x == 0) {
    st->rnorm = rnorm;
    st->iters = it + 1;
    info[0] = conv ? (double)(it + 1) : 0.0;
    info[1] = st->bnorm > 0.0 ? rnorm / st->bnorm : 0.0;
    if (conv) st->done = 1;
  }
}

// after the last step: iterations = max_iter + 1 when the tolerance was not met
__global__ void k_cg_finish(const CgState* st, int max_iter, double* info) {
  if (!st->done) info[0] = (double)(max_iter + 1);
  else if (st->bnorm == 0.0) info[0] = 0.0;
}

// C(m,n) = alpha sum_{k1,k0} A[m sAm + k0 sAk + k1 sA1] Bop[n sBn + k0 sBk + k1 sB1]
GemmProb gen(int M, int N, int K0, int K1, const double* a, long long sAm, long long sAk,
             long long sA1, const double* b, long long sBn, long long sBk, long long sB1,
             double* c, long long ldc, double alpha, bool accumulate, int grid) {
  GemmProb P{};
  P.kind = PK_GEN;
  P.M = M; P.N = N; P.K0 = K0; P.K1 = std::max(K1, 1);
  P.tiles_m = (M + F64_BM - 1) / F64_BM;
  P.tiles_n = (N + F64_BN - 1) / F64_BN;
  P.pa = a; P.sAm = sAm; P.sAk = sAk; P.sA1 = sA1;
  P.pb = b; P.sBn = sBn; P.sBk = sBk; P.sB1 = sB1;
  P.pc = c; P.ldc = ldc; P.alpha = alpha;
  P.accumulate = accumulate ? 1 : 0;
  const long long tiles = (long long)P.tiles_m * P.tiles_n;
  long long want = 1;
  if (accumulate && tiles > 0) want = std::max(1LL, (2LL * grid + tiles - 1) / tiles);
  want = std::min<long long>(want, P.K1);
  P.k1_chunk = (int)((P.K1 + want - 1) / want);
  P.ksplit = (P.K1 + P.k1_chunk - 1) / P.k1_chunk;
  P.ntiles = tiles * P.ksplit;
  return P;
}

void finish(std::vector<GemmProb>& v, long long& total) {
  std::stable_sort(v.begin(), v.end(), [](const GemmProb& a, const GemmProb& b) {
    return (double)a.K0 * a.k1_chunk > (double)b.K0 * b.k1_chunk;
  });
  total = 0;
  for (auto& P : v) { P.tile_begin = total; total += P.ntiles; }
}

struct Layout {
  size_t w, vv, r, z, p, ap, diag, rhs, c, de, st, ctr, desc, total;
};

constexpr int kDescLists = 6;   // Gamma^P, L'/L'', U/V, rhs terms, W, exchange product
constexpr size_t kDescBytes = 1 << 20;

Layout layout(long long o, long long v, long long X, int max_iter) {
  Layout L{};
  size_t off = 0;
  const size_t ov = (size_t)(o * v);
  L.w = off; off += al256((size_t)(o * o * X) * 8);
  L.vv = off; off += al256((size_t)(o * v * X) * 8);
  L.r = off; off += al256(ov * 8);
  L.z = off; off += al256(ov * 8);
  L.p = off; off += al256(ov * 8);
  L.ap = off; off += al256(ov * 8);
  L.diag = off; off += al256(ov * 8);
  L.rhs = off; off += al256(ov * 8);
  L.c = off; off += al256((size_t)X * 8);
  L.de = off; off += al256((size_t)X * 8);
  L.st = off; off += 256;
  L.ctr = off; off += al256((size_t)(2 * max_iter + 8) * 4);
  L.desc = off; off += kDescBytes;
  L.total = off;
  return L;
}

int iters_of(const rimp2_zvec_args* a) { return a->max_iter > 0 ? a->max_iter : 100; }

}  // namespace
}  // namespace rimp2

using namespace rimp2;

extern "C" {

int rimp2_zvec_workspace_size(int32_t nocc, int32_t nvir, int32_t naux, int32_t max_iter,
                              size_t* bytes) {
  if (!bytes || nocc < 0 || nvir < 0 || naux < 0 || max_iter < 0) return RIMP2_ERR_BAD_ARG;
  *bytes = layout(nocc, nvir, naux, max_iter > 0 ? max_iter : 100).total;
  return RIMP2_OK;
}

int rimp2_zvec_solve(const rimp2_zvec_args* A, void* workspace, size_t ws_bytes,
                     cudaStream_t s) {
  if (!A || A->nocc < 0 || A->nvir < 0 || A->naux < 0 || A->max_iter < 0 || A->tol < 0)
    return RIMP2_ERR_BAD_ARG;
  const int o = A->nocc, v = A->nvir, X = A->naux, n = o + v;
  const long long ov = (long long)o * v;
  const long long X_ = X;
  // pointers are required where their arrays have elements
  if (!A->info || ((long long)o * n > 0 && !A->lp) || ((long long)v * n > 0 && !A->lpp) ||
      (ov > 0 && !A->dai) || (n > 0 && !A->eps) || ((long long)n * n * X_ > 0 && !A->Bf) ||
      (ov * X_ > 0 && !A->gamma) || (o > 0 && !A->pij) || (v > 0 && !A->pab))
    return RIMP2_ERR_BAD_ARG;
  const int max_iter = iters_of(A);
  const double tol = A->tol > 0 ? A->tol : 1e-12;
  const Layout L = layout(o, v, X, max_iter);
  if (!workspace || ((uintptr_t)workspace & 255u) || ws_bytes < L.total) return RIMP2_ERR_WORKSPACE;
  char* ws = (char*)workspace;
  double* W = (double*)(ws + L.w);
  double* Vv = (double*)(ws + L.vv);
  double* r = (double*)(ws + L.r);
  double* z = (double*)(ws + L.z);
  double* p = (double*)(ws + L.p);
  double* Ap = (double*)(ws + L.ap);
  double* diag = (double*)(ws + L.diag);
  double* rhs = (double*)(ws + L.rhs);
  double* c = (double*)(ws + L.c);
  double* de = (double*)(ws + L.de);
  CgState* st = (CgState*)(ws + L.st);
  unsigned* ctr = (unsigned*)(ws + L.ctr);
  const int* done = &st->done;
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t x) { if (e == cudaSuccess) e = x; return e == cudaSuccess; };

  // outputs written by sums or accumulated
  if ((long long)o * n > 0) ok(cudaMemsetAsync(A->lp, 0, (size_t)o * n * 8, s));
  if ((long long)v * n > 0) ok(cudaMemsetAsync(A->lpp, 0, (size_t)v * n * 8, s));
  ok(cudaMemsetAsync(A->info, 0, 3 * 8, s));
  ok(cudaMemsetAsync(ctr, 0, (size_t)(2 * max_iter + 8) * 4, s));
  if (ov == 0) return e == cudaSuccess ? RIMP2_OK : RIMP2_ERR_CUDA;
  ok(cudaMemsetAsync(A->dai, 0, (size_t)ov * 8, s));

  const int grid = gemm_f64_occupancy_grid();
  const double* Bf = A->Bf;
  const long long nX = (long long)n * X, oX = (long long)o * X;
  std::vector<GemmProb> lists[kDescLists];
  // 0: Gamma^P[(i,a)][P] = sum_Q Gamma[(i,a)][Q] J^{-1/2}[P][Q]
  if (A->jmh && A->gamma_p)
    lists[0].push_back(gen((int)ov, X, X, 1, A->gamma, X, 1, 0, A->jmh, X, 1, 0, A->gamma_p, X,
                           1.0, false, grid));
  // 1: L'[i][q] = sum_(a,Q) Gamma[i][a][Q] B[q][o+a][Q]; L''[a][q] = sum_(i,Q) Gamma[i][a][Q] B[i][q][Q]
  lists[1].push_back(gen(o, n, X, v, A->gamma, (long long)v * X, 1, X, Bf + oX, nX, 1, X, A->lp, n,
                         1.0, true, grid));
  lists[1].push_back(gen(v, n, X, o, A->gamma, X, 1, (long long)v * X, Bf, X, 1, nX, A->lpp, n,
                         1.0, true, grid));
  // 2: U[i][l][Q] = sum_k D_kl B[i][k][Q];  V[i][c][Q] = sum_b D_bc B[i][o+b][Q]
  for (int i = 0; i < o; ++i) {
    lists[2].push_back(gen(o, X, o, 1, A->pij, o, 1, 0, Bf + (long long)i * nX, 1, X, 0,
                           W + (long long)i * oX, X, 1.0, false, grid));
    lists[2].push_back(gen(v, X, v, 1, A->pab, v, 1, 0, Bf + (long long)i * nX + oX, 1, X, 0,
                           Vv + (long long)i * v * X, X, 1.0, false, grid));
  }
  // 3: rhs[i][a] += sum_(l,Q) B[l][o+a][Q] U[i][l][Q] + sum_(c,Q) B[o+a][o+c][Q] V[i][c][Q]
  lists[3].push_back(gen(o, v, X, o, W, oX, 1, X, Bf + oX, X, 1, nX, rhs, v, 1.0, true, grid));
  lists[3].push_back(gen(o, v, X, v, Vv, (long long)v * X, 1, X, Bf + (long long)o * nX + oX, nX, 1,
                         X, rhs, v, 1.0, true, grid));
  // 4: W[i][j][Q] = sum_b p[j][b] B[i][o+b][Q]
  for (int i = 0; i < o; ++i)
    lists[4].push_back(gen(o, X, v, 1, p, v, 1, 0, Bf + (long long)i * nX + oX, 1, X, 0,
                           W + (long long)i * oX, X, 1.0, false, grid));
  // 5: Ap[i][a] -= sum_(j,Q) B[j][o+a][Q] W[i][j][Q]
  lists[5].push_back(gen(o, v, X, o, W, oX, 1, X, Bf + oX, X, 1, nX, Ap, v, -1.0, true, grid));

  std::vector<char> host(kDescBytes, 0);
  size_t doff[kDescLists];
  long long tiles[kDescLists];
  size_t off = 0;
  for (int k = 0; k < kDescLists; ++k) {
    finish(lists[k], tiles[k]);
    doff[k] = off;
    const size_t bytes = lists[k].size() * sizeof(GemmProb);
    if (off + bytes > kDescBytes) return RIMP2_ERR_UNSUPPORTED;
    if (bytes) memcpy(host.data() + off, lists[k].data(), bytes);
    off = (off + bytes + 255) / 256 * 256;
  }
  char* desc = ws + L.desc;
  ok(cudaMemcpyAsync(desc, host.data(), off, cudaMemcpyHostToDevice, s));
  Bases bs{};
  int next_ctr = 0;
  auto gemm = [&](int k, const int* skip) {
    if (e != cudaSuccess || tiles[k] == 0) return;
    ok(launch_gemm_f64((const GemmProb*)(desc + doff[k]), (int)lists[k].size(), tiles[k], bs,
                       ctr + next_ctr++, grid, s, skip));
  };
  const unsigned row_blocks = (unsigned)((ov + 7) / 8);
  const dim3 col_grid((unsigned)((X + 255) / 256), 1);
  auto colsum = [&](const double* base, long long s1, long long s0, int R1, int R0,
                    const double* w, double* out, const int* skip) {
    const long long R = (long long)R1 * R0;
    if (e != cudaSuccess || X == 0 || R == 0) return;
    const long long per = std::max<long long>(kColRows, (R + 65534) / 65535);
    const dim3 g(col_grid.x, (unsigned)((R + per - 1) / per));
    k_colsum<<<g, 256, 0, s>>>(base, s1, s0, R1, R0, w, X, (int)per, out, skip);
    ok(cudaGetLastError());
  };

  gemm(0, nullptr);
  gemm(1, nullptr);
  // d + e
  ok(cudaMemsetAsync(de, 0, (size_t)X * 8, s));
  colsum(Bf, nX, X, o, o, A->pij, de, nullptr);
  colsum(Bf + (long long)o * nX + oX, nX, X, v, v, A->pab, de, nullptr);
  if (e == cudaSuccess) {
    k_rows<<<row_blocks, 256, 0, s>>>(Bf, A->eps, o, v, X, de, 0, A->lp, A->lpp, rhs, diag,
                                      nullptr, nullptr, nullptr);
    ok(cudaGetLastError());
  }
  gemm(2, nullptr);
  gemm(3, nullptr);
  if (e == cudaSuccess) {
    k_cg_init<<<1, kCgThreads, 0, s>>>(ov, rhs, diag, A->dai, r, z, p, c, X, st, A->info);
    ok(cudaGetLastError());
  }
  for (int it = 0; it < max_iter && e == cudaSuccess; ++it) {
    // Ap = A p
    colsum(Bf + oX, nX, X, o, v, p, c, done);
    if (e == cudaSuccess) {
      k_rows<<<row_blocks, 256, 0, s>>>(Bf, A->eps, o, v, X, c, 1, nullptr, nullptr, nullptr,
                                        nullptr, p, Ap, done);
      ok(cudaGetLastError());
    }
    gemm(4, done);
    gemm(5, done);
    if (e == cudaSuccess) {
      k_cg_step<<<1, kCgThreads, 0, s>>>(ov, diag, A->dai, r, z, p, Ap, c, X, tol, it, st, A->info);
      ok(cudaGetLastError());
    }
  }
  if (e == cudaSuccess) {
    k_cg_finish<<<1, 1, 0, s>>>(st, max_iter, A->info);
    ok(cudaGetLastError());
  }
  return e == cudaSuccess ? RIMP2_OK : RIMP2_ERR_CUDA;
}

}  // extern "C"
