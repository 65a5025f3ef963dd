// FP64 kernels of the RI-MP2 hot path: grouped persistent DFMA GEMM for the four
// contractions (Eq. MP2_ints for V; Appendix Gamma, D^MP2_ab, D^MP2_ij), the amplitude
// pass (T -> Tt = 2T - T^T and the pair energies), the compensated energy reduction,
// and input checks.  CUDA-core FP64 on sm_103a: the GEMM keeps a 64x64 tile per CTA
// with a 4x4 register block per thread; work tiles come from a device queue (an
// atomic counter) in the order the host sorted them (largest K first).
#include <math.h>

#include "rimp2_internal.cuh"

namespace rimp2 {

__device__ __forceinline__ int find_prob(const GemmProb* __restrict__ probs, int nprobs,
                                         long long t) {
  int lo = 0, hi = nprobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (probs[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Upper-triangle enumeration, column by column: t -> (r, c) with r <= c.
__device__ __forceinline__ void tri_index(long long t, int& r, int& c) {
  long long cc = (long long)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while (cc * (cc + 1) / 2 > t) --cc;
  while ((cc + 1) * (cc + 2) / 2 <= t) ++cc;
  c = (int)cc;
  r = (int)(t - cc * (cc + 1) / 2);
}

template <typename F>
__device__ __forceinline__ int find_frag(const FragDev* __restrict__ frags, int nfrag,
                                         long long t, F key) {
  int lo = 0, hi = nfrag - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (key(frags[mid]) <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ------------------------------------------------------------------ grouped GEMM

__global__ void __launch_bounds__(256, 2)
k_gemm_f64(const GemmProb* __restrict__ probs, int nprobs, long long total, Bases bs,
           unsigned* __restrict__ counter, const int* __restrict__ skip) {
  __shared__ double As[F64_BK][F64_BM + 1];
  __shared__ double Bs[F64_BK][F64_BN + 1];
  __shared__ long long s_tile;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  if (skip && *(volatile const int*)skip) return;

  for (;;) {
    if (tid == 0) s_tile = (long long)atomicAdd(counter, 1u);
    __syncthreads();
    const long long t = s_tile;
    if (t >= total) break;
    const GemmProb P = probs[find_prob(probs, nprobs, t)];
    const long long lt = t - P.tile_begin;
    const int ks = (int)(lt % P.ksplit);
    const long long tt = lt / P.ksplit;
    int tm, tn;
    if (P.kind == PK_V) tri_index(tt, tm, tn);
    else { tm = (int)(tt / P.tiles_n); tn = (int)(tt % P.tiles_n); }
    const int m0 = tm * F64_BM, n0 = tn * F64_BN;
    const double* __restrict__ A =
        P.kind == PK_GEN ? P.pa : (P.kind == PK_V ? bs.B : bs.ws) + P.a_off;
    const double* __restrict__ Bo = P.kind == PK_GEN ? P.pb : (P.b_from_B ? bs.B : bs.ws) + P.b_off;
    const bool a_kc = (P.sAk == 1), b_kc = (P.sBk == 1);

    double acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;

    const int k1b = ks * P.k1_chunk;
    const int k1e = min(P.K1, k1b + P.k1_chunk);
    for (int k1 = k1b; k1 < k1e; ++k1) {
      for (int k0 = 0; k0 < P.K0; k0 += F64_BK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int e = tid + 256 * q;
          int mm, kk;
          if (a_kc) { kk = e & 15; mm = e >> 4; } else { mm = e & 63; kk = e >> 6; }
          const int gm = m0 + mm, gk = k0 + kk;
          double val = 0.0;
          if (gm < P.M && gk < P.K0)
            val = A[(long long)gm * P.sAm + (long long)gk * P.sAk + (long long)k1 * P.sA1];
          As[kk][mm] = val;
          int nn, kb;
          if (b_kc) { kb = e & 15; nn = e >> 4; } else { nn = e & 63; kb = e >> 6; }
          const int gn = n0 + nn, gkb = k0 + kb;
          double vb = 0.0;
          if (gn < P.N && gkb < P.K0)
            vb = Bo[(long long)gn * P.sBn + (long long)gkb * P.sBk + (long long)k1 * P.sB1];
          Bs[kb][nn] = vb;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < F64_BK; ++kk) {
          double a[4], b[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
          for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
      }
    }

    // epilogue
    if (P.kind == PK_V) {
      double* __restrict__ C = bs.ws + P.c_off;
      const double* eo = bs.eps + P.eo_off;
      const double* ev = bs.eps + P.ev_off;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int m = m0 + ty + 16 * r;
        if (m >= P.M) continue;
        const int i = m / P.v, a = m - i * P.v;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int n = n0 + tx + 16 * c;
          if (n >= P.N) continue;
          const int j = n / P.v, b = n - j * P.v;
          const double D = eo[i] + eo[j] - ev[a] - ev[b];
          const double T = acc[r][c] / D;
          C[(long long)m * P.ldc + n] = T;
          if (tm != tn) C[(long long)n * P.ldc + m] = T;
        }
      }
    } else {
      double* __restrict__ C =
          P.kind == PK_GEN ? P.pc
                           : (P.kind == PK_GAMMA ? bs.gamma : P.kind == PK_PAB ? bs.pab : bs.pij) +
                                 P.c_off;
      const bool store = P.ksplit == 1 && (P.kind == PK_GAMMA || (P.kind == PK_GEN && !P.accumulate));
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int m = m0 + ty + 16 * r;
        if (m >= P.M) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int n = n0 + tx + 16 * c;
          if (n >= P.N) continue;
          const double val = P.alpha * acc[r][c];
          if (store) C[(long long)m * P.ldc + n] = val;
          else atomicAdd(C + (long long)m * P.ldc + n, val);
        }
      }
    }
    __syncthreads();  // s_tile is rewritten at the top of the next iteration
  }
}

int gemm_f64_occupancy_grid() {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_gemm_f64, 256, 0);
  if (per < 1) per = 1;
  return sms * per;
}

cudaError_t launch_gemm_f64(const GemmProb* d_probs, int nprobs, long long total_tiles,
                            Bases bs, unsigned* counter, int grid, cudaStream_t s,
                            const int* skip) {
  if (total_tiles <= 0) return cudaSuccess;
  const long long g = total_tiles < grid ? total_tiles : grid;
  k_gemm_f64<<<(unsigned)g, 256, 0, s>>>(d_probs, nprobs, total_tiles, bs, counter, skip);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ amplitudes

// One CTA per pair block (i <= j) of one fragment.  Reads T_ij and writes
// Tt_ij = 2 T_ij - T_ij^T for the (i,j) block and, if i != j, Tt_ji = Tt_ij^T for the
// (j,i) block.  Pair energy e_ij = sum_ab Tt_ij(a,b) V_ij(a,b) with V = T * D, and its
// opposite-spin part sum_ab T_ij(a,b) V_ij(a,b).
__global__ void __launch_bounds__(256)
k_amplitude_f64(const FragDev* __restrict__ frags, int nfrag, Bases bs) {
  __shared__ double X[32][33];
  __shared__ double Y[32][33];
  __shared__ double red[8], red_os[8];
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const long long gp = blockIdx.x;
  const int f = find_frag(frags, nfrag, gp, [](const FragDev& F) { return F.pair_begin; });
  const FragDev F = frags[f];
  int i, j;
  tri_index(gp - F.pair_begin, i, j);
  const int v = F.v, o = F.o;
  const long long ov = (long long)o * v;
  const double* __restrict__ T = bs.ws + F.t_off;
  double* __restrict__ Tt = bs.ws + (F.tt_off >= 0 ? F.tt_off : 0);   // unused if < 0
  const double* eo = bs.eps + F.eo_off;
  const double* ev = bs.eps + F.ev_off;
  const double eij = eo[i] + eo[j];
  const long long rowI = (long long)i * v, rowJ = (long long)j * v;
  double e_part = 0.0, e_os = 0.0;
  const int nt = (v + 31) / 32;
  const long long npairs = (long long)nt * (nt + 1) / 2;

  for (long long q = 0; q < npairs; ++q) {
    int ta, tb;
    tri_index(q, ta, tb);
    // X = T_ij[ta-rows][tb-cols], Y = T_ij[tb-rows][ta-cols]
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int l = ty + 8 * r;
      const int a = ta * 32 + l, b = tb * 32 + tx;
      X[l][tx] = (a < v && b < v) ? T[(rowI + a) * ov + rowJ + b] : 0.0;
      const int a2 = tb * 32 + l, b2 = ta * 32 + tx;
      Y[l][tx] = (a2 < v && b2 < v) ? T[(rowI + a2) * ov + rowJ + b2] : 0.0;
    }
    __syncthreads();
    // tile (ta, tb) of the (i,j) block: Tt(a,b) = 2 X[a][b] - Y[b][a]
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int l = ty + 8 * r;
      const int a = ta * 32 + l, b = tb * 32 + tx;
      if (a < v && b < v) {
        const double t = X[l][tx];
        const double tt = 2.0 * t - Y[tx][l];
        if (F.tt_off >= 0) Tt[(rowI + a) * ov + rowJ + b] = tt;
        const double D = eij - ev[a] - ev[b];
        e_part += tt * (t * D);
        e_os += t * (t * D);
      }
      if (ta != tb) {  // tile (tb, ta): Tt(a,b) = 2 Y[a][b] - X[b][a]
        const int a2 = tb * 32 + l, b2 = ta * 32 + tx;
        if (a2 < v && b2 < v) {
          const double t = Y[l][tx];
          const double tt = 2.0 * t - X[tx][l];
          if (F.tt_off >= 0) Tt[(rowI + a2) * ov + rowJ + b2] = tt;
          const double D = eij - ev[a2] - ev[b2];
          e_part += tt * (t * D);
          e_os += t * (t * D);
        }
      }
    }
    if (i != j && F.tt_off >= 0) {
      // (j,i) block: Tt_ji(a',b') = Tt_ij(b',a'); rows a' from tb, cols b' from ta
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int l = ty + 8 * r;
        const int ap = tb * 32 + l, bp = ta * 32 + tx;   // Tt_ij(bp, ap), bp in ta, ap in tb
        if (ap < v && bp < v)
          Tt[(rowJ + ap) * ov + rowI + bp] = 2.0 * X[tx][l] - Y[l][tx];
        if (ta != tb) {
          const int ap2 = ta * 32 + l, bp2 = tb * 32 + tx;  // Tt_ij(bp2, ap2), bp2 in tb
          if (ap2 < v && bp2 < v)
            Tt[(rowJ + ap2) * ov + rowI + bp2] = 2.0 * Y[tx][l] - X[l][tx];
        }
      }
    }
    __syncthreads();
  }
  // block reduction of the pair energy
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    e_part += __shfl_down_sync(0xffffffffu, e_part, off);
    e_os += __shfl_down_sync(0xffffffffu, e_os, off);
  }
  if (tx == 0) { red[ty] = e_part; red_os[ty] = e_os; }
  __syncthreads();
  if (tid == 0) {
    double e = 0.0, eos = 0.0;
    for (int w = 0; w < 8; ++w) { e += red[w]; eos += red_os[w]; }
    double* ep = bs.ws + F.ep_off;
    ep[(long long)i * o + j] = e;
    ep[(long long)j * o + i] = e;
    if (F.epos_off >= 0) {
      double* eq = bs.ws + F.epos_off;
      eq[(long long)i * o + j] = eos;
      eq[(long long)j * o + i] = eos;
    }
  }
}

cudaError_t launch_amplitude_f64(const FragDev* d_frags, int nfrag, long long total_pairs,
                                 Bases bs, cudaStream_t s) {
  if (total_pairs <= 0) return cudaSuccess;
  k_amplitude_f64<<<(unsigned)total_pairs, 256, 0, s>>>(d_frags, nfrag, bs);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ energy reduction

__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  const double bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// One CTA per fragment: E = sum_ij e_pair[i][j] with compensated (TwoSum) sums in a
// fixed order; copies e_pair to the caller's buffer when requested.
__global__ void __launch_bounds__(256)
k_energy_reduce(const FragDev* __restrict__ frags, Bases bs) {
  __shared__ double ss[256], cc[256];
  const FragDev F = frags[blockIdx.x];
  const long long n = (long long)F.o * F.o;
  // compensated (TwoSum) sum of x[0..n): per-thread running sums, then a tree
  auto csum = [&](const double* x, double* copy_to) -> double {
    double s = 0.0, c = 0.0;
    for (long long e = threadIdx.x; e < n; e += blockDim.x) {
      const double y = x[e];
      double t, err;
      two_sum(s, y, t, err);
      s = t;
      c += err;
      if (copy_to) copy_to[e] = y;
    }
    ss[threadIdx.x] = s;
    cc[threadIdx.x] = c;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) {
        double t, err;
        two_sum(ss[threadIdx.x], ss[threadIdx.x + w], t, err);
        ss[threadIdx.x] = t;
        cc[threadIdx.x] += cc[threadIdx.x + w] + err;
      }
      __syncthreads();
    }
    const double r = ss[0] + cc[0];
    __syncthreads();   // ss / cc are reused by the next sum
    return r;
  };
  const double e = csum(bs.ws + F.ep_off, F.epair_off >= 0 ? bs.epair + F.epair_off : nullptr);
  if (threadIdx.x == 0) bs.energy[F.idx] = e;
  if ((bs.energy_os || bs.energy_scs) && F.epos_off >= 0) {
    const double eos = csum(bs.ws + F.epos_off, nullptr);
    if (threadIdx.x == 0) {
      if (bs.energy_os) bs.energy_os[F.idx] = eos;
      // spin-component scaling: c_os E_OS + c_ss E_SS with E_SS = E - E_OS
      if (bs.energy_scs) bs.energy_scs[F.idx] = bs.scs_os * eos + bs.scs_ss * (e - eos);
    }
  }
}

cudaError_t launch_energy_reduce(const FragDev* d_frags, int nfrag, Bases bs, cudaStream_t s) {
  if (nfrag <= 0) return cudaSuccess;
  k_energy_reduce<<<nfrag, 256, 0, s>>>(d_frags, bs);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ zero P outputs

__global__ void k_zero_p(const FragDev* __restrict__ frags, Bases bs) {
  const FragDev F = frags[blockIdx.y];
  const long long no = (long long)F.o * F.o, nv = (long long)F.v * F.v;
  const long long ng = (F.zero_gamma && F.gamma_off >= 0) ? (long long)F.o * F.v * F.X : 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < no + nv + ng;
       e += stride) {
    if (e < no) { if (F.pij_off >= 0) bs.pij[F.pij_off + e] = 0.0; }
    else if (e < no + nv) { if (F.pab_off >= 0) bs.pab[F.pab_off + (e - no)] = 0.0; }
    else bs.gamma[F.gamma_off + (e - no - nv)] = 0.0;
  }
}

cudaError_t launch_zero_p(const FragDev* d_frags, int nfrag, Bases bs, cudaStream_t s) {
  if (nfrag <= 0) return cudaSuccess;
  k_zero_p<<<dim3(256, nfrag), 256, 0, s>>>(d_frags, bs);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ input checks

// Denominators must be negative for every (i,j,a,b): max(eps_occ) < min(eps_vir).
// B and eps must be finite.  Violations set bits of the status word.
__global__ void k_check_inputs(const FragDev* __restrict__ frags, Bases bs) {
  const FragDev F = frags[blockIdx.y];
  bool bad_nf = false;
  const long long nb = (long long)F.o * F.v * F.X;
  const double* B = bs.B + F.b_off;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nb; e += stride)
    bad_nf |= !finite_bits(B[e]);
  if (blockIdx.x == 0) {
    __shared__ double smax[256], smin[256];
    double mx = -INFINITY, mn = INFINITY;
    for (int e = threadIdx.x; e < F.o; e += blockDim.x) {
      const double x = bs.eps[F.eo_off + e];
      bad_nf |= !isfinite(x);
      mx = fmax(mx, x);
    }
    for (int e = threadIdx.x; e < F.v; e += blockDim.x) {
      const double x = bs.eps[F.ev_off + e];
      bad_nf |= !isfinite(x);
      mn = fmin(mn, x);
    }
    smax[threadIdx.x] = mx;
    smin[threadIdx.x] = mn;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) {
        smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + w]);
        smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + w]);
      }
      __syncthreads();
    }
    if (threadIdx.x == 0 && F.o > 0 && F.v > 0 && !(smax[0] < smin[0]))
      atomicOr(bs.status, ST_DENOM);
  }
  if (bad_nf) atomicOr(bs.status, ST_NONFINITE);
}

cudaError_t launch_check_inputs(const FragDev* d_frags, int nfrag, long long max_bx, Bases bs,
                                cudaStream_t s) {
  if (nfrag <= 0) return cudaSuccess;
  const unsigned bx = (unsigned)(max_bx < 1 ? 1 : (max_bx > 256 ? 256 : max_bx));
  k_check_inputs<<<dim3(bx, nfrag), 256, 0, s>>>(d_frags, bs);
  return cudaGetLastError();
}

}  // namespace rimp2
