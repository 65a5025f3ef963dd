// MBE3 around the fragment engine (include/rimp2_mbe.h): polymer formation and the
// inclusion-exclusion coefficients on the host, the weighted energy sum on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <vector>

#include "rimp2_mbe.h"

namespace {

double dist(const double* c, int a, int b) {
  const double dx = c[3 * a] - c[3 * b], dy = c[3 * a + 1] - c[3 * b + 1],
               dz = c[3 * a + 2] - c[3 * b + 2];
  return std::sqrt(dx * dx + dy * dy + dz * dz);
}

__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  const double bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// One CTA: fixed-order per-thread TwoSum accumulation, then a TwoSum tree.
__global__ void __launch_bounds__(256)
k_mbe_combine(const double* __restrict__ E, const int* __restrict__ c, long long n, double* out) {
  __shared__ double ss[256], cc[256];
  double s = 0.0, comp = 0.0;
  for (long long f = threadIdx.x; f < n; f += blockDim.x) {
    double t, err;
    const double x = (double)c[f] * E[f];   // |c| is a small integer: exact product
    two_sum(s, x, t, err);
    s = t;
    comp += err;
  }
  ss[threadIdx.x] = s;
  cc[threadIdx.x] = comp;
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
  if (threadIdx.x == 0) *out = ss[0] + cc[0];
}

__global__ void k_mbe_corrections(const double* __restrict__ E, const int* __restrict__ terms,
                                  const int* __restrict__ sign, long long n, int k, double* out,
                                  float* out_log) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  double s = 0.0;
  for (int q = 0; q < k; ++q) s += (double)sign[q] * E[terms[t * k + q]];
  out[t] = s;
  if (out_log) out_log[t] = (float)log10(fabs(s) + 1e-16);
}

}  // namespace

extern "C" int rimp2_mbe_corrections(const double* energy, const int32_t* terms,
                                     const int32_t* sign, int64_t n, int32_t k, double* out,
                                     float* out_log10, void* stream) {
  if (n < 0 || k <= 0 || k > 16 || (n > 0 && (!energy || !terms || !sign || !out)))
    return RIMP2_ERR_BAD_ARG;
  if (n == 0) return RIMP2_OK;
  k_mbe_corrections<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      energy, terms, sign, n, k, out, out_log10);
  return cudaGetLastError() == cudaSuccess ? RIMP2_OK : RIMP2_ERR_CUDA;
}

extern "C" int rimp2_mbe_polymers(const double* c, int32_t n, double r_dimer, double r_trimer,
                                  int32_t rule, int32_t* dimers, int64_t cap_d, int64_t* n_dimers,
                                  int32_t* trimers, int64_t cap_t, int64_t* n_trimers) {
  if (n < 0 || (n > 0 && !c) || !n_dimers || !n_trimers) return RIMP2_ERR_BAD_ARG;
  if ((cap_d > 0 && !dimers) || (cap_t > 0 && !trimers)) return RIMP2_ERR_BAD_ARG;
  if (rule != RIMP2_TRIMER_MAX_PAIR && rule != RIMP2_TRIMER_TWO_PAIRS) return RIMP2_ERR_BAD_ARG;
  std::vector<double> d((size_t)n * n, 0.0);
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) d[(size_t)a * n + b] = dist(c, a, b);
  int64_t nd = 0, nt = 0;
  for (int a = 0; a < n; ++a)
    for (int b = a + 1; b < n; ++b)
      if (d[(size_t)a * n + b] <= r_dimer) {
        if (nd < cap_d) { dimers[2 * nd] = a; dimers[2 * nd + 1] = b; }
        ++nd;
      }
  for (int a = 0; a < n; ++a)
    for (int b = a + 1; b < n; ++b)
      for (int e = b + 1; e < n; ++e) {
        const double dab = d[(size_t)a * n + b], dae = d[(size_t)a * n + e], dbe = d[(size_t)b * n + e];
        bool keep;
        if (rule == RIMP2_TRIMER_MAX_PAIR) keep = std::max(dab, std::max(dae, dbe)) <= r_trimer;
        else keep = (int)(dab <= r_trimer) + (int)(dae <= r_trimer) + (int)(dbe <= r_trimer) >= 2;
        if (keep) {
          if (nt < cap_t) { trimers[3 * nt] = a; trimers[3 * nt + 1] = b; trimers[3 * nt + 2] = e; }
          ++nt;
        }
      }
  *n_dimers = nd;
  *n_trimers = nt;
  return RIMP2_OK;
}

extern "C" int rimp2_mbe_coefficients(int32_t n, const int32_t* dimers, int64_t nd,
                                      const int32_t* trimers, int64_t nt, int32_t* frags,
                                      int32_t* coeff, int64_t cap, int64_t* nfrag) {
  if (n < 0 || nd < 0 || nt < 0 || !nfrag || (nd > 0 && !dimers) || (nt > 0 && !trimers) ||
      (cap > 0 && (!frags || !coeff)))
    return RIMP2_ERR_BAD_ARG;
  using Key = std::array<int, 3>;
  std::map<Key, long long> cf;   // ordered: monomers < pairs < triples by the key layout
  auto add = [&](int a, int b, int e, long long w) {
    Key k;
    if (b < 0) k = {a, -1, -1};
    else if (e < 0) k = {std::min(a, b), std::max(a, b), -1};
    else {
      int v[3] = {a, b, e};
      std::sort(v, v + 3);
      k = {v[0], v[1], v[2]};
    }
    cf[k] += w;
  };
  for (int I = 0; I < n; ++I) add(I, -1, -1, 1);
  for (int64_t q = 0; q < nd; ++q) {
    const int I = dimers[2 * q], J = dimers[2 * q + 1];
    if (I < 0 || J < 0 || I >= n || J >= n || I == J) return RIMP2_ERR_BAD_ARG;
    add(I, J, -1, 1);
    add(I, -1, -1, -1);
    add(J, -1, -1, -1);
  }
  for (int64_t q = 0; q < nt; ++q) {
    const int I = trimers[3 * q], J = trimers[3 * q + 1], K = trimers[3 * q + 2];
    if (I < 0 || J < 0 || K < 0 || I >= n || J >= n || K >= n || I == J || J == K || I == K)
      return RIMP2_ERR_BAD_ARG;
    add(I, J, K, 1);
    add(I, J, -1, -1);
    add(I, K, -1, -1);
    add(J, K, -1, -1);
    add(I, -1, -1, 1);
    add(J, -1, -1, 1);
    add(K, -1, -1, 1);
  }
  // every sub-pair of a kept trimer is needed even when its coefficient cancels to 0
  std::vector<std::pair<Key, long long>> out;
  for (auto& kv : cf) out.push_back(kv);
  std::stable_sort(out.begin(), out.end(), [](const auto& x, const auto& y) {
    const int ox = (x.first[1] >= 0) + (x.first[2] >= 0), oy = (y.first[1] >= 0) + (y.first[2] >= 0);
    if (ox != oy) return ox < oy;
    return x.first < y.first;
  });
  *nfrag = (int64_t)out.size();
  for (int64_t f = 0; f < (int64_t)out.size() && f < cap; ++f) {
    frags[3 * f] = out[f].first[0];
    frags[3 * f + 1] = out[f].first[1];
    frags[3 * f + 2] = out[f].first[2];
    coeff[f] = (int32_t)out[f].second;
  }
  return RIMP2_OK;
}

extern "C" int rimp2_mbe_combine(const double* energy, const int32_t* coeff, int64_t nfrag,
                                 double* out, void* stream) {
  if (nfrag < 0 || !out || (nfrag > 0 && (!energy || !coeff))) return RIMP2_ERR_BAD_ARG;
  k_mbe_combine<<<1, 256, 0, (cudaStream_t)stream>>>(energy, coeff, nfrag, out);
  if (cudaGetLastError() != cudaSuccess) return RIMP2_ERR_CUDA;
  return RIMP2_OK;
}
