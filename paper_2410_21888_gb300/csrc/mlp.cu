// Learned trimer screen kernels (include/rimp2_mlp.h): features, forward/backward,
// Adam, inference for the 9-64-64-64-1 SiLU network.  One warp per sample; lane l owns
// hidden units l and l + 32 of every layer; activations move between lanes by
// shuffles.  The forward pass uses BF16-rounded weights with FP32 accumulation.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "rimp2_mlp.h"

namespace {

constexpr int IN = RIMP2_MLP_IN, H = RIMP2_MLP_HIDDEN, P = RIMP2_MLP_PARAMS;
constexpr int OW1 = 0, OB1 = OW1 + H * IN, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H,
              OB3 = OW3 + H * H, OW4 = OB3 + H, OB4 = OW4 + H;
static_assert(OB4 + 1 == P, "parameter layout");

__device__ __forceinline__ float bf16_round(float x) {
  return __bfloat162float(__float2bfloat16_rn(x));
}
__device__ __forceinline__ float sigm(float z) { return 1.f / (1.f + expf(-z)); }

struct Act {
  float xs[IN];
  float z1[2], h1[2], z2[2], h2[2], z3[2], h3[2];
  float y;
};

// forward of one sample by one warp; W points to the BF16-rounded parameters in smem
__device__ __forceinline__ void forward(const float* W, const float* x, const float* mean,
                                        const float* stdv, int lane, Act& a) {
#pragma unroll
  for (int i = 0; i < IN; ++i) a.xs[i] = (x[i] - mean[i]) / stdv[i];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int j = lane + 32 * s;
    float z = W[OB1 + j];
#pragma unroll
    for (int i = 0; i < IN; ++i) z = fmaf(W[OW1 + j * IN + i], a.xs[i], z);
    a.z1[s] = z;
    a.h1[s] = z * sigm(z);
  }
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int j = lane + 32 * s;
    a.z2[s] = W[OB2 + j];
  }
  for (int k = 0; k < H; ++k) {
    const float hk = __shfl_sync(0xffffffffu, a.h1[k >> 5], k & 31);
    a.z2[0] = fmaf(W[OW2 + lane * H + k], hk, a.z2[0]);
    a.z2[1] = fmaf(W[OW2 + (lane + 32) * H + k], hk, a.z2[1]);
  }
#pragma unroll
  for (int s = 0; s < 2; ++s) a.h2[s] = a.z2[s] * sigm(a.z2[s]);
#pragma unroll
  for (int s = 0; s < 2; ++s) a.z3[s] = W[OB3 + lane + 32 * s];
  for (int k = 0; k < H; ++k) {
    const float hk = __shfl_sync(0xffffffffu, a.h2[k >> 5], k & 31);
    a.z3[0] = fmaf(W[OW3 + lane * H + k], hk, a.z3[0]);
    a.z3[1] = fmaf(W[OW3 + (lane + 32) * H + k], hk, a.z3[1]);
  }
#pragma unroll
  for (int s = 0; s < 2; ++s) a.h3[s] = a.z3[s] * sigm(a.z3[s]);
  float part = W[OW4 + lane] * a.h3[0] + W[OW4 + lane + 32] * a.h3[1];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
  a.y = part + W[OB4];
}

__device__ __forceinline__ float dsilu(float z) {
  const float s = sigm(z);
  return s * (1.f + z * (1.f - s));
}

__global__ void k_zero(float* p, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = 0.f;
}

__global__ void __launch_bounds__(256)
k_mlp_grad(const float* __restrict__ master, const float* __restrict__ feats,
           const float* __restrict__ y, const int* __restrict__ idx, int n,
           const float* __restrict__ mean, const float* __restrict__ stdv, float* grad,
           float* loss) {
  extern __shared__ float smem_mlp[];   // W[P] then G[P] (72 KB, opt-in)
  float* W = smem_mlp;
  float* G = smem_mlp + P;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    W[i] = bf16_round(master[i]);
    G[i] = 0.f;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  float lsum = 0.f;
  for (int s = warp; s < n; s += nwarps) {
    const int row = idx ? idx[s] : s;
    Act a;
    forward(W, feats + (long long)row * IN, mean, stdv, lane, a);
    const float r = a.y - y[row];
    lsum += r * r;
    const float dy = 2.f * r / (float)n;
    // layer 4
    if (lane == 0) atomicAdd(&G[OB4], dy);
    float dz3[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int j = lane + 32 * q;
      atomicAdd(&G[OW4 + j], dy * a.h3[q]);
      dz3[q] = dy * W[OW4 + j] * dsilu(a.z3[q]);
      atomicAdd(&G[OB3 + j], dz3[q]);
    }
    // layer 3 weights and dh2 = W3^T dz3
    float dh2[2] = {0.f, 0.f};
    for (int k = 0; k < H; ++k) {
      const float h2k = __shfl_sync(0xffffffffu, a.h2[k >> 5], k & 31);
      atomicAdd(&G[OW3 + lane * H + k], dz3[0] * h2k);
      atomicAdd(&G[OW3 + (lane + 32) * H + k], dz3[1] * h2k);
      // contribution of rows lane, lane+32 to column k of W3^T dz3; reduced below
      float c = W[OW3 + lane * H + k] * dz3[0] + W[OW3 + (lane + 32) * H + k] * dz3[1];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
      if ((k & 31) == lane) dh2[k >> 5] = c;
    }
    float dz2[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      dz2[q] = dh2[q] * dsilu(a.z2[q]);
      atomicAdd(&G[OB2 + lane + 32 * q], dz2[q]);
    }
    float dh1[2] = {0.f, 0.f};
    for (int k = 0; k < H; ++k) {
      const float h1k = __shfl_sync(0xffffffffu, a.h1[k >> 5], k & 31);
      atomicAdd(&G[OW2 + lane * H + k], dz2[0] * h1k);
      atomicAdd(&G[OW2 + (lane + 32) * H + k], dz2[1] * h1k);
      float c = W[OW2 + lane * H + k] * dz2[0] + W[OW2 + (lane + 32) * H + k] * dz2[1];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
      if ((k & 31) == lane) dh1[k >> 5] = c;
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int j = lane + 32 * q;
      const float dz1 = dh1[q] * dsilu(a.z1[q]);
      atomicAdd(&G[OB1 + j], dz1);
#pragma unroll
      for (int i = 0; i < IN; ++i) atomicAdd(&G[OW1 + j * IN + i], dz1 * a.xs[i]);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < P; i += blockDim.x)
    if (G[i] != 0.f) atomicAdd(&grad[i], G[i]);
  if (loss && lane == 0) atomicAdd(loss, lsum / (float)n);
}

__global__ void k_mlp_adam(float* w, const float* g, float* m, float* v, float c1, float c2,
                           float lr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

__global__ void __launch_bounds__(256)
k_mlp_predict(const float* __restrict__ master, const float* __restrict__ feats, long long n,
              const float* __restrict__ mean, const float* __restrict__ stdv,
              float* __restrict__ out) {
  __shared__ float W[P];
  for (int i = threadIdx.x; i < P; i += blockDim.x) W[i] = bf16_round(master[i]);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long warp = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long s = warp; s < n; s += nwarps) {
    Act a;
    forward(W, feats + s * IN, mean, stdv, lane, a);
    if (lane == 0) out[s] = a.y;
  }
}

__device__ __forceinline__ void sort3(float& a, float& b, float& c) {
  float t;
  if (a > b) { t = a; a = b; b = t; }
  if (b > c) { t = b; b = c; c = t; }
  if (a > b) { t = a; a = b; b = t; }
}

__global__ void k_screen_features(const double* __restrict__ cen, const int* __restrict__ nocc,
                                  int n, const int* __restrict__ tri, long long nt,
                                  const double* __restrict__ dde, float* __restrict__ f) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const int I = tri[3 * t], J = tri[3 * t + 1], K = tri[3 * t + 2];
  auto d = [&](int a, int b) {
    const double dx = cen[3 * a] - cen[3 * b], dy = cen[3 * a + 1] - cen[3 * b + 1],
                 dz = cen[3 * a + 2] - cen[3 * b + 2];
    return (float)sqrt(dx * dx + dy * dy + dz * dz);
  };
  float d0 = d(I, J), d1 = d(I, K), d2 = d(J, K);
  sort3(d0, d1, d2);
  float n0 = (float)nocc[I], n1 = (float)nocc[J], n2 = (float)nocc[K];
  sort3(n0, n1, n2);
  float e0 = (float)log10(fabs(dde[(long long)I * n + J]) + 1e-16);
  float e1 = (float)log10(fabs(dde[(long long)I * n + K]) + 1e-16);
  float e2 = (float)log10(fabs(dde[(long long)J * n + K]) + 1e-16);
  sort3(e0, e1, e2);
  float* o = f + t * IN;
  o[0] = d0; o[1] = d1; o[2] = d2;
  o[3] = n0; o[4] = n1; o[5] = n2;
  o[6] = e0; o[7] = e1; o[8] = e2;
}

int check(cudaError_t e) {
  if (e != cudaSuccess) { cudaGetLastError(); return RIMP2_ERR_CUDA; }
  return RIMP2_OK;
}

}  // namespace

extern "C" int rimp2_screen_features(const double* centroids, const int32_t* nocc, int32_t n,
                                     const int32_t* trimers, int64_t nt, const double* dimer_de,
                                     float* feats, void* stream) {
  if (n < 0 || nt < 0 || (nt > 0 && (!centroids || !nocc || !trimers || !dimer_de || !feats)))
    return RIMP2_ERR_BAD_ARG;
  if (nt == 0) return RIMP2_OK;
  k_screen_features<<<(unsigned)((nt + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      centroids, nocc, n, trimers, nt, dimer_de, feats);
  return check(cudaGetLastError());
}

extern "C" int rimp2_mlp_grad(const float* master, const float* feats, const float* y,
                              const int32_t* idx, int32_t n, const float* mean, const float* stdv,
                              float* grad, float* loss, void* stream) {
  if (n <= 0 || !master || !feats || !y || !mean || !stdv || !grad) return RIMP2_ERR_BAD_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  k_zero<<<(P + 255) / 256, 256, 0, s>>>(grad, P);
  if (loss) k_zero<<<1, 32, 0, s>>>(loss, 1);
  int blocks = (n + 63) / 64;
  if (blocks > 64) blocks = 64;
  const int smem = 2 * P * (int)sizeof(float);
  if (cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
      cudaSuccess)
    return check(cudaGetLastError());
  k_mlp_grad<<<blocks, 256, smem, s>>>(master, feats, y, idx, n, mean, stdv, grad, loss);
  return check(cudaGetLastError());
}

extern "C" int rimp2_mlp_adam(float* master, const float* grad, float* m, float* v, int32_t t,
                              float lr, void* stream) {
  if (!master || !grad || !m || !v || t < 1) return RIMP2_ERR_BAD_ARG;
  const float c1 = 1.f - powf(0.9f, (float)t), c2 = 1.f - powf(0.999f, (float)t);
  k_mlp_adam<<<(P + 255) / 256, 256, 0, (cudaStream_t)stream>>>(master, grad, m, v, c1, c2, lr);
  return check(cudaGetLastError());
}

extern "C" int rimp2_mlp_predict(const float* master, const float* feats, int64_t n,
                                 const float* mean, const float* stdv, float* out, void* stream) {
  if (n < 0 || (n > 0 && (!master || !feats || !mean || !stdv || !out))) return RIMP2_ERR_BAD_ARG;
  if (n == 0) return RIMP2_OK;
  long long blocks = (n + 7) / 8;
  if (blocks > 4096) blocks = 4096;
  k_mlp_predict<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(master, feats, n, mean, stdv, out);
  return check(cudaGetLastError());
}
