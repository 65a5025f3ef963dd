// FP64 throughput of this GPU's two FP64 units, measured in place: the CUDA-core DFMA
// pipe and the FP64 tensor path (mma.sync m8n8k4).  They are the denominators of the
// plain FP64 path's roofline.  Register-resident dependent chains, several independent
// per thread or warp, no memory traffic inside the timed loop.
#include <cuda_runtime.h>

#include "rimp2_testing.h"

namespace {

constexpr int kChains = 8;

__global__ void k_dfma_chains(double* out, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// one warp-wide m8n8k4 FP64 MMA: D(8x8) = A(8x4) B(4x8) + C; per thread one element of A
// and of B and two of C / D
__device__ __forceinline__ void dmma(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

__global__ void k_dmma_chains(double* out, int iters, double a, double b) {
  double d[kChains][2];
#pragma unroll
  for (int c = 0; c < kChains; ++c) { d[c][0] = threadIdx.x + c; d[c][1] = c; }
  const double av = a * (1 + (threadIdx.x & 3)), bv = b * (1 + (threadIdx.x >> 3));
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) dmma(d[c][0], d[c][1], av, bv);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += d[c][0] + d[c][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int rimp2_testing_fp64_peak(int32_t kind, double* tflops) {
  if (!tflops || (kind != 0 && kind != 1)) return RIMP2_ERR_BAD_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return RIMP2_ERR_CUDA;
  }
  const int blocks = sms * 8, threads = 256;
  const int iters = kind == 0 ? (1 << 13) : (1 << 11);
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t s = nullptr;
  int rc = RIMP2_OK;
  if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
    rc = RIMP2_ERR_CUDA;
  float best = 0.f;
  for (int rep = 0; rep < 4 && rc == RIMP2_OK; ++rep) {   // the first run warms up
    cudaEventRecord(e0, s);
    if (kind == 0) k_dfma_chains<<<blocks, threads, 0, s>>>(out, iters, 0.999999, 1e-7);
    else k_dmma_chains<<<blocks, threads, 0, s>>>(out, iters, 0.999999, 1e-7);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) { rc = RIMP2_ERR_CUDA; break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (rc == RIMP2_OK && best > 0.f) {
    // DFMA: 2 FLOP per thread and chain step; DMMA: 2 x 8 x 8 x 4 FLOP per warp and MMA
    const double fl = kind == 0 ? 2.0 * kChains * iters * (double)blocks * threads
                                : 512.0 * kChains * iters * (double)blocks * (threads / 32);
    *tflops = fl / (best * 1e-3) / 1e12;
  }
  if (cudaGetLastError() != cudaSuccess && rc == RIMP2_OK) rc = RIMP2_ERR_CUDA;
  if (out) cudaFree(out);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  return rc;
}
