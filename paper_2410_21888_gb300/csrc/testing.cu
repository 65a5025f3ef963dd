// Test hooks (include/rimp2_testing.h): the split GEMM kernel on raw digit planes.
#include <cuda_runtime.h>

#include <cstring>

#include "rimp2_testing.h"
#include "split_gemm.cuh"

using namespace rimp2;

extern "C" int rimp2_testing_set_wait_limit(int64_t ns) {
  if (split_gemm_set_consumer_wait((long long)ns) != cudaSuccess) {
    cudaGetLastError();
    return RIMP2_ERR_CUDA;
  }
  return RIMP2_OK;
}

extern "C" int rimp2_testing_slice_gemm(int32_t M, int32_t N, int32_t K, int32_t kpad,
                                        int32_t slices, const void* A, const void* B, double* C,
                                        void* stream) {
  return rimp2_testing_slice_gemm_k(M, N, K, kpad, slices, 32, 0, A, B, C, stream);
}

extern "C" int rimp2_testing_slice_gemm_k(int32_t M, int32_t N, int32_t K, int32_t kpad,
                                          int32_t slices, int32_t stage_k, int32_t fp8,
                                          const void* A, const void* B, double* C,
                                          void* stream) {
  if (M <= 0 || N <= 0 || K < 0 || kpad < K || kpad % (fp8 ? 16 : 8) != 0 || slices < 2 ||
      slices > (fp8 ? 16 : 8) || !A || !B || !C)
    return RIMP2_ERR_BAD_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (!fp8 && stage_k != 16 && stage_k != 32) return RIMP2_ERR_BAD_ARG;
  const SplitLaunch cfg = split_launch_config(slices, stage_k, 0, fp8 != 0);
  const int E8 = fp8 ? SG_LB_FP8 : SG_LB_BF16;   // EA = EB = bits per digit: product scale 2^0
  const int esz = fp8 ? 1 : 2;
  if (split_gemm_prepare() != cudaSuccess) { cudaGetLastError(); return RIMP2_ERR_CUDA; }
  SplitProb P;
  memset(&P, 0, sizeof(P));
  P.kind = PK_RAW;
  P.M = M; P.N = N; P.n_tile = cfg.n_tile_max;
  P.tiles_m = (M + SG_BM - 1) / SG_BM;
  P.tiles_n = (N + cfg.n_tile_max - 1) / cfg.n_tile_max;
  P.ksplit = 1; P.k0_blocks = (K + cfg.bk - 1) / cfg.bk; P.k1_count = 1; P.k1_chunk = 1;
  P.a_mode = P.b_mode = TM_3D; P.div5 = 1;
  P.ea_rows = P.eb_rows = 0;
  P.ea_off = sizeof(SplitProb); P.eb_off = sizeof(SplitProb);   // int 8 stored there
  P.c_off = 0; P.ldc = N; P.alpha = 1.0;
  P.ntiles = (long long)P.tiles_m * P.tiles_n;
  const uint64_t dA[3] = {(uint64_t)(K > 0 ? K : 1), (uint64_t)M, (uint64_t)slices};
  const uint64_t sA[2] = {(uint64_t)kpad * esz, (uint64_t)M * kpad * esz};
  const uint64_t dB[3] = {(uint64_t)(K > 0 ? K : 1), (uint64_t)N, (uint64_t)slices};
  const uint64_t sB[2] = {(uint64_t)kpad * esz, (uint64_t)N * kpad * esz};
  const uint32_t boxA[3] = {(uint32_t)cfg.bk, SG_BM, (uint32_t)slices}, boxB[3] = {(uint32_t)cfg.bk, (uint32_t)cfg.n_tile_max, (uint32_t)slices};
  if (encode_tmap(&P.tmA, A, 3, dA, sA, boxA, esz) != RIMP2_OK ||
      encode_tmap(&P.tmB, B, 3, dB, sB, boxB, esz) != RIMP2_OK)
    return RIMP2_ERR_UNSUPPORTED;
  const size_t bytes = sizeof(SplitProb) + 256;
  char* buf = nullptr;
  if (cudaMalloc(&buf, bytes) != cudaSuccess) { cudaGetLastError(); return RIMP2_ERR_NOMEM; }
  char host[sizeof(SplitProb) + 256];
  memset(host, 0, sizeof(host));
  memcpy(host, &P, sizeof(P));
  memcpy(host + sizeof(SplitProb), &E8, sizeof(int));   // EA + EB - 2 bits = 0
  int rc = RIMP2_OK;
  unsigned* counter = (unsigned*)(buf + sizeof(SplitProb) + 64);
  unsigned* status = (unsigned*)(buf + sizeof(SplitProb) + 128);
  if (cudaMemcpy(buf, host, bytes, cudaMemcpyHostToDevice) != cudaSuccess) rc = RIMP2_ERR_CUDA;
  if (rc == RIMP2_OK) {
    Bases bs{};
    bs.ws = (double*)buf;
    bs.gamma = C;
    bs.status = status;
    if (launch_split_gemm((const SplitProb*)buf, nullptr, 1, P.ntiles, bs, counter, cfg, split_gemm_grid(), s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      rc = RIMP2_ERR_CUDA;
  }
  if (rc == RIMP2_OK) {
    unsigned st = 0;
    if (cudaMemcpy(&st, status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) rc = RIMP2_ERR_CUDA;
    else if (st & ST_TIMEOUT) rc = RIMP2_ERR_TIMEOUT;
  }
  cudaGetLastError();
  cudaFree(buf);
  return rc;
}
