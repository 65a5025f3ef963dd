// rimp2_energy_fp64_noalloc: the FP64 energy chain of one fragment (input checks, V GEMM
// with the T = V / D epilogue, pair energies, compensated energy sum) for callers that
// cannot allocate device memory: an allocator that has reserved the whole device, a
// latency-bound loop in which cudaMalloc's implicit synchronisation is not acceptable,
// or a plug-in whose host audits every allocation.  Its scratch is a file-scope device
// array instead of a caller workspace; the compute kernels are the ones
// rimp2_energy_grad launches.  The scratch header (descriptors, queue counter, status
// word) is written by a one-thread kernel whose parameters carry it by value, so no host
// buffer is read after the call returns.
#include <cuda_runtime.h>

#include <mutex>

#include "rimp2_internal.cuh"

using namespace rimp2;

namespace {

// Scratch shared by every call on a device: a header (status word, queue counter and
// the two descriptors), then T[ov][ov] and the pair energies [o][o].
static __device__ __align__(256) unsigned char g_noalloc_scratch[RIMP2_NOALLOC_SCRATCH_BYTES];

constexpr size_t kHeader = 4096;
constexpr size_t kCounterOff = 256;
constexpr size_t kFragOff = 512;
constexpr size_t kProbOff = 1024;
static_assert(sizeof(FragDev) <= kProbOff - kFragOff, "descriptor layout");
static_assert(sizeof(GemmProb) <= kHeader - kProbOff, "descriptor layout");

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};
int g_grid[kMaxDevices] = {};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Writes the header from its by-value parameters: zero status word and queue counter,
// the fragment and the V problem descriptors.
__global__ void k_noalloc_header(unsigned char* scratch, FragDev fd, GemmProb P) {
  if (threadIdx.x == 0) {
    *(unsigned*)scratch = 0u;
    *(unsigned*)(scratch + kCounterOff) = 0u;
    *(FragDev*)(scratch + kFragOff) = fd;
    *(GemmProb*)(scratch + kProbOff) = P;
  }
}

// After the chain: a non-zero status word (a denominator that is not negative, or a
// non-finite input, found by the input check) turns the energy into NaN.
__global__ void k_noalloc_flag(const unsigned* status, double* energy) {
  if (threadIdx.x == 0 && *status != 0u) energy[0] = __longlong_as_double(0x7ff8000000000000ll);
}

// Once per device, with that device current: the device address of the scratch
// array (its host-side name is only a stand-in, never a device pointer).
int setup(int dev, void** ptr, int* grid) {
  if (dev < 0 || dev >= kMaxDevices) return RIMP2_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return RIMP2_ERR_CUDA;
    }
    g_grid[dev] = gemm_f64_occupancy_grid();
    g_scratch_ptr[dev] = p;
  }
  *ptr = g_scratch_ptr[dev];
  *grid = g_grid[dev];
  return RIMP2_OK;
}

}  // namespace

extern "C" int rimp2_energy_fp64_noalloc(int32_t nocc, int32_t nvir, int32_t naux,
                                         const double* B, const double* eps, double* energy,
                                         double* epair, void* stream) {
  if (nocc < 0 || nvir < 0 || naux < 0) return RIMP2_ERR_BAD_ARG;
  if (!energy || ((long long)nocc * nvir * naux > 0 && !B) || (nocc + nvir > 0 && !eps))
    return RIMP2_ERR_BAD_ARG;
  const size_t ov = (size_t)nocc * nvir;
  if (ov > (1u << 20)) return RIMP2_ERR_WORKSPACE;
  const size_t t_bytes = align256(ov * ov * sizeof(double));
  const size_t ep_bytes = align256((size_t)nocc * nocc * sizeof(double));
  if (kHeader + t_bytes + ep_bytes > RIMP2_NOALLOC_SCRATCH_BYTES) return RIMP2_ERR_WORKSPACE;

  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return RIMP2_ERR_CUDA; }
  void* base = nullptr;
  int grid = 0;
  int rc = setup(dev, &base, &grid);
  if (rc != RIMP2_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  char* scratch = (char*)base;

  // descriptors: one fragment, one V problem (element offsets from the bases below)
  FragDev fd{};
  fd.o = nocc; fd.v = nvir; fd.X = naux; fd.idx = 0;
  fd.b_off = 0; fd.eo_off = 0; fd.ev_off = nocc;
  fd.t_off = 0;
  fd.tt_off = -1;             // energy only: the pair energies are formed in registers
  fd.ep_off = (long long)(t_bytes / sizeof(double));
  fd.gamma_off = fd.pij_off = fd.pab_off = -1;
  fd.epair_off = epair ? 0 : -1;
  fd.pair_begin = 0;
  fd.epos_off = -1;
  GemmProb P{};
  long long tiles = 0;
  if (ov > 0) {
    P.kind = PK_V; P.frag = 0;
    P.M = P.N = (int)ov; P.K0 = naux; P.K1 = 1;
    P.tiles_m = P.tiles_n = (int)((ov + F64_BM - 1) / F64_BM);
    P.ksplit = 1; P.k1_chunk = 1;
    P.ntiles = (long long)P.tiles_m * (P.tiles_m + 1) / 2;
    P.tile_begin = 0;
    P.a_off = 0; P.b_off = 0; P.c_off = fd.t_off;
    P.sAm = naux; P.sAk = 1; P.sA1 = 0; P.sBn = naux; P.sBk = 1; P.sB1 = 0;
    P.ldc = (long long)ov; P.alpha = 1.0;
    P.eo_off = 0; P.ev_off = nocc; P.v = nvir; P.b_from_B = 1;
    tiles = P.ntiles;
  }
  k_noalloc_header<<<1, 32, 0, s>>>((unsigned char*)scratch, fd, P);
  cudaError_t e = cudaGetLastError();
  Bases bs{};
  bs.B = B; bs.eps = eps; bs.ws = (double*)(scratch + kHeader);
  bs.epair = epair; bs.energy = energy;
  bs.status = (unsigned*)scratch;
  const FragDev* d_fd = (const FragDev*)(scratch + kFragOff);
  if (e == cudaSuccess)
    e = launch_check_inputs(d_fd, 1, ((long long)ov * naux + 255) / 256, bs, s);
  if (e == cudaSuccess)
    e = launch_gemm_f64((const GemmProb*)(scratch + kProbOff), 1, tiles, bs,
                        (unsigned*)(scratch + kCounterOff), grid, s);
  if (e == cudaSuccess)
    e = launch_amplitude_f64(d_fd, 1, (long long)nocc * (nocc + 1) / 2, bs, s);
  if (e == cudaSuccess) e = launch_energy_reduce(d_fd, 1, bs, s);
  if (e == cudaSuccess) {
    k_noalloc_flag<<<1, 32, 0, s>>>(bs.status, energy);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) { cudaGetLastError(); return RIMP2_ERR_CUDA; }
  return RIMP2_OK;
}
