// Split-precision path (placeholder until the tensor-core kernels land).
#include <cstring>

#include "split_path.cuh"

namespace rimp2 {

int split_plan_init(SplitPlan& sp, int precision, const rimp2_options& opt) {
  sp.precision = precision;
  sp.slices_v = opt.slices_v;
  sp.slices_t = opt.slices_t;
  return RIMP2_ERR_UNSUPPORTED;
}
void split_plan_release(SplitPlan&) {}
size_t split_frag_ws_elems(const SplitPlan&, const rimp2_frag&) { return 0; }
int split_build_wave(SplitPlan&, const rimp2_frag*, const std::vector<int>&,
                     std::vector<FragDev>&, SplitWave&, long long&, long long&) {
  return RIMP2_ERR_UNSUPPORTED;
}
size_t split_layout_wave(SplitWave& w, size_t off) { w.off = off; return off + w.bytes; }
void split_fill_wave(const SplitWave& w, char* host_block) {
  if (w.bytes) memcpy(host_block + w.off, w.host.data(), w.bytes);
}
int split_enqueue_wave(SplitPlan&, SplitWave&, char*, const FragDev*, int, long long, Bases,
                       unsigned*, cudaStream_t, int*, long long*) {
  return RIMP2_ERR_UNSUPPORTED;
}

}  // namespace rimp2
