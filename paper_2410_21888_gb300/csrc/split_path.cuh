// Split-precision (integer-slice tensor-core) path: plan/wave interface used by the
// host API.  Implemented in split_path.cu.
#pragma once

#include <vector>

#include "rimp2_internal.cuh"

namespace rimp2 {

struct SplitPlan {
  int precision = 0;
  int slices_v = 0, slices_t = 0;
  bool ready = false;
};

struct SplitWave {
  size_t off = 0, bytes = 0;
  std::vector<char> host;  // descriptors copied into the plan's device block
};

int split_plan_init(SplitPlan& sp, int precision, const rimp2_options& opt);
void split_plan_release(SplitPlan& sp);
size_t split_frag_ws_elems(const SplitPlan& sp, const rimp2_frag& f);
int split_build_wave(SplitPlan& sp, const rimp2_frag* frags, const std::vector<int>& members,
                     std::vector<FragDev>& fdev, SplitWave& w, long long& total_pairs,
                     long long& max_b);
size_t split_layout_wave(SplitWave& w, size_t off);
void split_fill_wave(const SplitWave& w, char* host_block);
int split_enqueue_wave(SplitPlan& sp, SplitWave& w, char* dblk, const FragDev* dfd, int nf,
                       long long total_pairs, Bases bs, unsigned* ctr, cudaStream_t s,
                       int* launches, long long* tiles);

}  // namespace rimp2
