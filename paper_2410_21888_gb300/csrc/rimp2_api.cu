// Host side of librimp2: the C ABI declared in include/rimp2.h.
//
// A plan holds the fragment shapes, splits the batch into waves that share one
// workspace, and builds per-wave problem descriptors for the grouped kernels (element
// offsets only; base pointers are kernel arguments).  The launch sequence of a call is
// captured once into a CUDA graph on a private stream and replayed on the caller's
// stream; a change of pointers or offsets rebuilds descriptors and graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <string>
#include <cstring>
#include <new>
#include <vector>

#include "rimp2_internal.cuh"
#include "split_path.cuh"

using namespace rimp2;

namespace {

constexpr size_t kAlignElems = 32;  // 256-byte alignment of workspace regions
constexpr int kEv = 6;               // stage events per wave

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct WaveDesc {
  std::vector<int> frags;             // batch indices in this wave
  std::vector<FragDev> fdev;
  std::vector<GemmProb> probs_v;      // stage 1: V (+ T epilogue)
  std::vector<GemmProb> probs_c;      // stage 2: Gamma, P_ab, P_ij
  long long tiles_v = 0, tiles_c = 0, total_pairs = 0, max_b = 0;
  size_t off_fdev = 0, off_pv = 0, off_pc = 0;  // byte offsets into the plan device block
  SplitWave split;                    // split-path descriptors (split_path.cu)
};

struct Key {
  const void* p[10];
  std::vector<rimp2_frag> frags;
  bool operator==(const Key& o) const {
    if (memcmp(p, o.p, sizeof(p)) != 0 || frags.size() != o.frags.size()) return false;
    return memcmp(frags.data(), o.frags.data(), frags.size() * sizeof(rimp2_frag)) == 0;
  }
};

}  // namespace

struct rimp2_plan {
  int device = 0;
  int precision = RIMP2_FP64;
  rimp2_options opt{};
  std::vector<rimp2_frag> frags;
  std::vector<std::vector<int>> wave_members;
  size_t ws_bytes = 0;
  int gemm_grid = 0;
  // device block
  char* dblk = nullptr;
  size_t dblk_bytes = 0;
  unsigned* d_status = nullptr;
  unsigned* d_counters = nullptr;
  std::vector<WaveDesc> waves;
  bool have_desc = false;
  Key key{};
  // graph
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaEvent_t done = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  bool timing_pending = false;
  rimp2_stats stats{};
  SplitPlan split;
  std::vector<cudaEvent_t> stage_ev;   // kEv per wave when profile_stages (or autotune)
  // autotune: 0 off, 1 trials running, 2 done.  A trial is one call with one tile shape
  // per launch (an index into the split plan's candidate lists; kBestShapes: the fastest
  // found so far, per launch) and one contraction-stage variant.
  int tune_state = 0;
  int tune_next = 0;
  int tune_cur = -1;                   // trial whose times are pending
  int variant = 0;                     // contraction-stage variant in use
  struct Trial { int shape, variant; };
  std::vector<Trial> trials;
  std::vector<double> tr_v, tr_p, tr_g, tr_c;   // per trial: V, P launch, Gamma launch, stage 3
  uint64_t tune_key = 0;
  std::string cache_path;
};

extern "C" {

const char* rimp2_version(void) { return "rimp2 0.1 sm_103a"; }

const char* rimp2_status_string(int s) {
  switch (s) {
    case RIMP2_OK: return "ok";
    case RIMP2_ERR_BAD_ARG: return "bad argument";
    case RIMP2_ERR_SHAPE: return "batch shapes differ from the plan";
    case RIMP2_ERR_DENOM: return "non-negative orbital-energy denominator (e_a <= e_i)";
    case RIMP2_ERR_NONFINITE: return "non-finite input";
    case RIMP2_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case RIMP2_ERR_CUDA: return "CUDA runtime error";
    case RIMP2_ERR_TIMEOUT: return "bounded device wait expired";
    case RIMP2_ERR_UNSUPPORTED: return "unsupported option or size";
    case RIMP2_ERR_NOMEM: return "allocation failed";
    default: return "unknown status";
  }
}

void rimp2_default_options(rimp2_options* opt) {
  if (!opt) return;
  memset(opt, 0, sizeof(*opt));
  opt->slices_v = 0;   // 0: the precision's default (BF16 V 5, P 6, Gamma 5; FP8 8, 10, 10)
  opt->slices_t = 0;
  opt->slices_g = 0;
  opt->use_graph = 1;
  opt->check_inputs = 1;
  opt->autotune = 0;
  opt->max_workspace_bytes = 0;
  opt->scs_os = 6.0 / 5.0;   // SCS-MP2 weights (Grimme)
  opt->scs_ss = 1.0 / 3.0;
}

}  // extern "C"

namespace {

bool wants_tt(const rimp2_frag& f) { return f.gamma_off >= 0 || f.pij_off >= 0 || f.pab_off >= 0; }

// Workspace of one fragment on the FP64 path; build_fp64_wave lays out exactly this:
// T, Tt (when an output needs it), pair energies and their opposite-spin part.
size_t frag_ws_elems_fp64(const rimp2_frag& f) {
  const size_t ov = (size_t)f.nocc * f.nvir;
  return align_up(ov * ov, kAlignElems) * (wants_tt(f) ? 2 : 1) +
         align_up(2 * (size_t)f.nocc * f.nocc, kAlignElems);
}

size_t frag_ws_elems(const rimp2_plan* p, const rimp2_frag& f) {
  if (p->precision == RIMP2_FP64) return frag_ws_elems_fp64(f);
  return (split_frag_ws_bytes(p->split, f) + 7) / 8;
}

int check_frag_shapes(const rimp2_frag* frags, int nfrag) {
  for (int f = 0; f < nfrag; ++f) {
    const rimp2_frag& x = frags[f];
    if (x.nocc < 0 || x.nvir < 0 || x.naux < 0) return RIMP2_ERR_BAD_ARG;
    // index arithmetic uses 32-bit row/column indices within one fragment
    if ((long long)x.nocc * x.nvir > (1LL << 30) || x.naux > (1 << 30)) return RIMP2_ERR_UNSUPPORTED;
  }
  return RIMP2_OK;
}

// split-K factor over the outer K index so that small M x N problems fill the GPU
void choose_split(GemmProb& P, int grid, int mul) {
  const long long tiles = (long long)P.tiles_m * P.tiles_n;
  long long want = std::max(1LL, ((long long)mul * grid + tiles - 1) / tiles);
  want = std::min<long long>(want, P.K1);
  int chunk = (int)((P.K1 + want - 1) / want);
  if (chunk < 1) chunk = 1;
  P.k1_chunk = chunk;
  P.ksplit = (P.K1 + chunk - 1) / chunk;
  if (P.ksplit < 1) P.ksplit = 1;
}

void finish_probs(std::vector<GemmProb>& v, long long& total) {
  // largest work per tile first (LPT order of the device queue)
  std::stable_sort(v.begin(), v.end(), [](const GemmProb& a, const GemmProb& b) {
    const double ca = (double)a.K0 * a.k1_chunk, cb = (double)b.K0 * b.k1_chunk;
    return ca > cb;
  });
  total = 0;
  for (auto& P : v) {
    P.tile_begin = total;
    total += P.ntiles;
  }
}

int build_fp64_wave(rimp2_plan* p, const rimp2_frag* frags, WaveDesc& w) {
  size_t ws = 0;
  long long pairs = 0;
  for (int idx : w.frags) {
    const rimp2_frag& f = frags[idx];
    FragDev d{};
    d.o = f.nocc; d.v = f.nvir; d.X = f.naux; d.idx = idx;
    d.b_off = f.b_off; d.eo_off = f.eo_off; d.ev_off = f.ev_off;
    const size_t ov = (size_t)f.nocc * f.nvir;
    d.t_off = (long long)ws; ws += align_up(ov * ov, kAlignElems);
    d.tt_off = -1;
    if (wants_tt(f)) { d.tt_off = (long long)ws; ws += align_up(ov * ov, kAlignElems); }
    d.ep_off = (long long)ws;                  // pair energies, then opposite-spin ones
    d.epos_off = d.ep_off + (long long)f.nocc * f.nocc;
    ws += align_up(2 * (size_t)f.nocc * f.nocc, kAlignElems);
    d.gamma_off = f.gamma_off; d.pij_off = f.pij_off; d.pab_off = f.pab_off;
    d.epair_off = f.epair_off;
    d.pair_begin = pairs;
    pairs += (long long)f.nocc * (f.nocc + 1) / 2;
    w.fdev.push_back(d);
    w.max_b = std::max<long long>(w.max_b, (long long)ov * f.naux);
    if (ov == 0) continue;
    const int o = f.nocc, v = f.nvir, X = f.naux;
    // V: rows (i,a), cols (j,b), K = Q; upper triangle of tiles
    {
      GemmProb P{};
      P.kind = PK_V; P.frag = idx;
      P.M = P.N = (int)ov; P.K0 = X; P.K1 = 1;
      P.tiles_m = P.tiles_n = (int)((ov + F64_BM - 1) / F64_BM);
      P.ksplit = 1; P.k1_chunk = 1;
      P.ntiles = (long long)P.tiles_m * (P.tiles_m + 1) / 2;
      P.a_off = f.b_off; P.b_off = f.b_off; P.c_off = d.t_off;
      P.sAm = X; P.sAk = 1; P.sA1 = 0; P.sBn = X; P.sBk = 1; P.sB1 = 0; P.ldc = (long long)ov;
      P.alpha = 1.0; P.eo_off = f.eo_off; P.ev_off = f.ev_off; P.v = v; P.b_from_B = 1;
      w.probs_v.push_back(P);  // naux = 0 still writes T = 0
    }
    if (f.gamma_off >= 0 && X > 0) {  // Gamma[(i,a)][Q] = sum_(j,b) Tt[(i,a)][(j,b)] B[(j,b)][Q]
      GemmProb P{};
      P.kind = PK_GAMMA; P.frag = idx;
      P.M = (int)ov; P.N = X; P.K0 = (int)ov; P.K1 = 1;
      P.tiles_m = (int)((ov + F64_BM - 1) / F64_BM); P.tiles_n = (X + F64_BN - 1) / F64_BN;
      P.ksplit = 1; P.k1_chunk = 1;
      P.ntiles = (long long)P.tiles_m * P.tiles_n;
      P.a_off = d.tt_off; P.b_off = f.b_off; P.c_off = f.gamma_off;
      P.sAm = (long long)ov; P.sAk = 1; P.sA1 = 0;
      P.sBn = 1; P.sBk = X; P.sB1 = 0; P.ldc = X;
      P.alpha = 1.0; P.v = v; P.b_from_B = 1;
      w.probs_c.push_back(P);
    }
    if (f.pab_off >= 0) {  // P_ab = sum_i Tt[i][a][:] . T[i][b][:]
      GemmProb P{};
      P.kind = PK_PAB; P.frag = idx;
      P.M = P.N = v; P.K0 = (int)ov; P.K1 = o;
      P.tiles_m = P.tiles_n = (v + F64_BM - 1) / F64_BM;
      P.a_off = d.tt_off; P.b_off = d.t_off; P.c_off = f.pab_off;
      P.sAm = (long long)ov; P.sAk = 1; P.sA1 = (long long)v * ov;
      P.sBn = (long long)ov; P.sBk = 1; P.sB1 = (long long)v * ov; P.ldc = v;
      P.alpha = 1.0; P.v = v; P.b_from_B = 0;
      choose_split(P, p->gemm_grid, 2 << p->variant);
      P.ntiles = (long long)P.tiles_m * P.tiles_n * P.ksplit;
      w.probs_c.push_back(P);
    }
    if (f.pij_off >= 0) {  // P_ij = -sum_(k,b) sum_a Tt[k][b][i][a] T[k][b][j][a]
      GemmProb P{};
      P.kind = PK_PIJ; P.frag = idx;
      P.M = P.N = o; P.K0 = v; P.K1 = (int)ov;
      P.tiles_m = P.tiles_n = (o + F64_BM - 1) / F64_BM;
      P.a_off = d.tt_off; P.b_off = d.t_off; P.c_off = f.pij_off;
      P.sAm = v; P.sAk = 1; P.sA1 = (long long)ov;
      P.sBn = v; P.sBk = 1; P.sB1 = (long long)ov; P.ldc = o;
      P.alpha = -1.0; P.v = v; P.b_from_B = 0;
      choose_split(P, p->gemm_grid, 2 << p->variant);
      P.ntiles = (long long)P.tiles_m * P.tiles_n * P.ksplit;
      w.probs_c.push_back(P);
    }
  }
  w.total_pairs = pairs;
  finish_probs(w.probs_v, w.tiles_v);
  finish_probs(w.probs_c, w.tiles_c);
  // the layout must fit the workspace the plan sized with frag_ws_elems_fp64
  if (ws * sizeof(double) + 256 > p->ws_bytes) return RIMP2_ERR_WORKSPACE;
  return RIMP2_OK;
}

int upload_descriptors(rimp2_plan* p, const rimp2_frag* frags, const double* B, void* ws) {
  p->waves.clear();
  p->split.variant = p->variant;
  for (auto& m : p->wave_members) {
    WaveDesc w;
    w.frags = m;
    if (p->precision == RIMP2_FP64) {
      int rc = build_fp64_wave(p, frags, w);
      if (rc != RIMP2_OK) return rc;
    } else {
      int rc = split_build_wave(p->split, frags, m, B, ws, w.fdev, w.split, w.total_pairs, w.max_b);
      if (rc != RIMP2_OK) return rc;
    }
    p->waves.push_back(std::move(w));
  }
  for (int k = 0; k < 4; ++k) p->stats.tc_flops[k] = 0.0;
  for (const auto& w : p->waves) {
    p->stats.tc_flops[0] += w.split.mma_v;
    p->stats.tc_flops[1] += w.split.mma_c;
    p->stats.tc_flops[2] += w.split.mma_g;
  }
  // layout of the device block
  size_t off = 256;                                        // status word
  const size_t nctr = p->waves.size() * 8;
  size_t ctr_off = off;
  off = align_up(off + nctr * sizeof(unsigned), 256);
  for (auto& w : p->waves) {
    w.off_fdev = off; off = align_up(off + w.fdev.size() * sizeof(FragDev), 256);
    w.off_pv = off; off = align_up(off + w.probs_v.size() * sizeof(GemmProb), 256);
    w.off_pc = off; off = align_up(off + w.probs_c.size() * sizeof(GemmProb), 256);
    off = split_layout_wave(w.split, off);
  }
  if (off > p->dblk_bytes) {
    if (p->dblk) cudaFree(p->dblk);
    p->dblk = nullptr;
    p->dblk_bytes = 0;
    if (cudaMalloc(&p->dblk, off) != cudaSuccess) { cudaGetLastError(); return RIMP2_ERR_NOMEM; }
    p->dblk_bytes = off;
    if (cudaMemset(p->dblk, 0, off) != cudaSuccess) return RIMP2_ERR_CUDA;
  }
  p->d_status = (unsigned*)p->dblk;
  p->d_counters = (unsigned*)(p->dblk + ctr_off);
  std::vector<char> host(off, 0);
  for (auto& w : p->waves) {
    if (!w.fdev.empty()) memcpy(host.data() + w.off_fdev, w.fdev.data(), w.fdev.size() * sizeof(FragDev));
    if (!w.probs_v.empty()) memcpy(host.data() + w.off_pv, w.probs_v.data(), w.probs_v.size() * sizeof(GemmProb));
    if (!w.probs_c.empty()) memcpy(host.data() + w.off_pc, w.probs_c.data(), w.probs_c.size() * sizeof(GemmProb));
    split_fill_wave(w.split, host.data());
  }
  // keep the status word, rewrite the rest
  if (cudaMemcpy(p->dblk + 256, host.data() + 256, off - 256, cudaMemcpyHostToDevice) != cudaSuccess)
    return RIMP2_ERR_CUDA;
  p->have_desc = true;
  return RIMP2_OK;
}

int enqueue(rimp2_plan* p, const rimp2_batch* b, void* ws, cudaStream_t s) {
  Bases bs{};
  bs.B = b->B; bs.eps = b->eps; bs.ws = (double*)ws;
  bs.gamma = b->gamma; bs.pij = b->pij; bs.pab = b->pab; bs.epair = b->epair;
  bs.energy = b->energy; bs.energy_os = b->energy_os; bs.status = p->d_status;
  bs.energy_scs = b->energy_scs; bs.scs_os = p->opt.scs_os; bs.scs_ss = p->opt.scs_ss;
  int launches = 0;
  long long tiles = 0;
  if (cudaMemsetAsync(p->d_counters, 0, p->waves.size() * 8 * sizeof(unsigned), s) != cudaSuccess)
    return RIMP2_ERR_CUDA;
  for (size_t wi = 0; wi < p->waves.size(); ++wi) {
    WaveDesc& w = p->waves[wi];
    const FragDev* dfd = (const FragDev*)(p->dblk + w.off_fdev);
    const int nf = (int)w.fdev.size();
    unsigned* ctr = p->d_counters + wi * 8;
    cudaError_t e = cudaSuccess;
    cudaEvent_t* ev = p->stage_ev.empty() ? nullptr : &p->stage_ev[wi * kEv];
    if (ev && cudaEventRecordWithFlags(ev[0], s, cudaEventRecordExternal) != cudaSuccess) return RIMP2_ERR_CUDA;
    if (p->opt.check_inputs) {
      e = launch_check_inputs(dfd, nf, (w.max_b + 255) / 256, bs, s);
      ++launches;
      if (e != cudaSuccess) return RIMP2_ERR_CUDA;
    }
    if (p->precision == RIMP2_FP64) {
      if (ev) cudaEventRecordWithFlags(ev[1], s, cudaEventRecordExternal);
      e = launch_gemm_f64((const GemmProb*)(p->dblk + w.off_pv), (int)w.probs_v.size(), w.tiles_v,
                          bs, ctr + 0, p->gemm_grid, s);
      launches += w.tiles_v > 0;
      if (ev) cudaEventRecordWithFlags(ev[2], s, cudaEventRecordExternal);
      if (e == cudaSuccess) { e = launch_amplitude_f64(dfd, nf, w.total_pairs, bs, s); launches += w.total_pairs > 0; }
      if (e == cudaSuccess) { e = launch_energy_reduce(dfd, nf, bs, s); ++launches; }
      if (e == cudaSuccess) { e = launch_zero_p(dfd, nf, bs, s); ++launches; }
      if (ev) cudaEventRecordWithFlags(ev[3], s, cudaEventRecordExternal);
      if (e == cudaSuccess) {
        e = launch_gemm_f64((const GemmProb*)(p->dblk + w.off_pc), (int)w.probs_c.size(), w.tiles_c,
                            bs, ctr + 1, p->gemm_grid, s);
        launches += w.tiles_c > 0;
      }
      tiles += w.tiles_v + w.tiles_c;
      if (ev) cudaEventRecordWithFlags(ev[4], s, cudaEventRecordExternal);
      if (ev) cudaEventRecordWithFlags(ev[5], s, cudaEventRecordExternal);
      if (e != cudaSuccess) return RIMP2_ERR_CUDA;
    } else {
      int nl = 0;
      long long nt = 0;
      int rc = split_enqueue_wave(p->split, w.split, p->dblk, dfd, nf, w.total_pairs, bs, ctr, s,
                                  &nl, &nt, ev);
      launches += nl;
      tiles += nt;
      if (rc != RIMP2_OK) return rc;
    }
  }
  p->stats.launches_per_call = launches;
  p->stats.tiles_per_call = tiles;
  return RIMP2_OK;
}

void drop_graph(rimp2_plan* p) {
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  if (p->graph) cudaGraphDestroy(p->graph);
  p->gexec = nullptr;
  p->graph = nullptr;
}

constexpr int kFp64Variants = 3;   // FP64 path: split-K target 2, 4, 8 x grid

uint64_t fnv(uint64_t h, uint64_t x) {
  for (int b = 0; b < 8; ++b) {
    h ^= (x >> (8 * b)) & 0xFF;
    h *= 1099511628211ull;
  }
  return h;
}

uint64_t tune_key(const rimp2_plan* p) {
  uint64_t h = 1469598103934665603ull;
  h = fnv(h, (uint64_t)p->precision);
  h = fnv(h, (uint64_t)p->opt.slices_v);
  h = fnv(h, (uint64_t)p->opt.slices_t);
  h = fnv(h, (uint64_t)p->opt.slices_g);
  h = fnv(h, (uint64_t)p->frags.size());
  for (const auto& f : p->frags) {
    h = fnv(h, ((uint64_t)f.nocc << 42) ^ ((uint64_t)f.nvir << 21) ^ (uint64_t)f.naux);
    h = fnv(h, (uint64_t)((f.gamma_off >= 0) | ((f.pij_off >= 0) << 1) | ((f.pab_off >= 0) << 2)));
  }
  return h;
}

constexpr int kBestShapes = -2;

// A cache line is "<key> <variant> <shape V> <shape P> <shape Gamma>" (hex key; the
// shapes are indices into the plan's candidate lists, which the options determine).
bool cache_lookup(const std::string& path, uint64_t key, int out[4]) {
  if (path.empty()) return false;
  FILE* fh = fopen(path.c_str(), "r");
  if (!fh) return false;
  char line[256];
  bool found = false;
  while (fgets(line, sizeof(line), fh)) {
    unsigned long long k = 0;
    int v[4] = {-1, 0, 0, 0};
    if (sscanf(line, "%llx %d %d %d %d", &k, &v[0], &v[1], &v[2], &v[3]) >= 2 && k == key) {
      for (int i = 0; i < 4; ++i) out[i] = v[i];
      found = true;
    }
  }
  fclose(fh);
  return found;
}

void cache_store(const std::string& path, uint64_t key, const int v[4]) {
  if (path.empty()) return;
  FILE* fh = fopen(path.c_str(), "a");
  if (!fh) return;
  fprintf(fh, "%016llx %d %d %d %d\n", (unsigned long long)key, v[0], v[1], v[2], v[3]);
  fclose(fh);
}

// device time between stage events a and b of the last call, summed over the waves
double span_ms(rimp2_plan* p, int a, int b) {
  double ms = 0.0;
  for (size_t w = 0; w < p->wave_members.size(); ++w) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, p->stage_ev[w * kEv + a], p->stage_ev[w * kEv + b]) == cudaSuccess)
      ms += t;
    cudaGetLastError();
  }
  return ms;
}

void publish_shapes(rimp2_plan* p) {
  if (p->precision == RIMP2_FP64) return;
  const SplitLaunch* c[3] = {&p->split.cfg_v, &p->split.cfg_t, &p->split.cfg_g};
  for (int i = 0; i < 3; ++i) {
    p->stats.n_tile[i] = c[i]->n_tile_max;
    p->stats.stage_k[i] = c[i]->bk;
  }
}

// per launch, the candidate shape of the fastest shape trial
void set_best_shapes(rimp2_plan* p) {
  const std::vector<double>* t[3] = {&p->tr_v, &p->tr_p, &p->tr_g};
  int best[3] = {-1, -1, -1};
  for (int l = 0; l < 3; ++l)
    for (size_t i = 0; i < p->trials.size(); ++i)
      if (p->trials[i].shape >= 0 && (best[l] < 0 || (*t[l])[i] < (*t[l])[best[l]]))
        best[l] = (int)i;
  if (best[0] < 0) return;
  split_set_shapes(p->split, p->trials[best[0]].shape, p->trials[best[1]].shape,
                   p->trials[best[2]].shape);
}

double frag_flops(const rimp2_frag& f) {
  const double o = f.nocc, v = f.nvir, X = f.naux;
  return o * (o + 1) * v * v * X + 2 * o * o * v * v * X + 2 * o * o * v * v * v + 2 * o * o * o * v * v;
}

}  // namespace

extern "C" {

int rimp2_plan_create(const rimp2_frag* frags, int32_t nfrag, int32_t precision,
                      const rimp2_options* opt, rimp2_plan** out) {
  if (!out) return RIMP2_ERR_BAD_ARG;
  *out = nullptr;
  if (nfrag < 0 || (nfrag > 0 && !frags)) return RIMP2_ERR_BAD_ARG;
  if (precision != RIMP2_FP64 && precision != RIMP2_BF16_SPLIT && precision != RIMP2_FP8_SPLIT)
    return RIMP2_ERR_UNSUPPORTED;
  int rc = check_frag_shapes(frags, nfrag);
  if (rc != RIMP2_OK) return rc;
  rimp2_options o;
  rimp2_default_options(&o);
  if (opt) o = *opt;
  const bool fp8 = precision == RIMP2_FP8_SPLIT;
  if (o.slices_v == 0) o.slices_v = fp8 ? 8 : 5;
  if (o.slices_t == 0) o.slices_t = fp8 ? 10 : 6;
  if (o.slices_g == 0) o.slices_g = fp8 ? o.slices_t : 5;
  const int smax = fp8 ? 16 : 8;   // levels x tile width must fit the 512 TMEM columns
  if (precision != RIMP2_FP64 &&
      (o.slices_v < 2 || o.slices_v > smax || o.slices_t < 2 || o.slices_t > smax ||
       o.slices_g < 2 || o.slices_g > smax ||
       (o.stage_k != 0 && o.stage_k != 16 && o.stage_k != 32) ||
       (o.n_tile != 0 && o.n_tile != 48 && o.n_tile != 64 && o.n_tile != 80 && o.n_tile != 96)))
    return RIMP2_ERR_UNSUPPORTED;
  rimp2_plan* p = new (std::nothrow) rimp2_plan();
  if (!p) return RIMP2_ERR_NOMEM;
  p->precision = precision;
  p->opt = o;
  p->frags.assign(frags, frags + nfrag);
  if (cudaGetDevice(&p->device) != cudaSuccess) { delete p; return RIMP2_ERR_CUDA; }
  p->gemm_grid = gemm_f64_occupancy_grid();
  if (precision != RIMP2_FP64) {
    rc = split_plan_init(p->split, precision, o);
    if (rc != RIMP2_OK) { delete p; return rc; }
  }
  // waves: batch order, a new wave when the workspace budget would be exceeded
  size_t cur = 0, worst = 0;
  std::vector<int> wave;
  for (int f = 0; f < nfrag; ++f) {
    const size_t need = frag_ws_elems(p, frags[f]) * sizeof(double);
    if (o.max_workspace_bytes > 0 && !wave.empty() && cur + need > o.max_workspace_bytes) {
      p->wave_members.push_back(wave);
      worst = std::max(worst, cur);
      wave.clear();
      cur = 0;
    }
    wave.push_back(f);
    cur += need;
  }
  if (!wave.empty() || p->wave_members.empty()) p->wave_members.push_back(wave);
  worst = std::max(worst, cur);
  p->ws_bytes = worst + 256;
  p->stats.waves = (int)p->wave_members.size();
  p->stats.slices[0] = o.slices_v;
  p->stats.slices[1] = o.slices_t;
  p->stats.slices[2] = o.slices_g;
  double fl = 0;
  for (int f = 0; f < nfrag; ++f) fl += frag_flops(frags[f]);
  p->stats.flops_per_call = fl;
  if (cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreate(&p->t0) != cudaSuccess || cudaEventCreate(&p->t1) != cudaSuccess) {
    cudaGetLastError();
    rimp2_plan_destroy(p);
    return RIMP2_ERR_CUDA;
  }
  if (o.autotune) {
    p->tune_key = tune_key(p);
    if (o.autotune_cache) p->cache_path = o.autotune_cache;
    const int ncand = precision == RIMP2_FP64 ? kFp64Variants : kSplitVariants;
    int cached[4] = {-1, 0, 0, 0};
    if (cache_lookup(p->cache_path, p->tune_key, cached) && cached[0] >= 0 && cached[0] < ncand) {
      p->variant = cached[0];
      if (precision != RIMP2_FP64) split_set_shapes(p->split, cached[1], cached[2], cached[3]);
      p->tune_state = 2;
    } else {
      // split paths: first one trial per tile shape (each launch takes its own i-th
      // candidate), then the other contraction variants with each launch's fastest shape
      if (precision == RIMP2_FP64) {
        for (int v = 0; v < ncand; ++v) p->trials.push_back({-1, v});
      } else {
        const size_t ns = std::max(p->split.cand_v.size(),
                                   std::max(p->split.cand_t.size(), p->split.cand_g.size()));
        for (size_t i = 0; i < ns; ++i) p->trials.push_back({(int)i, 0});
        for (int v = 1; v < ncand; ++v) p->trials.push_back({kBestShapes, v});
      }
      p->tr_v.assign(p->trials.size(), 0.0);
      p->tr_p = p->tr_g = p->tr_c = p->tr_v;
      p->tune_state = 1;
    }
    p->stats.tune_done = p->tune_state == 2;
    p->stats.tune_variant = p->variant;
    p->stats.tune_trials = (int)p->trials.size();
  }
  publish_shapes(p);
  if (o.profile_stages || o.autotune) {
    p->stage_ev.assign(p->wave_members.size() * kEv, nullptr);
    for (auto& e : p->stage_ev)
      if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); rimp2_plan_destroy(p); return RIMP2_ERR_CUDA; }
  }
  // device block with a zero status word
  p->dblk_bytes = 4096;
  if (cudaMalloc(&p->dblk, p->dblk_bytes) != cudaSuccess) {
    cudaGetLastError();
    p->dblk = nullptr;
    rimp2_plan_destroy(p);
    return RIMP2_ERR_NOMEM;
  }
  cudaMemset(p->dblk, 0, p->dblk_bytes);
  p->d_status = (unsigned*)p->dblk;
  *out = p;
  return RIMP2_OK;
}

int rimp2_workspace_size(const rimp2_plan* p, size_t* bytes) {
  if (!p || !bytes) return RIMP2_ERR_BAD_ARG;
  *bytes = p->ws_bytes;
  return RIMP2_OK;
}

int rimp2_energy_grad(rimp2_plan* p, const rimp2_batch* b, void* workspace, size_t ws_bytes,
                      void* stream) {
  if (!p || !b) return RIMP2_ERR_BAD_ARG;
  if (b->nfrag != (int)p->frags.size() || (b->nfrag > 0 && !b->frags)) return RIMP2_ERR_SHAPE;
  for (int f = 0; f < b->nfrag; ++f) {
    const rimp2_frag& x = b->frags[f];
    const rimp2_frag& y = p->frags[f];
    if (x.nocc != y.nocc || x.nvir != y.nvir || x.naux != y.naux) return RIMP2_ERR_SHAPE;
    if ((x.gamma_off >= 0 && y.gamma_off < 0) || (x.pij_off >= 0 && y.pij_off < 0) ||
        (x.pab_off >= 0 && y.pab_off < 0))
      return RIMP2_ERR_SHAPE;
    if (x.b_off < 0 || x.eo_off < 0 || x.ev_off < 0) return RIMP2_ERR_BAD_ARG;
    if ((x.gamma_off >= 0 && !b->gamma) || (x.pij_off >= 0 && !b->pij) ||
        (x.pab_off >= 0 && !b->pab) || (x.epair_off >= 0 && !b->epair))
      return RIMP2_ERR_BAD_ARG;
  }
  if (b->nfrag > 0 && (!b->B || !b->eps || !b->energy)) return RIMP2_ERR_BAD_ARG;
  if (p->ws_bytes > 256 && (!workspace || ws_bytes < p->ws_bytes)) return RIMP2_ERR_WORKSPACE;
  if (((uintptr_t)workspace & 255) != 0) return RIMP2_ERR_WORKSPACE;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != p->device) return RIMP2_ERR_BAD_ARG;
  cudaStream_t s = (cudaStream_t)stream;

  if (p->tune_state == 1) {
    // in-situ trials (the paper's runtime GEMM variant selection): read the times of the
    // previous call's trial, then set up the next trial or, after the last one, the
    // fastest shapes and variant
    if (p->tune_cur >= 0) {
      if (cudaEventSynchronize(p->done) != cudaSuccess) return RIMP2_ERR_CUDA;
      const int t = p->tune_cur;
      p->tr_v[t] = span_ms(p, 1, 2);
      p->tr_p[t] = span_ms(p, 3, 4);
      p->tr_g[t] = span_ms(p, 4, 5);
      p->tr_c[t] = span_ms(p, 3, 5);
      if (p->trials[t].variant < 4) p->stats.tune_ms[p->trials[t].variant] = p->tr_c[t];
      p->tune_cur = -1;
    }
    const bool split = p->precision != RIMP2_FP64;
    if (p->tune_next < (int)p->trials.size()) {
      const int t = p->tune_next++;
      const auto tr = p->trials[t];
      if (split && tr.shape >= 0) split_set_shapes(p->split, tr.shape, tr.shape, tr.shape);
      if (split && tr.shape == kBestShapes) set_best_shapes(p);
      p->variant = tr.variant;
      p->tune_cur = t;
      p->have_desc = false;   // rebuild descriptors and graph for this trial
    } else {
      int best = -1;
      double best_ms = 0.0;
      if (split) {
        set_best_shapes(p);
        // variant 0 with the fastest shapes: the sum of the two launches' best times
        double v0p = -1.0, v0g = -1.0;
        for (size_t i = 0; i < p->trials.size(); ++i)
          if (p->trials[i].shape >= 0) {
            if (v0p < 0 || p->tr_p[i] < v0p) v0p = p->tr_p[i];
            if (v0g < 0 || p->tr_g[i] < v0g) v0g = p->tr_g[i];
          }
        best = 0;
        best_ms = v0p + v0g;
        p->stats.tune_ms[0] = best_ms;
      }
      for (size_t i = 0; i < p->trials.size(); ++i)
        if (!(split && p->trials[i].shape >= 0) && (best < 0 || p->tr_c[i] < best_ms)) {
          best = p->trials[i].variant;
          best_ms = p->tr_c[i];
        }
      p->variant = best;
      p->tune_state = 2;
      p->stats.tune_done = 1;
      const int rec[4] = {best, p->split.shape_v, p->split.shape_t, p->split.shape_g};
      cache_store(p->cache_path, p->tune_key, rec);
      p->have_desc = false;
    }
    p->stats.tune_variant = p->variant;
    publish_shapes(p);
  }
  Key k{};
  k.p[0] = b->B; k.p[1] = b->eps; k.p[2] = workspace; k.p[3] = b->gamma; k.p[4] = b->pij;
  k.p[5] = b->pab; k.p[6] = b->epair; k.p[7] = b->energy; k.p[8] = b->energy_os;
  k.p[9] = b->energy_scs;
  k.frags.assign(b->frags, b->frags + b->nfrag);
  const bool changed = !p->have_desc || !(k == p->key);
  if (changed) {
    if (cudaEventSynchronize(p->done) != cudaSuccess) return RIMP2_ERR_CUDA;
    drop_graph(p);
    int rc = upload_descriptors(p, b->frags, b->B, workspace);
    if (rc != RIMP2_OK) { p->have_desc = false; return rc; }
    p->key = k;
  }
  if (p->timing_pending) {  // read the previous call's device time if it finished
    float ms = 0;
    if (cudaEventQuery(p->t1) == cudaSuccess && cudaEventElapsedTime(&ms, p->t0, p->t1) == cudaSuccess)
      p->stats.last_ms = ms;
    cudaGetLastError();
    p->timing_pending = false;
  }
  if (cudaEventRecord(p->t0, s) != cudaSuccess) return RIMP2_ERR_CUDA;
  if (p->opt.use_graph) {
    if (!p->gexec) {
      if (cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return RIMP2_ERR_CUDA;
      int rc = enqueue(p, b, workspace, p->cap);
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(p->cap, &g);
      if (rc != RIMP2_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return rc != RIMP2_OK ? rc : RIMP2_ERR_CUDA;
      }
      p->graph = g;
      if (cudaGraphInstantiate(&p->gexec, g, 0) != cudaSuccess) {
        cudaGetLastError();
        drop_graph(p);
        return RIMP2_ERR_CUDA;
      }
      p->stats.graph_captures++;
    }
    if (cudaGraphLaunch(p->gexec, s) != cudaSuccess) return RIMP2_ERR_CUDA;
  } else {
    int rc = enqueue(p, b, workspace, s);
    if (rc != RIMP2_OK) return rc;
  }
  if (cudaEventRecord(p->t1, s) != cudaSuccess || cudaEventRecord(p->done, s) != cudaSuccess)
    return RIMP2_ERR_CUDA;
  p->timing_pending = true;
  p->stats.calls++;
  return RIMP2_OK;
}

int rimp2_get_status(rimp2_plan* p) {
  if (!p) return RIMP2_ERR_BAD_ARG;
  if (cudaEventSynchronize(p->done) != cudaSuccess) return RIMP2_ERR_CUDA;
  if (p->timing_pending) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, p->t0, p->t1) == cudaSuccess) p->stats.last_ms = ms;
    cudaGetLastError();
    p->timing_pending = false;
  }
  unsigned st = 0;
  if (cudaMemcpy(&st, p->d_status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess)
    return RIMP2_ERR_CUDA;
  if (st && cudaMemset(p->d_status, 0, sizeof(unsigned)) != cudaSuccess) return RIMP2_ERR_CUDA;
  int rc = RIMP2_OK;
  if (st & ST_DENOM) rc = RIMP2_ERR_DENOM;
  else if (st & ST_NONFINITE) rc = RIMP2_ERR_NONFINITE;
  else if (st & ST_TIMEOUT) rc = RIMP2_ERR_TIMEOUT;
  else if (st & ST_INTERNAL) rc = RIMP2_ERR_UNSUPPORTED;
  p->stats.status = rc;
  return rc;
}

int rimp2_get_stats(rimp2_plan* p, rimp2_stats* out) {
  if (!p || !out) return RIMP2_ERR_BAD_ARG;
  if (!p->stage_ev.empty() && p->stats.calls > 0) {
    if (cudaEventSynchronize(p->done) != cudaSuccess) { cudaGetLastError(); return RIMP2_ERR_CUDA; }
    for (int k = 0; k < 4; ++k) p->stats.stage_ms[k] = 0.0;
    p->stats.launch_ms[0] = p->stats.launch_ms[1] = 0.0;
    // events per wave: start, after slicing, after V, after the amplitude stage, after
    // the P_ab / P_ij (and Gamma) launch, after the separate Gamma launch
    auto span = [&](size_t w, int a, int b) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, p->stage_ev[w * kEv + a], p->stage_ev[w * kEv + b]) != cudaSuccess)
        ms = 0.f;
      cudaGetLastError();
      return (double)ms;
    };
    for (size_t w = 0; w < p->wave_members.size(); ++w) {
      for (int k = 0; k < 3; ++k) p->stats.stage_ms[k] += span(w, k, k + 1);
      p->stats.stage_ms[3] += span(w, 3, 5);
      p->stats.launch_ms[0] += span(w, 3, 4);
      p->stats.launch_ms[1] += span(w, 4, 5);
    }
  }
  *out = p->stats;
  return RIMP2_OK;
}

void rimp2_plan_destroy(rimp2_plan* p) {
  if (!p) return;
  if (p->done) cudaEventSynchronize(p->done);
  drop_graph(p);
  split_plan_release(p->split);
  if (p->dblk) cudaFree(p->dblk);
  if (p->cap) cudaStreamDestroy(p->cap);
  if (p->done) cudaEventDestroy(p->done);
  if (p->t0) cudaEventDestroy(p->t0);
  if (p->t1) cudaEventDestroy(p->t1);
  for (auto e : p->stage_ev)
    if (e) cudaEventDestroy(e);
  cudaGetLastError();
  delete p;
}

}  // extern "C"
