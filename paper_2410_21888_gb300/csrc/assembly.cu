// MBE3 assembly of the fragments' gradient intermediates over the system's index spaces
// (include/rimp2_mbe.h).  E_MBE3 = sum_f c_f E_f over restrictions of one global B and
// one orbital-energy set, so dE/dB = 4 Gamma_sys, dE/de = 2 diag P_sys with
//   Gamma_sys[(I,J,K)] = sum_f c_f Gamma_f restricted to the block, P_sys = sum_f c_f P_f
// scattered; the trimer coefficients are 1 (Sec. "Asynchronous time steps").
//
// The host builds, per output block, the list of contributing fragment blocks in fragment
// order; the device gathers each output element from its contributors in that order
// (deterministic, no atomics).  Every fragment element is read once.
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "rimp2_mbe.h"

namespace {

// One contribution: fragment element (i, a, q) of the block lives at base + i s0 + a s1 + q
struct Contrib {
  long long base, s0;
  int s1, coeff;
};

// One output block: element (i, a, q) at out_off + i ld0 + a ld1 + q, q < n2 (P: n2 = 1)
struct OutBlock {
  long long out_off, ld0;
  int ld1, n0, n1, n2;
  int c_begin, c_end;
};

__global__ void __launch_bounds__(256)
k_assemble_rows(const OutBlock* __restrict__ blocks, const Contrib* __restrict__ con,
                const int2* __restrict__ items, const double* __restrict__ pool,
                double* __restrict__ out, int accumulate) {
  // one CTA per (block, row i): the n1 x n2 elements of that row of the block
  const int2 it = items[blockIdx.x];
  const OutBlock b = blocks[it.x];
  const int i = it.y;
  const long long ne = (long long)b.n1 * b.n2;
  for (long long e = threadIdx.x; e < ne; e += blockDim.x) {
    const int a = (int)(e / b.n2);
    const int q = (int)(e - (long long)a * b.n2);
    double* o = out + b.out_off + (long long)i * b.ld0 + (long long)a * b.ld1 + q;
    double s = accumulate ? *o : 0.0;
    for (int c = b.c_begin; c < b.c_end; ++c) {
      const Contrib k = con[c];
      s += (double)k.coeff * pool[k.base + (long long)i * k.s0 + (long long)a * k.s1 + q];
    }
    *o = s;
  }
}

struct Table {
  std::vector<OutBlock> blocks;
  std::vector<Contrib> con;
  std::vector<int2> items;
  // device copies (inside the handle's buffer)
  const OutBlock* d_blocks = nullptr;
  const Contrib* d_con = nullptr;
  const int2* d_items = nullptr;
};

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

struct rimp2_assembly {
  int n = 0;
  long long O = 0, V = 0, G = 0;
  std::vector<long long> block_index;
  Table gamma, pij, pab;
  void* dmem = nullptr;
  int device = 0;
};

namespace {

void finish_items(Table& t) {
  for (int b = 0; b < (int)t.blocks.size(); ++b)
    for (int i = 0; i < t.blocks[b].n0; ++i) t.items.push_back(make_int2(b, i));
}

}  // namespace

extern "C" {

int rimp2_assembly_create(int32_t n, const int32_t* nocc, const int32_t* nvir,
                          const int32_t* naux, int64_t nfrag, const int32_t* frag_mon,
                          const int32_t* coeff, const int64_t* gamma_off, const int64_t* pij_off,
                          const int64_t* pab_off, rimp2_assembly** out) {
  if (!out) return RIMP2_ERR_BAD_ARG;
  *out = nullptr;
  if (n <= 0 || n > 2048 || nfrag < 0 || !nocc || !nvir || !naux ||
      (nfrag > 0 && (!frag_mon || !coeff || !gamma_off || !pij_off || !pab_off)))
    return RIMP2_ERR_BAD_ARG;
  for (int m = 0; m < n; ++m)
    if (nocc[m] < 0 || nvir[m] < 0 || naux[m] < 0) return RIMP2_ERR_BAD_ARG;
  rimp2_assembly* a = new (std::nothrow) rimp2_assembly();
  if (!a) return RIMP2_ERR_NOMEM;
  a->n = n;
  std::vector<long long> oo(n + 1, 0), vo(n + 1, 0);
  for (int m = 0; m < n; ++m) {
    oo[m + 1] = oo[m] + nocc[m];
    vo[m + 1] = vo[m] + nvir[m];
  }
  a->O = oo[n];
  a->V = vo[n];
  // fragments: validate, local offsets
  struct FragInfo { int k; int m[3]; long long fo[4], fv[4], fx[4]; };
  std::vector<FragInfo> fi((size_t)nfrag);
  for (int64_t f = 0; f < nfrag; ++f) {
    FragInfo& x = fi[(size_t)f];
    x.k = 0;
    for (int p = 0; p < 3; ++p) {
      const int mm = frag_mon[3 * f + p];
      if (mm < 0) break;
      if (mm >= n) { delete a; return RIMP2_ERR_BAD_ARG; }
      for (int q = 0; q < x.k; ++q)
        if (x.m[q] == mm) { delete a; return RIMP2_ERR_BAD_ARG; }
      x.m[x.k++] = mm;
    }
    if (x.k == 0) { delete a; return RIMP2_ERR_BAD_ARG; }
    x.fo[0] = x.fv[0] = x.fx[0] = 0;
    for (int p = 0; p < x.k; ++p) {
      x.fo[p + 1] = x.fo[p] + nocc[x.m[p]];
      x.fv[p + 1] = x.fv[p] + nvir[x.m[p]];
      x.fx[p + 1] = x.fx[p] + naux[x.m[p]];
    }
  }
  // Gamma blocks: every monomer triple held by some fragment, in (I, J, K) order
  std::map<std::tuple<int, int, int>, std::vector<Contrib>> gmap;
  std::map<std::pair<int, int>, std::vector<Contrib>> pimap, pamap;
  for (int64_t f = 0; f < nfrag; ++f) {
    const FragInfo& x = fi[(size_t)f];
    const long long of = x.fo[x.k], vf = x.fv[x.k], Xf = x.fx[x.k];
    for (int p = 0; p < x.k; ++p)
      for (int q = 0; q < x.k; ++q) {
        const int I = x.m[p], J = x.m[q];
        auto& lp = pimap[{I, J}];
        auto& la = pamap[{I, J}];
        if (pij_off[f] >= 0)
          lp.push_back({pij_off[f] + x.fo[p] * of + x.fo[q], of, 1, coeff[f]});
        if (pab_off[f] >= 0)
          la.push_back({pab_off[f] + x.fv[p] * vf + x.fv[q], vf, 1, coeff[f]});
        for (int r = 0; r < x.k; ++r) {
          const int K = x.m[r];
          auto& lg = gmap[{I, J, K}];
          if (gamma_off[f] >= 0)
            lg.push_back({gamma_off[f] + (x.fo[p] * vf + x.fv[q]) * Xf + x.fx[r], vf * Xf,
                          (int)Xf, coeff[f]});
        }
      }
  }
  a->block_index.assign((size_t)n * n * n, -1);
  long long goff = 0;
  for (auto& kv : gmap) {
    const int I = std::get<0>(kv.first), J = std::get<1>(kv.first), K = std::get<2>(kv.first);
    OutBlock b{};
    b.out_off = goff;
    b.n0 = nocc[I]; b.n1 = nvir[J]; b.n2 = naux[K];
    b.ld0 = (long long)b.n1 * b.n2; b.ld1 = b.n2;
    b.c_begin = (int)a->gamma.con.size();
    a->gamma.con.insert(a->gamma.con.end(), kv.second.begin(), kv.second.end());
    b.c_end = (int)a->gamma.con.size();
    a->block_index[((size_t)I * n + J) * n + K] = goff;
    goff += (long long)b.n0 * b.n1 * b.n2;
    if (b.n0 > 0 && b.n1 > 0 && b.n2 > 0) a->gamma.blocks.push_back(b);
  }
  a->G = goff;
  auto pblocks = [&](std::map<std::pair<int, int>, std::vector<Contrib>>& mp, Table& t,
                     const std::vector<long long>& off, const int32_t* sz, long long ld) {
    for (auto& kv : mp) {
      if (kv.second.empty()) continue;
      const int I = kv.first.first, J = kv.first.second;
      OutBlock b{};
      b.out_off = off[I] * ld + off[J];
      b.ld0 = ld; b.ld1 = 1;
      b.n0 = sz[I]; b.n1 = sz[J]; b.n2 = 1;
      b.c_begin = (int)t.con.size();
      t.con.insert(t.con.end(), kv.second.begin(), kv.second.end());
      b.c_end = (int)t.con.size();
      if (b.n0 > 0 && b.n1 > 0) t.blocks.push_back(b);
    }
  };
  pblocks(pimap, a->pij, oo, nocc, a->O);
  pblocks(pamap, a->pab, vo, nvir, a->V);
  finish_items(a->gamma);
  finish_items(a->pij);
  finish_items(a->pab);
  // device tables
  Table* ts[3] = {&a->gamma, &a->pij, &a->pab};
  size_t bytes = 0;
  for (Table* t : ts)
    bytes += al256(t->blocks.size() * sizeof(OutBlock) + 1) + al256(t->con.size() * sizeof(Contrib) + 1) +
             al256(t->items.size() * sizeof(int2) + 1);
  if (cudaGetDevice(&a->device) != cudaSuccess || cudaMalloc(&a->dmem, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete a;
    return RIMP2_ERR_CUDA;
  }
  std::vector<char> host(bytes, 0);
  size_t off = 0;
  for (Table* t : ts) {
    const size_t nb = t->blocks.size() * sizeof(OutBlock), nc = t->con.size() * sizeof(Contrib),
                 ni = t->items.size() * sizeof(int2);
    if (nb) memcpy(host.data() + off, t->blocks.data(), nb);
    t->d_blocks = (const OutBlock*)((char*)a->dmem + off);
    off += al256(nb + 1);
    if (nc) memcpy(host.data() + off, t->con.data(), nc);
    t->d_con = (const Contrib*)((char*)a->dmem + off);
    off += al256(nc + 1);
    if (ni) memcpy(host.data() + off, t->items.data(), ni);
    t->d_items = (const int2*)((char*)a->dmem + off);
    off += al256(ni + 1);
  }
  if (cudaMemcpy(a->dmem, host.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(a->dmem);
    delete a;
    return RIMP2_ERR_CUDA;
  }
  *out = a;
  return RIMP2_OK;
}

int rimp2_assembly_sizes(const rimp2_assembly* a, int64_t* gamma_elems, int64_t* o_total,
                         int64_t* v_total) {
  if (!a) return RIMP2_ERR_BAD_ARG;
  if (gamma_elems) *gamma_elems = a->G;
  if (o_total) *o_total = a->O;
  if (v_total) *v_total = a->V;
  return RIMP2_OK;
}

int rimp2_assembly_block_index(const rimp2_assembly* a, int64_t* index) {
  if (!a || !index) return RIMP2_ERR_BAD_ARG;
  memcpy(index, a->block_index.data(), a->block_index.size() * sizeof(int64_t));
  return RIMP2_OK;
}

int rimp2_assembly_run(const rimp2_assembly* a, const double* gamma, const double* pij,
                       const double* pab, double* gamma_sys, double* pij_sys, double* pab_sys,
                       int32_t accumulate, void* stream) {
  if (!a) return RIMP2_ERR_BAD_ARG;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != a->device) return RIMP2_ERR_BAD_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const Table* ts[3] = {&a->gamma, &a->pij, &a->pab};
  const double* in[3] = {gamma, pij, pab};
  double* outp[3] = {gamma_sys, pij_sys, pab_sys};
  const long long dense[3] = {0, a->O * a->O, a->V * a->V};
  for (int k = 0; k < 3; ++k) {
    if (!outp[k]) continue;
    const Table& t = *ts[k];
    if (!t.con.empty() && !in[k]) return RIMP2_ERR_BAD_ARG;
    if (!accumulate && k > 0 && dense[k] > 0 &&
        cudaMemsetAsync(outp[k], 0, (size_t)dense[k] * sizeof(double), s) != cudaSuccess)
      return RIMP2_ERR_CUDA;
    if (t.items.empty()) continue;
    k_assemble_rows<<<(unsigned)t.items.size(), 256, 0, s>>>(t.d_blocks, t.d_con, t.d_items,
                                                            in[k], outp[k], accumulate ? 1 : 0);
    if (cudaGetLastError() != cudaSuccess) return RIMP2_ERR_CUDA;
  }
  return RIMP2_OK;
}

void rimp2_assembly_destroy(rimp2_assembly* a) {
  if (!a) return;
  if (a->dmem) cudaFree(a->dmem);
  delete a;
}

}  // extern "C"
