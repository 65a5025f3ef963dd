// Split-precision tensor-core GEMM for sm_103a: TMA-fed, tcgen05.mma (kind::f16, BF16
// in, FP32 TMEM accumulators), one persistent CTA per SM pulling tiles from a device
// queue in LPT order.  Roles: warp 0 issues TMA loads, warp 1 allocates TMEM and issues
// the MMAs from one thread, the 8 or 16 epilogue warps (warps 2..) drain TMEM every K
// chunk (512 BF16 / 8192 FP8 elements) into double-float registers and run the problem's
// epilogue (two accumulator sets alternate when both fit the 512 TMEM columns).
//
// Every mbarrier wait is bounded (globaltimer, 2 s): on expiry the CTA records
// ST_TIMEOUT in the status word and stops all roles; the MMA issuer commits the MMAs it
// has issued to an mbarrier and waits for them, the TMA producer waits for its own loads
// in flight (both bounded by the normal limit), and only then is TMEM freed and the CTA
// returns.
#include <cudaTypedefs.h>

#include <algorithm>

#include "split_gemm.cuh"

namespace rimp2 {

// ------------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

__device__ __forceinline__ uint32_t mbar_try_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok;
}

// non-blocking probe of the same phase
__device__ __forceinline__ uint32_t mbar_test_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // a healthy wait takes microseconds

// Limit of the consumer-side waits (the MMA issuer and the epilogue warps).  A test hook
// (rimp2_testing_set_wait_limit) shortens it so that those waits expire on purpose; the
// producer's waits and the drains after an abort always keep kWaitLimitNs.
__device__ unsigned long long g_sg_consumer_wait_ns = kWaitLimitNs;

// Bounded wait for the phase of parity `parity`; false on timeout or abort.  A limit of 0
// (test hook) gives up unless one non-blocking probe finds the phase complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag,
                                          uint64_t limit_ns = kWaitLimitNs) {
  if (limit_ns == 0) {
    if (mbar_test_wait(b, parity)) return true;
    *abort_flag = 1;
    return false;
  }
  if (mbar_try_wait(b, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(b, parity)) return true;
    if ((it & 63u) == 0) {
      if (*abort_flag) return false;
      if (global_ns() - t0 > limit_ns) {
        *abort_flag = 1;
        return false;
      }
    }
  }
}

// The same wait for a whole warp whose lanes all call it: the lanes leave together, on
// success once every lane has seen the phase complete (it stays complete until this warp
// arrives on the paired barrier), on timeout or abort by lane 0's decision, so that no
// lane runs ahead into a .sync.aligned tcgen05 instruction without the others.
__device__ __forceinline__ bool mbar_wait_warp(uint64_t* b, uint32_t parity,
                                               volatile int* abort_flag, uint64_t limit_ns) {
  const bool lead = (threadIdx.x & 31) == 0;
  if (limit_ns == 0) {   // uniform across the warp
    if (__all_sync(0xffffffffu, mbar_test_wait(b, parity))) return true;
    if (lead) *abort_flag = 1;
    __syncwarp();
    return false;
  }
  const uint64_t t0 = lead ? global_ns() : 0;
  for (uint32_t it = 1;; ++it) {
    if (__all_sync(0xffffffffu, mbar_try_wait(b, parity))) return true;
    if ((it & 63u) == 0) {
      int give_up = 0;
      if (lead) give_up = (*abort_flag != 0) || (global_ns() - t0 > limit_ns);
      if (__shfl_sync(0xffffffffu, give_up, 0)) {
        if (lead) *abort_flag = 1;
        __syncwarp();
        return false;
      }
    }
  }
}

__device__ __forceinline__ void tma_3d(uint32_t dst, const CUtensorMap* tm, uint64_t* bar, int c0,
                                       int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
      "l"(tm), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

__device__ __forceinline__ void tma_4d(uint32_t dst, const CUtensorMap* tm, uint64_t* bar, int c0,
                                       int c1, int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(dst),
      "l"(tm), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
      : "memory");
}

__device__ __forceinline__ void tma_5d(uint32_t dst, const CUtensorMap* tm, uint64_t* bar, int c0,
                                       int c1, int c2, int c3, int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6, %7}], [%2];" ::"r"(dst),
      "l"(tm), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_f8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                        uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r0, r1, r2, r3, r4, r5, r6, r7;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3), "=r"(r4), "=r"(r5), "=r"(r6), "=r"(r7)
               : "r"(taddr)
               : "memory");
  v[0] = __uint_as_float(r0); v[1] = __uint_as_float(r1);
  v[2] = __uint_as_float(r2); v[3] = __uint_as_float(r3);
  v[4] = __uint_as_float(r4); v[5] = __uint_as_float(r5);
  v[6] = __uint_as_float(r6); v[7] = __uint_as_float(r7);
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float* v) {
  uint32_t r0, r1, r2, r3;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(taddr)
               : "memory");
  v[0] = __uint_as_float(r0); v[1] = __uint_as_float(r1);
  v[2] = __uint_as_float(r2); v[3] = __uint_as_float(r3);
}

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Columns c .. c+NC-1 of this warp's 32 TMEM lanes (NC a multiple of 4), issued without
// waiting; the values are valid after tmem_wait_ld and tmem_hold.
template <int NC>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, float (&v)[NC]) {
#pragma unroll
  for (int g = 0; g < NC / 8; ++g) tmem_ld8(taddr + (uint32_t)(g * 8), v + g * 8);
  if constexpr (NC % 8 == 4) tmem_ld4(taddr + (uint32_t)(NC - 4), v + NC - 4);
}

// Ties the registers of an asynchronous TMEM load to the point after tcgen05.wait::ld, so
// that no computation on them is scheduled before the wait.
template <int NC>
__device__ __forceinline__ void tmem_hold(float (&v)[NC]) {
#pragma unroll
  for (int g = 0; g < NC / 8; ++g)
    asm volatile("" : "+f"(v[g * 8 + 0]), "+f"(v[g * 8 + 1]), "+f"(v[g * 8 + 2]), "+f"(v[g * 8 + 3]),
                 "+f"(v[g * 8 + 4]), "+f"(v[g * 8 + 5]), "+f"(v[g * 8 + 6]), "+f"(v[g * 8 + 7]));
  if constexpr (NC % 8 == 4)
    asm volatile("" : "+f"(v[NC - 4]), "+f"(v[NC - 3]), "+f"(v[NC - 2]), "+f"(v[NC - 1]));
}

// UMMA shared-memory descriptor of a K-major operand with ROWB-byte rows (64 or 32)
// and the matching swizzle: 8-row core groups 8 ROWB bytes apart (SBO), descriptor
// version 1, layout SWIZZLE_64B (4) for 64-byte rows, SWIZZLE_32B (6) for 32-byte rows.
template <int ROWB>
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  constexpr uint64_t layout = ROWB == 64 ? 4u : 6u;
  constexpr uint64_t sbo = (8u * ROWB) >> 4;
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1u << 16) | (sbo << 32) |
         ((uint64_t)1u << 46) | (layout << 61);
}

// All MMAs of one pipeline stage for S slices, unrolled: for each K step of 16 (BF16) or
// 32 (FP8) elements and each A slice p, one MMA against the contiguous B slices
// q0 .. q0+nq-1 (nq * NT <= 256 columns) writes the column block of B_q into the level-(p+q)
// accumulator at TMEM column (p+q) * NT.  `desc` is the shared-memory descriptor of the
// stage base; every operand tile starts a constant number of 16-byte units above it and
// shared addresses stay below 256 KB, so the 14-bit start field never carries.  The first
// stage of a TMEM chunk (fresh) overwrites the accumulators through the p = 0 MMAs.
template <int S, int NT, int ROWB, bool F8>
__device__ __forceinline__ void mma_stage(uint32_t tmem_base, uint64_t desc, uint32_t idesc_m,
                                          bool fresh) {
  if constexpr (S * NT <= 512) {
    constexpr int kGroup = 256 / NT;
    constexpr uint32_t A16 = (SG_BM * ROWB) >> 4, B16 = (NT * ROWB) >> 4;
#pragma unroll
    for (int k16 = 0; k16 < ROWB / 32; ++k16) {
#pragma unroll
      for (int p = 0; p < S; ++p) {
#pragma unroll
        for (int q0 = 0; q0 + p < S; q0 += kGroup) {
          const int nq = kGroup < S - p - q0 ? kGroup : S - p - q0;
          const uint64_t adesc = desc + (uint64_t)(p * A16 + k16 * 2);
          const uint64_t bdesc = desc + (uint64_t)(S * A16 + q0 * B16 + k16 * 2);
          const uint32_t idesc = idesc_m | ((uint32_t)((nq * NT) >> 3) << 17);
          const uint32_t acc = (fresh && k16 == 0 && p == 0) ? 0u : 1u;
          if (F8) umma_f8(tmem_base + (uint32_t)((p + q0) * NT), adesc, bdesc, idesc, acc);
          else umma_bf16(tmem_base + (uint32_t)((p + q0) * NT), adesc, bdesc, idesc, acc);
        }
      }
    }
  }
}

// ------------------------------------------------------------------ double-float

struct df { float h, l; };

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}

__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.h, b.h);
  s.l += a.l + b.l;
  return fast_two_sum(s.h, s.l);
}

// a / b in double-float: q1 = a_h / b_h (correctly rounded), then two correction terms
// from the remainders, q2 = (a - q1 b) / b_h and q3 = (a - q1 b - q2 b) / b_h, each
// remainder formed with the exact product error of q b_h (FMA) and the b_l term, and the
// division by b_h done with its correctly rounded reciprocal.  One correction term alone
// leaves q2's error, whose part (b_l / b_h) (a - q1 b) / b_h is correlated with q2 and
// biases |T| low by ~6e-16 relative (measured by exact rational arithmetic on 4e4
// quotients), i.e. ~1e-15 of the energy; the third term removes it (mean error below
// 2e-17, rms 1.6e-15).  The products are written with __fmul_rn so that the compiler
// cannot contract them into the additions of the error-free transformations.
__device__ __forceinline__ df df_div(df a, df b) {
  const float q1 = __fdiv_rn(a.h, b.h);
  const float rc = __frcp_rn(b.h);
  const float ph = __fmul_rn(q1, b.h);
  const float pl = fmaf(q1, b.h, -ph);
  const float r = fmaf(-q1, b.l, __fadd_rn(__fsub_rn(__fsub_rn(a.h, ph), pl), a.l));
  const float q2 = __fmul_rn(r, rc);
  const float ph2 = __fmul_rn(q2, b.h);
  const float pl2 = fmaf(q2, b.h, -ph2);
  const float r2 = fmaf(-q2, b.l, __fsub_rn(__fsub_rn(r, ph2), pl2));
  const float q3 = __fmul_rn(r2, rc);
  const df s = fast_two_sum(q1, q2);
  return fast_two_sum(s.h, __fadd_rn(s.l, q3));
}

// Two FP32 lanes in one 64-bit register for the packed f32x2 arithmetic of sm_100+
// (add/sub/mul/fma.rn.f32x2: each lane rounds exactly like the scalar instruction)
typedef unsigned long long f2x;
__device__ __forceinline__ f2x f2_pack(float a, float b) {
  f2x r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(f2x r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ f2x f2_add(f2x a, f2x b) {
  f2x d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x f2_sub(f2x a, f2x b) {
  f2x d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x f2_mul(f2x a, f2x b) {
  f2x d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x f2_fma(f2x a, f2x b, f2x c) {
  f2x d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2x f2_neg(f2x a) {
  f2x d;
  asm("xor.b64 %0, %1, 0x8000000080000000;" : "=l"(d) : "l"(a));
  return d;
}
// two_sum on two lanes: s = a + b and its exact rounding error
__device__ __forceinline__ void f2_two_sum(f2x a, f2x b, f2x& s, f2x& e) {
  s = f2_add(a, b);
  const f2x bb = f2_sub(s, a);
  e = f2_add(f2_sub(a, f2_sub(s, bb)), f2_sub(b, bb));
}

// fast_two_sum on two lanes (|a| >= |b| in each)
__device__ __forceinline__ void f2_fast_two_sum(f2x a, f2x b, f2x& s, f2x& e) {
  s = f2_add(a, b);
  e = f2_sub(b, f2_sub(s, a));
}

// df_add and df_div on two lanes (two column pairs of double-floats): the same operations
// in the same order as the scalar versions, so each lane's result is bit-identical; only
// the correctly rounded quotient and reciprocal run per lane.
__device__ __forceinline__ void df_add2(f2x ah, f2x al, f2x bh, f2x bl, f2x& h, f2x& l) {
  f2x sh, sl;
  f2_two_sum(ah, bh, sh, sl);
  sl = f2_add(sl, f2_add(al, bl));
  f2_fast_two_sum(sh, sl, h, l);
}
__device__ __forceinline__ void df_div2(f2x ah, f2x al, f2x bh, f2x bl, f2x& h, f2x& l) {
  float a0, a1, b0, b1;
  f2_unpack(ah, a0, a1);
  f2_unpack(bh, b0, b1);
  const f2x q1 = f2_pack(__fdiv_rn(a0, b0), __fdiv_rn(a1, b1));
  const f2x rc = f2_pack(__frcp_rn(b0), __frcp_rn(b1));
  const f2x ph = f2_mul(q1, bh);
  const f2x pl = f2_fma(q1, bh, f2_neg(ph));
  const f2x r = f2_fma(f2_neg(q1), bl, f2_add(f2_sub(f2_sub(ah, ph), pl), al));
  const f2x q2 = f2_mul(r, rc);
  const f2x ph2 = f2_mul(q2, bh);
  const f2x pl2 = f2_fma(q2, bh, f2_neg(ph2));
  const f2x r2 = f2_fma(f2_neg(q2), bl, f2_sub(f2_sub(r, ph2), pl2));
  const f2x q3 = f2_mul(r2, rc);
  f2x sh, sl;
  f2_fast_two_sum(q1, q2, sh, sl);
  f2_fast_two_sum(sh, f2_add(sl, q3), h, l);
}

// 2^e as float for e in [-252, 254] via two normal factors
__device__ __forceinline__ void pow2_pair(int e, float& s1, float& s2) {
  e = max(-252, min(254, e));
  const int e1 = e / 2, e2 = e - e1;
  s1 = __int_as_float((e1 + 127) << 23);
  s2 = __int_as_float((e2 + 127) << 23);
}

// ------------------------------------------------------------------ tile decode

struct TileInfo {
  const SplitProb* P;
  int tm, tn, k1b, k1e, nK;
  bool skip;
};

// Problem of work-queue entry t: binary search over the problems' first entries, in the
// compact array `begins` when given (a few L1 lines) or else in the descriptors.
__device__ __forceinline__ int find_problem(const SplitProb* __restrict__ probs,
                                            const long long* __restrict__ begins, int nprobs,
                                            long long t) {
  int lo = 0, hi = nprobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const long long b = begins ? begins[mid] : probs[mid].tile_begin;
    if (b <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ TileInfo decode_tile(const SplitProb* __restrict__ probs, int pi,
                                                long long t, int nt) {
  TileInfo ti;
  ti.P = probs + pi;
  const SplitProb* P = ti.P;
  const long long lt = t - P->tile_begin;
  const long long per = (long long)P->tiles_m * P->tiles_n;
  int ks;
  long long tt;
  if (P->ks_outer) { ks = (int)(lt / per); tt = lt - (long long)ks * per; }
  else { ks = (int)(lt % P->ksplit); tt = lt / P->ksplit; }
  if (P->group_m > 1) {
    // groups of group_m rows, walked column by column: the group's A rows stay in L2
    // while each column block of B is used by group_m tiles that run side by side
    const long long gsz = (long long)P->group_m * P->tiles_n;
    const int g = (int)(tt / gsz);
    const int first = g * P->group_m;
    const int gm = min(P->group_m, P->tiles_m - first);
    const int r = (int)(tt - g * gsz);
    ti.tm = first + r % gm;
    ti.tn = r / gm;
  } else {
    ti.tm = (int)(tt / P->tiles_n);
    ti.tn = (int)(tt % P->tiles_n);
  }
  ti.k1b = ks * ti.P->k1_chunk;
  ti.k1e = min(ti.P->k1_count, ti.k1b + ti.P->k1_chunk);
  ti.nK = max(0, ti.k1e - ti.k1b) * ti.P->k0_blocks;
  // V is symmetric: only tiles with some row index >= some column index are computed.
  // Their elements mostly lie below the diagonal and are stored through the mirror
  // T[n][m], where the 32 rows a warp holds are 32 consecutive addresses.
  ti.skip = (ti.P->kind == PK_V) && (ti.tm * SG_BM + SG_BM - 1 < ti.tn * nt);
  // symmetric accumulations (P_ab, P_ij): only tiles with some row <= some column
  if (ti.P->sym) ti.skip = ti.tm * SG_BM > ti.tn * nt + nt - 1;
  if (ti.skip) ti.nK = 0;
  return ti;
}

// End of the run of work-free entries that starts at the skipped entry t: for V, when t's
// column lies right of the diagonal of its whole row group (group raster) or row (row-major
// order), every later entry of that group or row is skipped too; otherwise t + 1.
__device__ __forceinline__ long long skipped_run_end(const TileInfo& ti, long long t, int nt) {
  const SplitProb* P = ti.P;
  if (P->kind != PK_V) return t + 1;
  const long long lt = t - P->tile_begin;   // V has no split-K
  if (P->group_m > 1) {
    const long long gsz = (long long)P->group_m * P->tiles_n;
    const long long g = lt / gsz;
    const int first = (int)g * P->group_m;
    const int gm = min(P->group_m, P->tiles_m - first);
    const int tn_max = ((first + gm - 1) * SG_BM + SG_BM - 1) / nt;   // last column with work
    if (ti.tn > tn_max) return P->tile_begin + g * gsz + (long long)gm * P->tiles_n;
  } else {
    const int tn_max = (ti.tm * SG_BM + SG_BM - 1) / nt;
    if (ti.tn > tn_max) return P->tile_begin + (long long)(ti.tm + 1) * P->tiles_n;
  }
  return t + 1;
}

__device__ __forceinline__ void tma_operand(uint32_t dst, const CUtensorMap* tm, uint64_t* bar,
                                            int mode, int x, int row, int k1, int div5, int slice) {
  if (mode == TM_3D) tma_3d(dst, tm, bar, x, row, slice);
  else if (mode == TM_3DK) tma_3d(dst, tm, bar, k1 * div5 + x, row, slice);
  else if (mode == TM_4D) tma_4d(dst, tm, bar, x, row, k1, slice);
  else tma_5d(dst, tm, bar, x, k1 / div5, k1 % div5, row, slice);
}

// ------------------------------------------------------------------ the kernel

// F8 = false: BF16 digits (9 bits each, kind::f16); true: FP8 e4m3 digits (5 bits each,
// kind::f8f6f4).  Both consume 32 bytes of K per MMA, so the tile geometry in bytes is
// the same: ROWB bytes of K per row and pipeline stage.
template <int NT, int ROWB, bool F8, int EPI>
__global__ void __launch_bounds__((2 + EPI) * 32, 1)
k_split_gemm(const SplitProb* __restrict__ probs, const long long* __restrict__ begins, int nprobs,
             long long total, Bases bs, unsigned* __restrict__ counter, int slices, int stages) {
  constexpr int NC = NT / (EPI / 4);         // columns per epilogue thread
  // two register buffers in the drain where the registers allow it (168 a thread with
  // 8 epilogue warps, 96 with 16)
  constexpr bool kDoubleBuf = EPI == 8 ? NC <= 24 : NC <= 12;
  constexpr uint32_t A_TILE = SG_BM * ROWB;  // bytes of one 128-row tile
  constexpr uint32_t B_TILE = NT * ROWB;
  constexpr int BKE = F8 ? ROWB : ROWB / 2;  // K elements per stage
  constexpr int CHUNK_STAGES = (F8 ? SG_CHUNK_K_FP8 : SG_CHUNK_K_BF16) / BKE;
  constexpr int LB = F8 ? SG_LB_FP8 : SG_LB_BF16;   // bits per digit
  // Levels l < EXACT are folded into the (hi, lo) accumulator by error-free sums (the
  // integer levels and, for BF16, level 2, whose FP32 sums can reach 2^24); the higher
  // levels carry at most 2^-24 of the value and are added into lo by an FMA.
  constexpr int EXACT = F8 ? 5 : 3;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned base for the swizzled tiles
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t stage_bytes = (uint32_t)slices * (A_TILE + B_TILE);
  uint64_t* full = (uint64_t*)(smem + (size_t)stages * stage_bytes);
  uint64_t* empty = full + stages;
  uint64_t* tmem_full = empty + stages;      // [2]: one per accumulator set
  uint64_t* tmem_empty = tmem_full + 2;      // [2]
  uint64_t* tile_full = tmem_empty + 2;      // [2]
  uint64_t* tile_empty = tile_full + 2;      // [2]
  uint64_t* mma_drain = tile_empty + 2;      // [1]: MMAs in flight at an abort
  long long* tile_idx = (long long*)(mma_drain + 1);   // [2]
  int* tile_prob = (int*)(tile_idx + 2);               // [2]: problem of the entry (producer)
  uint32_t* tmem_base_slot = (uint32_t*)(tile_prob + 2);
  volatile int* abort_flag = (volatile int*)(tmem_base_slot + 1);
  // V epilogue: per epilogue warp, its NC columns' denominator terms and exponents, loaded
  // at the start of a tile (while the first chunk's MMAs run) instead of in the element loop
  float2* stage_dn = (float2*)(smem + (size_t)stages * stage_bytes + 256);
  int* stage_eb = (int*)(stage_dn + EPI * NC);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(tmem_full + s, 1);
      mbar_init(tmem_empty + s, EPI);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(tile_full + s, 1);
      mbar_init(tile_empty + s, 1 + EPI);
    }
    mbar_init(mma_drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_base_slot)),
                 "r"(512u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_base_slot;
  const uint64_t cwait = g_sg_consumer_wait_ns;   // consumer-side wait limit
  // Two sets of level accumulators when both fit the 512 TMEM columns: the MMAs of the
  // next K chunk (or tile) then run while the epilogue warps drain the previous one.
  // Chunk c (counted over the CTA's whole tile sequence, identically by the MMA issuer
  // and the epilogue) uses set c % nbuf; its barrier phase is (c / nbuf) & 1.
  const uint32_t set_cols = (uint32_t)(slices * NT);
  const uint32_t nbuf = 2u * set_cols <= 512u ? 2u : 1u;

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      uint32_t st = 0, ph = 0;
      int tslot = 0;
      uint32_t tph = 0;
      bool pending[8] = {false, false, false, false, false, false, false, false};
      uint32_t pend_ph[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      for (;;) {
        const long long t = (long long)atomicAdd(counter, 1u);
        // the problem search is done here once per entry; the MMA and epilogue warps take
        // its result from shared memory
        const int pi = t < total ? find_problem(probs, begins, nprobs, t) : 0;
        TileInfo ti{};
        if (t < total) {
          ti = decode_tile(probs, pi, t, NT);
          if (ti.skip) {
            // a tile without work is not handed on; where it starts a run of them (the
            // columns of a V row group right of the diagonal), the queue moves past the run
            const long long run_end = skipped_run_end(ti, t, NT);
            if (run_end > t + 1) atomicMax(counter, (unsigned)min(run_end, total));
            continue;
          }
        }
        if (!mbar_wait(tile_empty + tslot, tph ^ 1u, abort_flag)) break;
        tile_idx[tslot] = t;
        tile_prob[tslot] = pi;
        mbar_arrive(tile_full + tslot);
        tslot ^= 1;
        if (tslot == 0) tph ^= 1u;
        if (t >= total) break;
        const SplitProb* P = ti.P;
        const int rowA = ti.tm * SG_BM, rowB = ti.tn * NT;
        bool ok = true;
        for (int kk = 0; kk < ti.nK; ++kk) {
          if (!mbar_wait(empty + st, ph ^ 1u, abort_flag)) { ok = false; break; }
          pending[st] = false;
          mbar_arrive_expect_tx(full + st, stage_bytes);
          pending[st] = true;
          pend_ph[st] = ph;
          const int k1 = ti.k1b + kk / P->k0_blocks;
          const int x = (kk % P->k0_blocks) * BKE;
          const uint32_t base = smem_u32(smem + (size_t)st * stage_bytes);
          // one box per operand covers all slices (the outermost tensor dimension): slice
          // p of A lands at p * A_TILE, slice q of B at slices * A_TILE + q * B_TILE
          tma_operand(base, &P->tmA, full + st, P->a_mode, x, rowA, k1, P->div5, 0);
          tma_operand(base + slices * A_TILE, &P->tmB, full + st, P->b_mode, x, rowB, k1, P->div5,
                      0);
          if (++st == (uint32_t)stages) { st = 0; ph ^= 1u; }
        }
        if (!ok) break;
      }
      if (*abort_flag) {
        // let our own copies in flight land before the CTA leaves (bounded)
        for (int s = 0; s < stages && s < 8; ++s)
          if (pending[s]) {
            const uint64_t t0 = global_ns();
            while (!mbar_try_wait(full + s, pend_ph[s]) && global_ns() - t0 < kWaitLimitNs) { }
          }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      // kind::f16 instruction descriptor without N: F32 accumulate, BF16 A and B, both
      // K-major, M = 128; N (a multiple of NT up to 256) is or-ed in per MMA
      constexpr uint32_t kFmt = F8 ? 0u : 1u;   // E4M3 (kind::f8f6f4) or BF16 (kind::f16)
      const uint32_t idesc_m = (1u << 4) | (kFmt << 7) | (kFmt << 10) | ((uint32_t)(SG_BM >> 4) << 24);
      uint32_t st = 0, ph = 0, cc = 0;
      int tslot = 0;
      uint32_t tph = 0;
      for (;;) {
        if (!mbar_wait(tile_full + tslot, tph, abort_flag, cwait)) break;
        const long long t = tile_idx[tslot];
        const int pi = tile_prob[tslot];
        mbar_arrive(tile_empty + tslot);
        tslot ^= 1;
        if (tslot == 0) tph ^= 1u;
        if (t >= total) break;
        const TileInfo ti = decode_tile(probs, pi, t, NT);
        const int chunks = (ti.nK + CHUNK_STAGES - 1) / CHUNK_STAGES;
        bool ok = true;
        for (int c = 0; c < chunks && ok; ++c) {
          const uint32_t set = cc % nbuf, use = cc / nbuf;
          ++cc;
          const uint32_t acc = tmem_base + set * set_cols;
          if (!mbar_wait(tmem_empty + set, (use & 1u) ^ 1u, abort_flag, cwait)) { ok = false; break; }
          tc_fence_after();
          const int kend = min(ti.nK, (c + 1) * CHUNK_STAGES);
          for (int kk = c * CHUNK_STAGES; kk < kend; ++kk) {
            if (!mbar_wait(full + st, ph, abort_flag, cwait)) { ok = false; break; }
            tc_fence_after();
            const uint64_t desc = smem_desc<ROWB>(smem_u32(smem + (size_t)st * stage_bytes));
            const bool fresh = kk == c * CHUNK_STAGES;
            switch (slices) {
              case 2: mma_stage<2, NT, ROWB, F8>(acc, desc, idesc_m, fresh); break;
              case 3: mma_stage<3, NT, ROWB, F8>(acc, desc, idesc_m, fresh); break;
              case 4: mma_stage<4, NT, ROWB, F8>(acc, desc, idesc_m, fresh); break;
              case 5: mma_stage<5, NT, ROWB, F8>(acc, desc, idesc_m, fresh); break;
              case 6: mma_stage<6, NT, ROWB, F8>(acc, desc, idesc_m, fresh); break;
              case 7: mma_stage<7, NT, ROWB, F8>(acc, desc, idesc_m, fresh); break;
              case 8: mma_stage<8, NT, ROWB, F8>(acc, desc, idesc_m, fresh); break;
              case 9: mma_stage<9, NT, ROWB, F8>(acc, desc, idesc_m, fresh); break;
              case 10: mma_stage<10, NT, ROWB, F8>(acc, desc, idesc_m, fresh); break;
              case 11: mma_stage<11, NT, ROWB, F8>(acc, desc, idesc_m, fresh); break;
              case 12: mma_stage<12, NT, ROWB, F8>(acc, desc, idesc_m, fresh); break;
              case 13: mma_stage<13, NT, ROWB, F8>(acc, desc, idesc_m, fresh); break;
              case 14: mma_stage<14, NT, ROWB, F8>(acc, desc, idesc_m, fresh); break;
              case 15: mma_stage<15, NT, ROWB, F8>(acc, desc, idesc_m, fresh); break;
              case 16: mma_stage<16, NT, ROWB, F8>(acc, desc, idesc_m, fresh); break;
              default: break;   // rejected by the host (slices in 2..16, slices * NT <= 512)
            }
            umma_commit(empty + st);   // frees this smem stage once its MMAs completed
            if (++st == (uint32_t)stages) { st = 0; ph ^= 1u; }
          }
          if (ok) umma_commit(tmem_full + set);
        }
        if (!ok) break;
      }
      if (*abort_flag) {
        // MMAs issued before the abort may still read shared memory and write TMEM:
        // commit them to an mbarrier and wait (bounded by the normal limit, whatever
        // the abort flag says) before the teardown frees TMEM
        umma_commit(mma_drain);
        const uint64_t t0 = global_ns();
        while (!mbar_try_wait(mma_drain, 0) && global_ns() - t0 < kWaitLimitNs) { }
      }
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------------- epilogue
    const int ew = warp - 2;                   // 0 .. EPI - 1
    const int quad = warp & 3;                 // TMEM lane quadrant this warp may access
    const int c0 = (ew >> 2) * NC;             // first column of this thread (group ew / 4)
    const int row = quad * 32 + lane;          // row within the tile
    const uint32_t lane_addr = tmem_base + ((uint32_t)(quad * 32) << 16);
    uint32_t cc = 0;
    int tslot = 0;
    uint32_t tph = 0;
    for (;;) {
      if (!mbar_wait_warp(tile_full + tslot, tph, abort_flag, cwait)) break;
      const long long t = tile_idx[tslot];
      const int pi = tile_prob[tslot];
      __syncwarp();
      if (lane == 0) mbar_arrive(tile_empty + tslot);
      tslot ^= 1;
      if (tslot == 0) tph ^= 1u;
      if (t >= total) break;
      const TileInfo ti = decode_tile(probs, pi, t, NT);
      if (ti.skip) continue;
      float2 dm_pre = make_float2(0.f, 0.f);
      int ea_pre = 0;
      float2* const sdn = stage_dn + ew * NC;
      int* const seb = stage_eb + ew * NC;
      if (ti.P->kind == PK_V) {
        const SplitProb* P = ti.P;
        const char* wsb = (const char*)bs.ws;
        __syncwarp();   // the previous tile's reads of this warp's slice are done
        for (int c = lane; c < NC; c += 32) {
          const int n = ti.tn * NT + c0 + c;
          if (n < P->N) {
            sdn[c] = ((const float2*)(wsb + P->d_off))[n];
            seb[c] = ((const int*)(wsb + P->eb_off))[n];
          }
        }
        const int m = ti.tm * SG_BM + row;
        if (m < P->M) {
          dm_pre = ((const float2*)(wsb + P->d_off))[m];
          ea_pre = ((const int*)(wsb + P->ea_off))[m];
        }
        __syncwarp();
      }
      const int chunks = (ti.nK + CHUNK_STAGES - 1) / CHUNK_STAGES;
      // the (hi, lo) accumulators of column pairs, folded with packed f32x2 arithmetic
      f2x acc_h2[NC / 2], acc_l2[NC / 2];
#pragma unroll
      for (int c = 0; c < NC / 2; ++c) { acc_h2[c] = 0ull; acc_l2[c] = 0ull; }
      bool ok = true;
      for (int ch = 0; ch < chunks; ++ch) {
        const uint32_t set = cc % nbuf, use = cc / nbuf;
        ++cc;
        const uint32_t set_addr = lane_addr + set * set_cols;
        if (!mbar_wait_warp(tmem_full + set, use & 1u, abort_flag, cwait)) { ok = false; break; }
        tc_fence_after();
        // levels from the highest down; the set is released as soon as level 0 is in
        // registers (its fold and the renormalisation run while the next MMAs do).  Up to
        // 24 columns a thread, two register buffers: the loads of level l-1 are in flight
        // while level l is folded (wider tiles would spill)
        auto fold = [&](int l, float (&v)[NC]) {
          const float sc = __int_as_float((127 - LB * l) << 23);   // 2^(-LB l)
          const f2x sc2 = f2_pack(sc, sc);
          if (l >= EXACT) {
#pragma unroll
            for (int c = 0; c < NC / 2; ++c)
              acc_l2[c] = f2_fma(f2_pack(v[2 * c], v[2 * c + 1]), sc2, acc_l2[c]);
          } else {
#pragma unroll
            for (int c = 0; c < NC / 2; ++c) {
              f2x s2, e2;
              f2_two_sum(acc_h2[c], f2_mul(f2_pack(v[2 * c], v[2 * c + 1]), sc2), s2, e2);
              acc_h2[c] = s2;
              acc_l2[c] = f2_add(acc_l2[c], e2);
            }
          }
        };
        auto release = [&]() {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(tmem_empty + set);
        };
        if constexpr (kDoubleBuf) {
          float va[NC], vb[NC];
          tmem_ld_cols<NC>(set_addr + (uint32_t)((slices - 1) * NT + c0), va);
          for (int l = slices - 1; l >= 0; l -= 2) {
            tmem_wait_ld();
            tmem_hold<NC>(va);
            if (l >= 1) tmem_ld_cols<NC>(set_addr + (uint32_t)((l - 1) * NT + c0), vb);
            else release();
            fold(l, va);
            if (l == 0) break;
            tmem_wait_ld();
            tmem_hold<NC>(vb);
            if (l >= 2) tmem_ld_cols<NC>(set_addr + (uint32_t)((l - 2) * NT + c0), va);
            else release();
            fold(l - 1, vb);
          }
        } else {
          for (int l = slices - 1; l >= 0; --l) {
            float v[NC];
            tmem_ld_cols<NC>(set_addr + (uint32_t)(l * NT + c0), v);
            tmem_wait_ld();
            tmem_hold<NC>(v);
            if (l == 0) release();
            fold(l, v);
          }
        }
        // renormalise so that lo stays within half an ulp of hi across chunks
#pragma unroll
        for (int c = 0; c < NC / 2; ++c) {
          f2x s2, e2;
          f2_two_sum(acc_h2[c], acc_l2[c], s2, e2);
          acc_h2[c] = s2;
          acc_l2[c] = e2;
        }
      }
      if (!ok) break;
      float acc_h[NC], acc_l[NC];
#pragma unroll
      for (int c = 0; c < NC / 2; ++c) {
        f2_unpack(acc_h2[c], acc_h[2 * c], acc_h[2 * c + 1]);
        f2_unpack(acc_l2[c], acc_l[2 * c], acc_l[2 * c + 1]);
      }
      // ---------------- problem epilogue (registers only; TMEM already released)
      const SplitProb* P = ti.P;
      const int m = ti.tm * SG_BM + row;
      unsigned emax = 0;
      if (m < P->M) {
        const int nbase = ti.tn * NT + c0;
        const char* wsb = (const char*)bs.ws;
        const int* EA = (const int*)(wsb + P->ea_off);
        const int* EB = (const int*)(wsb + P->eb_off);
        const int ea = (P->kind == PK_V ? ea_pre : (P->ea_rows ? EA[m] : EA[0])) + P->ea_add;
        if (P->kind == PK_V) {
          float* Th = (float*)(wsb + P->c_off);
          float* Tl = (float*)(wsb + P->c2_off);
          const float2 dm = dm_pre;
          const int im = m / P->v;
          // pair block of column n, advanced as n grows (no division per element)
          int jn = nbase / P->v, jn_end = (jn + 1) * P->v;
          const f2x dmh = f2_pack(dm.x, dm.x), dml = f2_pack(dm.y, dm.y);
          if constexpr (NC > 24) {   // wide tiles: scalar (the packed form would spill)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
              const int n = nbase + c;
              if (n >= P->N) continue;
              while (n >= jn_end) { ++jn; jn_end += P->v; }
              float s1, s2;
              pow2_pair(ea + seb[c] + P->eb_add - 2 * LB, s1, s2);   // V: one exponent per row
              df V = {(acc_h[c] * s1) * s2, (acc_l[c] * s1) * s2};
              if (n == m) {   // diagonal: the FP64 row sum of squares (see k_slice_b1)
                const float2 w = ((const float2*)(wsb + P->vd_off))[m];
                V = {w.x, w.y};
              }
              const float2 dn = sdn[c];
              const df D = df_add({dm.x, dm.y}, {dn.x, dn.y});
              const df T = df_div(V, D);
              if (im <= jn) {
                const long long ix = (long long)m * P->ldc + n + (long long)jn * (P->vpad - P->v);
                Th[ix] = T.h;
                Tl[ix] = T.l;
              }
              if (jn <= im) {
                const long long ix = (long long)n * P->ldc + m + (long long)im * (P->vpad - P->v);
                Th[ix] = T.h;
                Tl[ix] = T.l;
              }
              emax = max(emax, (__float_as_uint(T.h) >> 23) & 0xFFu);
            }
          } else {
            // column pairs in packed f32x2 arithmetic (columns past N are computed from
            // unused staging entries and not stored)
  #pragma unroll
            for (int k = 0; k < NC / 2; ++k) {
              float s1a, s2a, s1b, s2b;   // V: one exponent per row and per column
              pow2_pair(ea + seb[2 * k] + P->eb_add - 2 * LB, s1a, s2a);
              pow2_pair(ea + seb[2 * k + 1] + P->eb_add - 2 * LB, s1b, s2b);
              const f2x s1 = f2_pack(s1a, s1b), s2 = f2_pack(s2a, s2b);
              f2x Vh = f2_mul(f2_mul(acc_h2[k], s1), s2), Vl = f2_mul(f2_mul(acc_l2[k], s1), s2);
              const int n0 = nbase + 2 * k;
              if (n0 == m || n0 + 1 == m) {   // diagonal: the FP64 row sum of squares (see k_slice_b1)
                const float2 w = ((const float2*)(wsb + P->vd_off))[m];
                float h0, h1, l0, l1;
                f2_unpack(Vh, h0, h1);
                f2_unpack(Vl, l0, l1);
                if (n0 == m) { h0 = w.x; l0 = w.y; } else { h1 = w.x; l1 = w.y; }
                Vh = f2_pack(h0, h1);
                Vl = f2_pack(l0, l1);
              }
              const float2 dna = sdn[2 * k], dnb = sdn[2 * k + 1];
              f2x Dh, Dl, Th2, Tl2;
              df_add2(dmh, dml, f2_pack(dna.x, dnb.x), f2_pack(dna.y, dnb.y), Dh, Dl);
              df_div2(Vh, Vl, Dh, Dl, Th2, Tl2);
              df Tc[2];
              f2_unpack(Th2, Tc[0].h, Tc[1].h);
              f2_unpack(Tl2, Tc[0].l, Tc[1].l);
  #pragma unroll
              for (int u = 0; u < 2; ++u) {
                const int n = n0 + u;
                if (n >= P->N) continue;
                while (n >= jn_end) { ++jn; jn_end += P->v; }
                const df T = Tc[u];
                // the amplitude stage reads the pair blocks i <= j only: store (m, n) where
                // i(m) <= i(n) and the mirror (n, m) where i(n) <= i(m)
                if (im <= jn) {
                  const long long ix = (long long)m * P->ldc + n + (long long)jn * (P->vpad - P->v);
                  Th[ix] = T.h;
                  Tl[ix] = T.l;
                }
                if (jn <= im) {
                  const long long ix = (long long)n * P->ldc + m + (long long)im * (P->vpad - P->v);
                  Th[ix] = T.h;
                  Tl[ix] = T.l;
                }
                emax = max(emax, (__float_as_uint(T.h) >> 23) & 0xFFu);
              }
            }
          }
        } else {
          double* C = (P->kind == PK_GAMMA || P->kind == PK_RAW) ? bs.gamma
                      : P->kind == PK_PAB ? bs.pab : bs.pij;
          C += P->c_off;
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            const int n = nbase + c;
            if (n >= P->N) continue;
            const int e = ea + (P->eb_rows ? EB[n] : EB[0]) + P->eb_add - 2 * LB;
            const double val = ldexp((double)acc_h[c] + (double)acc_l[c], e);
            if ((P->kind == PK_GAMMA || P->kind == PK_RAW) && P->ksplit == 1) {
              C[(long long)m * P->ldc + n] = P->alpha * val;
            } else if (P->sym) {
              // each unordered pair once: (m,n) and its mirror for m < n, the diagonal once;
              // m > n is covered by the mirror of a computed tile
              if (m > n) continue;
              atomicAdd(C + (long long)m * P->ldc + n, P->alpha * val);
              if (m < n) atomicAdd(C + (long long)n * P->ldc + m, P->alpha * val);
            } else {
              atomicAdd(C + (long long)m * P->ldc + n, P->alpha * val);
            }
          }
        }
      }
      if (P->kind == PK_V) {   // uniform across the warp
        emax = __reduce_max_sync(0xffffffffu, emax);
        if (lane == 0 && emax) atomicMax((unsigned*)((char*)bs.ws + P->et_off), emax);
      }
    }
  }

  // ---------------------------------------------------------------- teardown
  tc_fence_before();
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) atomicOr(bs.status, ST_TIMEOUT);
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(512u)
                 : "memory");
  }
}

// ------------------------------------------------------------------ host side

SplitLaunch split_launch_config(int slices, int bk, int n_tile, bool fp8) {
  SplitLaunch c{};
  c.slices = slices;
  c.fp8 = fp8;
  if (fp8) {
    c.bk = 64;                       // 64 one-byte elements per 64-byte row
    c.n_tile_max = (n_tile == 32 || n_tile == 48 || n_tile == 64) && slices * n_tile <= 512
                       ? n_tile : (slices <= 8 ? 64 : (slices <= 10 ? 48 : 32));
  } else {
    c.bk = bk == 16 ? 16 : 32;
    // 64 columns when no width is asked for: with 5 or 6 slices a stage is then small
    // enough for three stages in shared memory.  (The plan asks per launch: 48 for V,
    // whose two accumulator sets then fit TMEM, 80 for Gamma, 64 for P_ab / P_ij.)
    const int widest = slices <= 5 ? 96 : (slices == 6 ? 80 : 64);
    c.n_tile_max = (n_tile == 48 || n_tile == 64 || n_tile == 80 || n_tile == 96)
                       ? std::min(n_tile, widest) : 64;
  }
  const size_t rowb = fp8 ? 64 : (size_t)c.bk * 2;
  const size_t stage = (size_t)slices * (SG_BM + c.n_tile_max) * rowb;
  // the V epilogue's staging area: per epilogue warp, its columns x 12 bytes
  // (8 warps x n_tile / 2 columns, or 16 x n_tile / 4)
  const size_t stage_area = (size_t)4 * c.n_tile_max * 12;
  const size_t budget = 227 * 1024 - 1024 - 256 - stage_area;
  int st = (int)(budget / stage);
  if (st > 8) st = 8;
  if (st < 1) st = 1;
  c.stages = st;
  c.smem = 1024 + (size_t)st * stage + 256 + stage_area;
  c.epi_warps = 8;
  return c;
}

// 16 epilogue warps are built for the 32-wide K stages only (the shapes small fragments
// use); other shapes run with 8
template <int NT, int ROWB, bool F8>
static cudaError_t launch_nt(const SplitProb* d_probs, const long long* d_begins, int nprobs,
                             long long total, Bases bs, unsigned* counter, const SplitLaunch& cfg,
                             int grid, cudaStream_t s) {
  if constexpr (ROWB == 64) {
    if (cfg.epi_warps == 16) {
      k_split_gemm<NT, ROWB, F8, 16><<<grid, (2 + 16) * 32, cfg.smem, s>>>(
          d_probs, d_begins, nprobs, total, bs, counter, cfg.slices, cfg.stages);
      return cudaGetLastError();
    }
  }
  k_split_gemm<NT, ROWB, F8, 8><<<grid, (2 + 8) * 32, cfg.smem, s>>>(
      d_probs, d_begins, nprobs, total, bs, counter, cfg.slices, cfg.stages);
  return cudaGetLastError();
}

// Opt in to the large dynamic shared memory once per device, outside any capture.
cudaError_t split_gemm_prepare() {
  const int bytes = 227 * 1024;
  cudaError_t e = cudaSuccess;
#define RIMP2_PREP(NT, ROWB, F8, EPI)                                                       \
  if (e == cudaSuccess)                                                                      \
    e = cudaFuncSetAttribute(k_split_gemm<NT, ROWB, F8, EPI>,                                \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  RIMP2_PREP(96, 64, false, 8) RIMP2_PREP(80, 64, false, 8) RIMP2_PREP(64, 64, false, 8)
  RIMP2_PREP(48, 64, false, 8)
  RIMP2_PREP(96, 32, false, 8) RIMP2_PREP(80, 32, false, 8) RIMP2_PREP(64, 32, false, 8)
  RIMP2_PREP(48, 32, false, 8)
  RIMP2_PREP(64, 64, true, 8) RIMP2_PREP(48, 64, true, 8) RIMP2_PREP(32, 64, true, 8)
  RIMP2_PREP(96, 64, false, 16) RIMP2_PREP(80, 64, false, 16) RIMP2_PREP(64, 64, false, 16)
  RIMP2_PREP(48, 64, false, 16)
  RIMP2_PREP(64, 64, true, 16) RIMP2_PREP(48, 64, true, 16) RIMP2_PREP(32, 64, true, 16)
#undef RIMP2_PREP
  return e;
}

cudaError_t launch_split_gemm(const SplitProb* d_probs, const long long* d_begins, int nprobs,
                              long long total_tiles, Bases bs, unsigned* counter,
                              const SplitLaunch& cfg, int grid, cudaStream_t s) {
  if (total_tiles <= 0) return cudaSuccess;
  const int g = (int)(total_tiles < grid ? total_tiles : grid);
  if (cfg.fp8) {
    if (cfg.n_tile_max == 64) return launch_nt<64, 64, true>(d_probs, d_begins, nprobs, total_tiles, bs, counter, cfg, g, s);
    if (cfg.n_tile_max == 48) return launch_nt<48, 64, true>(d_probs, d_begins, nprobs, total_tiles, bs, counter, cfg, g, s);
    return launch_nt<32, 64, true>(d_probs, d_begins, nprobs, total_tiles, bs, counter, cfg, g, s);
  }
  if (cfg.bk == 32) {
    switch (cfg.n_tile_max) {
      case 96: return launch_nt<96, 64, false>(d_probs, d_begins, nprobs, total_tiles, bs, counter, cfg, g, s);
      case 80: return launch_nt<80, 64, false>(d_probs, d_begins, nprobs, total_tiles, bs, counter, cfg, g, s);
      case 48: return launch_nt<48, 64, false>(d_probs, d_begins, nprobs, total_tiles, bs, counter, cfg, g, s);
      default: return launch_nt<64, 64, false>(d_probs, d_begins, nprobs, total_tiles, bs, counter, cfg, g, s);
    }
  }
  switch (cfg.n_tile_max) {
    case 96: return launch_nt<96, 32, false>(d_probs, d_begins, nprobs, total_tiles, bs, counter, cfg, g, s);
    case 80: return launch_nt<80, 32, false>(d_probs, d_begins, nprobs, total_tiles, bs, counter, cfg, g, s);
    case 48: return launch_nt<48, 32, false>(d_probs, d_begins, nprobs, total_tiles, bs, counter, cfg, g, s);
    default: return launch_nt<64, 32, false>(d_probs, d_begins, nprobs, total_tiles, bs, counter, cfg, g, s);
  }
}

cudaError_t split_gemm_set_consumer_wait(long long ns) {
  const unsigned long long v = ns < 0 ? kWaitLimitNs : (unsigned long long)ns;
  return cudaMemcpyToSymbol(g_sg_consumer_wait_ns, &v, sizeof(v));
}

int split_gemm_grid() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;  // one persistent CTA per SM (TMEM 512 columns and ~210 KB smem each)
}

int encode_tmap(CUtensorMap* tm, const void* base, int rank, const uint64_t* dims,
                const uint64_t* strides_bytes, const uint32_t* box, int elem_bytes) {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
      return RIMP2_ERR_CUDA;
    fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  cuuint64_t d[5], s[4];
  cuuint32_t b[5], es[5];
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    b[i] = box[i];
    es[i] = 1;
    if (i > 0) s[i - 1] = strides_bytes[i - 1];
  }
  const unsigned row_bytes = box[0] * (unsigned)elem_bytes;
  if ((elem_bytes != 1 && elem_bytes != 2) || (row_bytes != 32 && row_bytes != 64))
    return RIMP2_ERR_UNSUPPORTED;
  const CUtensorMapSwizzle sw = row_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B;
  const CUtensorMapDataType dt =
      elem_bytes == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const CUresult r = fn(tm, dt, (cuuint32_t)rank, const_cast<void*>(base),
                        d, s, b, es, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? RIMP2_OK : RIMP2_ERR_UNSUPPORTED;
}

}  // namespace rimp2
