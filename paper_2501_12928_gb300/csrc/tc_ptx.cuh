// Inline-PTX wrappers of the tcgen05 tensor-core kernels (sm_103a): mbarrier
// waits bounded by %globaltimer, TMA tensor loads, tcgen05.mma / commit /
// ld, the shared-memory and instruction descriptors, and the double-float
// sum of the four slice-product level accumulators.
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "beor_common.cuh"

namespace beor {

// limit of a CTA's wait for the copies and tensor-core work it issued itself
constexpr unsigned long long TC_DRAIN_NS = 2000000000ull;

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait of one role on another: false when `limit_ns` passed or
// another role aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, volatile int* abort_flag,
                                          unsigned long long limit_ns) {
  if (mbar_try(a, parity)) return true;
  const unsigned long long t0 = globaltimer();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try(a, parity)) return true;
    if ((it & 255u) == 255u) {
      if (*abort_flag) return false;
      if (globaltimer() - t0 > limit_ns) return false;
    }
  }
}
// Wait bounded by the deadline only (used to drain work this CTA issued).
__device__ __forceinline__ bool mbar_wait_deadline(uint32_t a, uint32_t parity) {
  const unsigned long long t0 = globaltimer();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try(a, parity)) return true;
    if ((it & 255u) == 255u && globaltimer() - t0 > TC_DRAIN_NS) return false;
  }
}
__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, int w,
                                            int u, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(u), "r"(mbar)
      : "memory");
}
// Bulk prefetch of a contiguous global range into L2 (size a multiple of 16 bytes).
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(reinterpret_cast<uint64_t>(p)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void prefetch_map(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float* v) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld2(uint32_t taddr, float* v) {
  uint32_t r[2];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(taddr));
  v[0] = __uint_as_float(r[0]);
  v[1] = __uint_as_float(r[1]);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// Pins four registers written by tcgen05.ld after the wait that completes the
// load, so that no use of them is scheduled before it.
__device__ __forceinline__ void reg_fence2(float* v) { asm volatile("" : "+f"(v[0]), "+f"(v[1])); }
__device__ __forceinline__ void reg_fence4(float* v) {
  asm volatile("" : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]));
}

// Shared-memory matrix descriptor: K-major operand without swizzle, made of
// 8-row x 16-byte core matrices: the two core matrices of one MMA's K = 16
// are 128 bytes apart (leading byte offset), 8-row groups 256 bytes apart
// (stride byte offset).  Every address it yields lies within 256 x (rows / 8)
// bytes of the start.
__device__ __forceinline__ uint64_t sdesc_kmajor(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);            // start address
  d |= (uint64_t)(128 >> 4) << 16;                      // leading byte offset: next K core matrix
  d |= (uint64_t)(256 >> 4) << 32;                      // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                               // descriptor version (sm_100 family)
  return d;                                             // swizzle mode 0: none
}
// The descriptor of an operand `bytes` further on: shared-memory addresses
// lie below 256 KB, so the 14-bit start-address field never carries.
__device__ __forceinline__ uint64_t sdesc_add(uint64_t d, uint32_t bytes) { return d + (uint64_t)(bytes >> 4); }
// Instruction descriptor: bf16 x bf16 -> fp32, K-major A and B, M = 128, N given.
__host__ __device__ constexpr uint32_t idesc_bf16(uint32_t negate_a, uint32_t n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (negate_a << 13) | ((n >> 3) << 17) |
         ((uint32_t)(128 >> 4) << 24);
}

// Sum of the four level accumulators as a double-float number.  Levels 0-2
// hold exact fp32 values (integers times 2^0, 2^-8, 2^-16 units), level 3 is
// rounded and about 2^-24 below level 0: two exact two-sums, then the small
// terms into the low part.
__device__ __forceinline__ dfl levels_sum(float l0, float l1, float l2, float l3) {
  const dfl a = df_two_sum(l0, l1);
  const dfl b = df_two_sum(a.hi, l2);
  return df_fast_two_sum(b.hi, b.lo + (a.lo + l3));
}
// The same sum in 10 operations, as an unnormalised double-float (hi, lo),
// for the accumulator drain, where every operation holds the tensor core
// idle (the normalisation below runs after tensor memory is released): levels 1 and 2 are split exactly into nearest integer and fraction
// (adding and subtracting 1.5 * 2^23 rounds to the nearest integer for
// |x| < 2^22; |l1| < 2^15, |l2| < 2^8); hi = l0 + int(l1) + int(l2) is an
// exact integer below 2^23, frac(l1) + frac(l2) is exact (multiples of 2^-16,
// |.| <= 1), and lo adds the rounded level 3 (|l3| < 2), so |lo| < 4.
// df_fast_two_sum(hi, lo) then normalises it exactly: for |hi| >= 4 the
// exponent of hi is the larger, for hi = 0 it is trivial, and for an
// integer |hi| <= 3 both s - hi and lo - (s - hi) are representable.
__device__ __forceinline__ dfl levels_sum_split(float l0, float l1, float l2, float l3) {
  const float m = 12582912.0f;   // 1.5 * 2^23
  const float r1 = __fsub_rn(__fadd_rn(l1, m), m);
  const float r2 = __fsub_rn(__fadd_rn(l2, m), m);
  const float hi = __fadd_rn(__fadd_rn(l0, r1), r2);
  const float lo = __fadd_rn(__fadd_rn(__fsub_rn(l1, r1), __fsub_rn(l2, r2)), l3);
  return {hi, lo};
}
// a - b for double-float numbers with |a.lo|, |b.lo| below half an ulp of
// their high parts: one exact two-sum of the high parts, the low parts added
// in fp32 (relative error ~2^-44), renormalised.
__device__ __forceinline__ dfl df_sub_quick(dfl a, dfl b) {
  const dfl s = df_two_sum(a.hi, -b.hi);
  return df_fast_two_sum(s.hi, s.lo + (a.lo - b.lo));
}

}  // namespace beor
