// Mixed-precision tile kernels of the batched Cholesky (sm_103a).
//
// The trailing update A_ij -= L_ik L_jk^H and the panel product
// L_ik = A_ik Linv_kk^H are complex GEMMs with K = 128.  They run on the
// tcgen05 tensor cores as *exact* bf16 slice products (an Ozaki-style
// splitting): every operand row r is scaled by 2^(7 - e_r) and cut into five
// balanced base-256 digits sigma_s (|sigma_s| <= 128), stored as bf16 values
// sigma_s * 2^(-8 s).  A product of two slices is exact in fp32, and a sum of
// 256 of them (one 128-complex block column, real and imaginary parts) stays
// below 2^24 units, so the fp32 accumulator of the tensor core is exact for
// the level-0 pair (0,0), the level-1 pairs (0,1), (1,0) and the level-2
// pairs (0,2), (1,1), (2,0) (at most 1.26e7 units of 2^-16).  All pairs with
// s + t >= 3 share a fourth accumulator whose rounding error (about 2^-19 of
// its size after ~1500 fp32 additions) lies about 2^-39 below the leading
// term.  The off-diagonal tiles of the trailing update take the reduced pair
// set (s + t <= 3 and (2, 2): the pairs dropped lie 2^-32 below the leading
// term and have no sign bias there); its diagonal tiles and the panel
// product take all pairs with s + t <= 4.  The epilogue adds the four
// levels as a double-float number,
// scales by 2^(e_r + e_c - 14) and updates the working matrix, itself kept as
// a double-float pair per real number.  The result is accurate to about
// 2^-40 of the operand row scales, which keeps log|Sigma| well inside the
// likelihood tolerance for Sigma as ill-conditioned as the eta / foreground
// degeneracy makes it (a float32-accumulated product does not).
//
// Kernel structure (one CTA per SM, persistent over output tiles of 128 rows
// x 64 complex columns).  The accumulators of a tile are four levels, each a
// [re | im] pair of 64 fp32 columns (level l at TMEM columns 128 l .. 128 l +
// 127, all 512 columns).  The complex product C += A B^H is computed as real
// products of one A part with a two-part window of B: Im A times the window
// (Im B, Re B) adds (Ai Bi, Ai Br) to (re, im), and Re A times (Re B, -Im B)
// adds (Ar Br, -Ar Bi), so one MMA covers the real and imaginary outputs of
// up to two levels (N up to 256): 11 MMAs per A part and K-chunk for the
// full pair set (7 for the reduced one) instead of 18 with separate re / im
// accumulators, which cuts the tensor cores' reads of A from shared memory
// by 40 %.  The slice planes hold the parts
// (Im, Re, -Im) of each slice for that reason.  Warp 0 issues TMA loads into
// a shared-memory ring of half-stages (one A part of 128 rows and its B
// window of 64 rows, one K-chunk of 16), fetched from the planes stored in
// the tensor cores' no-swizzle order as 512-byte rows: slices 0..3 in slots
// of 32 KB (7 of them) for the trailing update's off-diagonal tiles, all five
// slices in slots of 40 KB (5 of them) for its diagonal tiles and the panel
// product;
// warp 1 issues the tcgen05.mma instructions (M = 128, N = 128 or 256,
// K = 16, bf16 -> fp32); warps 2-9 (two per TMEM lane quarter, each with half
// the columns) drain TMEM and apply the update.  Every wait is bounded by a
// %globaltimer deadline; on expiry the kernel records an error code, drains
// what it issued and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <utility>
#include <vector>

#include "beor_common.cuh"
#include "beor_internal.h"
#include "tc_ptx.cuh"

namespace beor {

constexpr int MX_M = 128;                // output rows per tile
constexpr int MX_N = 64;                 // output complex columns per tile
constexpr int MX_KC = 16;                // complex K per pipeline stage
constexpr int MX_SLICE_A = MX_M * MX_KC * 2;                      // 4096: one slice of the A part
constexpr int MX_SLICE_B = 2 * MX_N * MX_KC * 2;                  // 4096: one slice of the B window
// Kernel modes: the trailing update's off-diagonal tiles (reduced pair set,
// slices 0..3), its diagonal tiles (full set) and the panel product (full
// set).  The diagonal tiles have a launch of their own so that the
// off-diagonal kernel, which does nearly all the work, carries no second
// product schedule: with one in the same loop its tensor-core products
// issued about a fifth slower.
enum { MODE_TRAIL = 0, MODE_PANEL = 1, MODE_TRAIL_DIAG = 2 };
// Operand ring per mode: slots of one half-stage (A part, then its B
// window), slices 0..3 (32 KB, 7 slots) for the reduced set, all five
// slices (40 KB, 5 slots) for the full one.
template <int MODE>
struct Ring {
  static constexpr int nslice = MODE == MODE_TRAIL ? 4 : BEOR_NSLICE;
  static constexpr int a_bytes = nslice * MX_SLICE_A;
  static constexpr int slot = nslice * (MX_SLICE_A + MX_SLICE_B);
  static constexpr int slots = MODE == MODE_TRAIL ? 7 : 5;
  static constexpr int smem = slots * slot + 1024 + 320;   // 230720 (reduced set), 206144 (full set)
  static constexpr int set = MODE == MODE_TRAIL ? SLICE_PAIRS_REDUCED : SLICE_PAIRS_FULL5;
};
constexpr int MX_EPI_WARPS = 8;        // two warps per TMEM lane quarter, each draining half the columns
constexpr int MX_THREADS = 64 + 32 * MX_EPI_WARPS;
constexpr uint32_t MX_TMEM_COLS = 512;
constexpr unsigned long long MX_TIMEOUT_NS = TC_DRAIN_NS;   // default role-wait limit

// Tiles of block step k.  Trailing update: the next block column (j = k + 1),
// the rest (j >= k + 2), or all (j >= k + 1), each as its off-diagonal tiles
// (i > j) and its diagonal tiles (i = j); panel product: i >= k + 1, j = k.
enum { KIND_COL = 0, KIND_REST = 1, KIND_PANEL = 2, KIND_ALL = 3, KIND_DCOL = 4, KIND_DREST = 5, KIND_DALL = 6,
       KIND_COUNT = 7 };
constexpr int MX_JOBS = 4;               // depth of the producer -> MMA / epilogue job ring
enum { ERR_TMA_WAIT = 11, ERR_MMA_WAIT = 12, ERR_ACC_WAIT = 13, ERR_EPI_WAIT = 14 };

struct MixedMaps {
  CUtensorMap panel_a[2];   // panel slices (two buffers by step parity), box: 128 rows x one K-chunk x 1 part x 5 slices
  CUtensorMap panel_b[2];   // the same, box 64 rows x 2 parts
  CUtensorMap linv_b;       // inverse-diagonal slices, box 64 rows x 2 parts
  CUtensorMap panel_a4[2];  // as panel_a / panel_b, slices 0..3 only (off-diagonal trailing tiles)
  CUtensorMap panel_b4[2];
  int64_t* d_prefix = nullptr;   // [KIND_COUNT][max_nt][P+1] tile prefix sums
  int* d_counter = nullptr;      // [KIND_COUNT][max_nt] dynamic tile counters, zeroed before every evaluation
  int max_nt = 0, P = 0;
  std::vector<int64_t> h_total[KIND_COUNT];
};

// ---------------------------------------------------------------------------
// tile decoding
// ---------------------------------------------------------------------------
struct TileJob {
  int p, i, j, h;   // problem (-1: no more work), output block row, block column, column sub-tile
};

__device__ __forceinline__ void tri_pair(int64_t u, int& a, int& b) {
  a = (int)((sqrtf(8.0f * (float)u + 1.0f) - 1.0f) * 0.5f);
  while ((int64_t)a * (a + 1) / 2 > u) --a;
  while ((int64_t)(a + 1) * (a + 2) / 2 <= u) ++a;
  b = (int)(u - (int64_t)a * (a + 1) / 2);
}

// Tile t of block step k (kind: next column, rest, or panel); valid = false
// for problems that failed earlier.
__device__ __forceinline__ bool decode_tile(const BatchView& v, const int64_t* prefix, int64_t t, int k, int kind,
                                            TileJob& jb) {
  int lo = 0, hi = v.P;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= t) lo = mid; else hi = mid;
  }
  const int p = lo;
  int64_t u = t - prefix[p];
  if (prob_skipped(v.status[p])) return false;
  k -= v.prob[p].k_off;   // this problem's block step
  jb.p = p;
  jb.h = (int)(u % (BEOR_TB / MX_N));
  u /= (BEOR_TB / MX_N);
  if (kind == KIND_REST || kind == KIND_ALL) {   // i > j >= j0
    const int j0 = kind == KIND_REST ? k + 2 : k + 1;
    int a, b;
    tri_pair(u, a, b);
    jb.i = j0 + a + 1;
    jb.j = j0 + b;
  } else if (kind == KIND_COL) {                 // i >= k + 2, j = k + 1
    jb.i = k + 2 + (int)u;
    jb.j = k + 1;
  } else if (kind == KIND_PANEL) {               // i >= k + 1, j = k
    jb.i = k + 1 + (int)u;
    jb.j = k;
  } else {                                       // diagonal: i = j >= j0
    const int j0 = kind == KIND_DREST ? k + 2 : k + 1;
    jb.i = jb.j = j0 + (int)u;
  }
  return jb.i < v.prob[p].nt;
}

// ---------------------------------------------------------------------------
// the slice GEMM
// ---------------------------------------------------------------------------
// Products of one half-stage: every A slice with its B window (schedule
// slice_mma_*, full or reduced pair set); ad, bd describe slice 0 of the A
// part and of the B window.  The first two products of a tile (K-chunk 0,
// part Im, slice 0) cover all 512 columns and overwrite them.
template <int SET>
__device__ __forceinline__ void issue_half_stage(uint32_t tmem, uint64_t ad, uint64_t bd, bool first) {
#pragma unroll
  for (int sa = 0; sa < BEOR_NSLICE; ++sa) {
#pragma unroll
    for (int q = 0; q < slice_mma_count(sa, SET); ++q) {
      const uint32_t acc = (first && sa == 0 && q < slice_mma_main(0)) ? 0u : 1u;
      tc_mma(tmem + (uint32_t)slice_mma_col(sa, q), sdesc_add(ad, sa * MX_SLICE_A),
             sdesc_add(bd, slice_mma_t(sa, q, SET) * MX_SLICE_B), idesc_bf16(0, (uint32_t)slice_mma_n(sa, q)), acc);
    }
  }
}

// map_a / map_b: the A and B boxes of one half-stage (Ring<MODE>::nslice
// slices).
template <int MODE>
__global__ void __launch_bounds__(MX_THREADS, 1)
    slice_gemm_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                      BatchView v, const int64_t* __restrict__ prefix, int64_t ntiles, int k, int kind,
                      int* __restrict__ counter, const int32_t* __restrict__ pexp) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  constexpr int SLOTS = Ring<MODE>::slots, SLOT = Ring<MODE>::slot, ABYTES = Ring<MODE>::a_bytes;
  constexpr bool TRAILING = MODE != MODE_PANEL;   // subtract from the working matrix (else store)
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + SLOTS * SLOT);
  // bars [0, SLOTS) full, [SLOTS, 2 SLOTS) empty, then acc_full, acc_empty,
  // drain, job_full[MX_JOBS], job_empty[MX_JOBS]; then the TMEM address, the
  // abort flag and the job ring (320 bytes in all)
  constexpr int NB = 2 * SLOTS + 3 + 2 * MX_JOBS;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + NB);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + NB + 1);
  TileJob* jobs = reinterpret_cast<TileJob*>(bars + NB + 2);   // MX_JOBS slots
  static_assert((NB + 2) * 8 + MX_JOBS * sizeof(TileJob) <= 320, "barrier area");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned long long wait_ns = v.wait_ns ? v.wait_ns : MX_TIMEOUT_NS;
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (SLOTS + s); };
  const uint32_t acc_full = bar0 + 8u * (2 * SLOTS), acc_empty = acc_full + 8u, drain = acc_full + 16u;
  auto job_full = [&](uint32_t q) { return bar0 + 8u * (2 * SLOTS + 3 + q); };
  auto job_empty = [&](uint32_t q) { return bar0 + 8u * (2 * SLOTS + 3 + MX_JOBS + q); };

  // After a bounded wait gave up anywhere in this evaluation, the remaining
  // launches return at once (read by one thread, so the whole CTA agrees)
  // instead of each running into its own deadline.
  {
    __shared__ int s_err;
    if (threadIdx.x == 0) s_err = *reinterpret_cast<volatile int*>(&v.flags->error);
    __syncthreads();
    if (s_err) return;
  }

  if (threadIdx.x == 0) {
    for (int s = 0; s < SLOTS; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, 32 * MX_EPI_WARPS);
    mbar_init(drain, 1);
    for (int q = 0; q < MX_JOBS; ++q) {
      mbar_init(job_full(q), 1);
      mbar_init(job_empty(q), 1 + MX_EPI_WARPS);   // the MMA thread and one lane per epilogue warp
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    prefetch_map(&map_a);
    prefetch_map(&map_b);
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                 "r"(MX_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    // Tiles are taken from a global counter (CTAs that start late, e.g. after
    // a concurrent kernel released their SM, simply take fewer) and published
    // to the MMA and epilogue warps through a ring of MX_JOBS slots.
    if (lane == 0) {
      uint32_t it = 0;           // half-stages issued
      uint32_t ps = 0, pph = 0;  // ring slot and phase of half-stage it
      uint32_t withheld = ~0u;   // half-stage whose copy the test switch withheld (never waited for)
      for (uint32_t n = 0;; ++n) {
        const uint32_t q = n % MX_JOBS;
        if (!mbar_wait(job_empty(q), ((n / MX_JOBS) & 1) ^ 1, abort_flag, wait_ns)) {
          atomicCAS(&v.flags->error, 0, ERR_TMA_WAIT);
          *abort_flag = 1;
          goto producer_done;
        }
        TileJob jb{-1, 0, 0, 0};
        for (;;) {
          const int64_t t = atomicAdd(counter, 1);
          if (t >= ntiles) break;
          if (decode_tile(v, prefix, t, k, kind, jb)) break;
          jb.p = -1;
        }
        jobs[q] = jb;
        mbar_arrive(job_full(q));
        if (jb.p < 0) break;
        const Prob pr = v.prob[jb.p];
        const int a_row = (int)(pr.row_off + (int64_t)jb.i * BEOR_TB);
        const int b_row = TRAILING ? (int)(pr.row_off + (int64_t)jb.j * BEOR_TB + jb.h * MX_N)
                                   : jb.p * BEOR_TB + jb.h * MX_N;
        BEOR_INBOUNDS(v.flags, a_row >= 0 && a_row + MX_M <= v.rows, BC_TMA_A);
        BEOR_INBOUNDS(v.flags, b_row >= 0 && b_row + MX_N <= (TRAILING ? v.rows : (int64_t)v.P * BEOR_TB),
                      BC_TMA_B);
        if (TRAILING) {
          // the epilogue will read this tile's 64 working-matrix columns (128 KB, contiguous)
          const float4* ct = reinterpret_cast<const float4*>(v.ws) + pr.ws_off +
                             tri_index(jb.i, jb.j) * BEOR_TILE_ELEMS + (int64_t)(jb.h * MX_N) * BEOR_TB;
          prefetch_l2(ct, (uint32_t)(MX_N * BEOR_TB * sizeof(float4)));
        }
        // two half-stages per K-chunk: h = 0 loads A part Im with the B window
        // (Im, Re), h = 1 A part Re with the window (Re, -Im)
        for (int kc = 0; kc < BEOR_TB / MX_KC; ++kc) {
          for (int h = 0; h < 2; ++h, ++it) {
            if (!mbar_wait(empty_bar(ps), pph ^ 1, abort_flag, wait_ns)) {
              atomicCAS(&v.flags->error, 0, ERR_TMA_WAIT);
              *abort_flag = 1;
              goto producer_done;
            }
            const uint32_t s = ps;
            if (++ps == SLOTS) {
              ps = 0;
              pph ^= 1;
            }
            if (TRAILING && v.test_skip_copy && blockIdx.x == 0 && n == 0 && kc == 3 && h == 0) {
              // test switch: no copy and no arrival for this slot, so the
              // MMA warp's wait on it can only end by its limit (the first
              // CTA of each trailing launch; once one wait has given up, the
              // later launches return at once)
              withheld = it;
              continue;
            }
            const uint32_t dst = sbase + s * SLOT;
            // x = 0 always (16-byte aligned); y counts pairs of 8-row groups
            mbar_expect_tx(full_bar(s), SLOT);
            tma_load_5d(dst, &map_a, 0, a_row / 16, kc, h, 0, full_bar(s));
            tma_load_5d(dst + ABYTES, &map_b, 0, b_row / 16, kc, h, 0, full_bar(s));
          }
        }
      }
    producer_done:
      // drain: every issued copy must have landed before the CTA may exit
      for (uint32_t q = (it >= SLOTS ? it - SLOTS : 0); q < it; ++q)
        if (q != withheld) mbar_wait_deadline(full_bar(q % SLOTS), (q / SLOTS) & 1);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      // ring position (slot rs, phase rph), advanced slot by slot without
      // divisions: the thread issues back to back and must not leave gaps
      // in the tensor pipe between half-stages
      uint32_t rs = 0, rph = 0, tcount = 0;
      const uint64_t desc0 = sdesc_kmajor(sbase);
      for (uint32_t n = 0;; ++n) {
        const uint32_t q = n % MX_JOBS;
        if (!mbar_wait(job_full(q), (n / MX_JOBS) & 1, abort_flag, wait_ns)) {
          atomicCAS(&v.flags->error, 0, ERR_MMA_WAIT);
          *abort_flag = 1;
          break;
        }
        const TileJob jb = jobs[q];
        mbar_arrive(job_empty(q));
        if (jb.p < 0) break;
        if (!mbar_wait(acc_empty, (tcount & 1) ^ 1, abort_flag, wait_ns)) {
          atomicCAS(&v.flags->error, 0, ERR_ACC_WAIT);
          *abort_flag = 1;
          break;
        }
        tc_fence_after();
        bool bad = false;
        for (int kc = 0; kc < BEOR_TB / MX_KC && !bad; ++kc) {
          for (int h = 0; h < 2; ++h) {
            if (!mbar_wait(full_bar(rs), rph, abort_flag, wait_ns)) {
              atomicCAS(&v.flags->error, 0, ERR_MMA_WAIT);
              *abort_flag = 1;
              bad = true;
              break;
            }
            tc_fence_after();
            const uint64_t ad = sdesc_add(desc0, rs * SLOT), bd = sdesc_add(ad, ABYTES);
            // A slice sa times B slices t contributes to level min(sa + t, 3)
            // (schedule: slice_mma_*); the window's slices lie at 4 KB steps in
            // shared memory, their two parts 64 rows apart, so that a product
            // over two levels reads 256 consecutive rows
            issue_half_stage<Ring<MODE>::set>(tmem, ad, bd, kc == 0 && h == 0);
            tc_commit(empty_bar(rs));
            if (++rs == SLOTS) {
              rs = 0;
              rph ^= 1;
            }
          }
        }
        if (bad) break;
        tc_commit(acc_full);
        ++tcount;
      }
      // drain outstanding tensor-core work before TMEM is released
      tc_commit(drain);
      mbar_wait_deadline(drain, 0);
    }
  } else {
    // ---------------- epilogue (warps 2..9) ----------------
    const int lane_base = 32 * (warp & 3);
    const int r = lane_base + lane;   // output row within the tile
    const int cbeg = ((warp - 2) >> 2) * (MX_N / 2);   // first of this warp's 32 columns
    uint32_t tcount = 0;
    for (uint32_t n = 0;; ++n) {
      const uint32_t q = n % MX_JOBS;
      if (!mbar_wait(job_full(q), (n / MX_JOBS) & 1, abort_flag, wait_ns)) {
        atomicCAS(&v.flags->error, 0, ERR_EPI_WAIT);
        *abort_flag = 1;
        break;
      }
      const TileJob jb = jobs[q];
      __syncwarp();
      if (lane == 0) mbar_arrive(job_empty(q));
      if (jb.p < 0) break;
      const Prob pr = v.prob[jb.p];
      const int out_j = jb.j;   // trail: block column j; panel: the panel column
      const bool tile_ok = BEOR_INBOUNDS(
          v.flags, pr.ws_off + (tri_index(jb.i, out_j) + 1) * BEOR_TILE_ELEMS <= v.ws_elems, BC_EPI_WS);
      const bool exp_ok = BEOR_INBOUNDS(
          v.flags,
          pr.row_off + (int64_t)jb.i * BEOR_TB + r < v.rows &&
              (TRAILING ? pr.row_off + (int64_t)jb.j * BEOR_TB + jb.h * MX_N + MX_N <= v.rows
                                  : (int64_t)jb.p * BEOR_TB + jb.h * MX_N + MX_N <= (int64_t)v.P * BEOR_TB),
          BC_EPI_EXP);
      const int e_r = exp_ok ? pexp[pr.row_off + (int64_t)jb.i * BEOR_TB + r] : -1000;
      const int32_t* ecol = TRAILING ? pexp + pr.row_off + (int64_t)jb.j * BEOR_TB + jb.h * MX_N
                                               : v.linv_exp + (int64_t)jb.p * BEOR_TB + jb.h * MX_N;
      float4* __restrict__ C = reinterpret_cast<float4*>(v.ws) + pr.ws_off + tri_index(jb.i, out_j) * BEOR_TILE_ELEMS +
                  (int64_t)(jb.h * MX_N) * BEOR_TB + r;
      const uint32_t trow = tmem + ((uint32_t)lane_base << 16);
      constexpr int NC = MX_N / 2;   // this warp's columns
      constexpr int EC = 4;          // columns per chunk
      // the first working-matrix columns do not depend on the product: load them before it is done
      float4 cv[EC];
      if (TRAILING && tile_ok) {
#pragma unroll
        for (int q = 0; q < EC; ++q) cv[q] = __ldcs(C + (int64_t)(cbeg + q) * BEOR_TB);
      }
      if (!mbar_wait(acc_full, tcount & 1, abort_flag, wait_ns)) {
        atomicCAS(&v.flags->error, 0, ERR_EPI_WAIT);
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      // Phase 1: the four level accumulators of each output, summed to an
      // unnormalised double-float, move from tensor memory to registers;
      // then tensor memory is released, and the next tile's products run
      // during phase 2, which normalises the sums.
      float prh[NC], prl[NC], pih[NC], pil[NC];
#pragma unroll
      for (int c0 = 0; c0 < NC; c0 += 4) {
        float lr[4][4], li[4][4];
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          tmem_ld4(trow + (uint32_t)(l * 128 + cbeg + c0), lr[l]);
          tmem_ld4(trow + (uint32_t)(l * 128 + MX_N + cbeg + c0), li[l]);
        }
        tmem_ld_wait();
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          reg_fence4(lr[l]);
          reg_fence4(li[l]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const dfl vr = levels_sum_split(lr[0][q], lr[1][q], lr[2][q], lr[3][q]);
          const dfl vi = levels_sum_split(li[0][q], li[1][q], li[2][q], li[3][q]);
          prh[c0 + q] = vr.hi;
          prl[c0 + q] = vr.lo;
          pih[c0 + q] = vi.hi;
          pil[c0 + q] = vi.lo;
        }
      }
      tc_fence_before();
      mbar_arrive(acc_empty);
      // Phase 2: scale by 2^(e_r + e_c - 14) and subtract from (trail) or
      // store into (panel) the working matrix.
#pragma unroll
      for (int c0 = 0; c0 < NC && tile_ok; c0 += EC) {
        float4 cn[EC];
        if (TRAILING && c0 + EC < NC) {
#pragma unroll
          for (int q = 0; q < EC; ++q) cn[q] = __ldcs(C + (int64_t)(cbeg + c0 + EC + q) * BEOR_TB);
        }
#pragma unroll
        for (int q = 0; q < EC; ++q) {
          const int c = cbeg + c0 + q;
          const int ec = exp_ok ? __ldg(ecol + c) : -1000;
          int ex = e_r + ec - 14;
          if (e_r <= -1000 || ec <= -1000) ex = 0;
          ex = max(-250, min(250, ex));
          const int e1 = ex >> 1, e2 = ex - e1;   // two exact power-of-two factors
          const float s1 = __int_as_float((e1 + 127) << 23), s2 = __int_as_float((e2 + 127) << 23);
          const dfl nr = df_fast_two_sum(prh[c0 + q], prl[c0 + q]);
          const dfl ni = df_fast_two_sum(pih[c0 + q], pil[c0 + q]);
          const dfl vr{nr.hi * s1 * s2, nr.lo * s1 * s2};
          const dfl vi{ni.hi * s1 * s2, ni.lo * s1 * s2};
          float4* cp = C + (int64_t)c * BEOR_TB;
          if (TRAILING) {
            const float4 w = cv[q];
            const dfl wr = df_sub_quick(dfl{w.x, w.y}, vr);
            const dfl wi = df_sub_quick(dfl{w.z, w.w}, vi);
            __stcs(cp, make_float4(wr.hi, wr.lo, wi.hi, wi.lo));
          } else {
            __stcs(cp, make_float4(vr.hi, vr.lo, vi.hi, vi.lo));
          }
        }
        if (TRAILING) {
#pragma unroll
          for (int q = 0; q < EC; ++q) cv[q] = cn[q];
        }
      }
      ++tcount;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(MX_TMEM_COLS));
  }
}

// ---------------------------------------------------------------------------
// slicing of the panel rows: rows of tiles (i, k), i > k, of every problem
// ---------------------------------------------------------------------------
constexpr int SL_R = 16;                                    // rows per group
constexpr int SL_GROUPS = 4;                                // groups per CTA (half a block row)
constexpr int SL_CTAS = BEOR_TB / (SL_R * SL_GROUPS);       // CTAs per block row
constexpr int SL_BUF = BEOR_TB * (SL_R + 1);                // float4 per buffer: [column][row], padded
constexpr int SL_SMEM = 2 * SL_BUF * (int)sizeof(float4);   // double buffer: 69632 bytes

__device__ __forceinline__ void cp_async16(float4* dst, const float4* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// Two CTAs per block row i of every problem, each taking four groups of 16
// rows in turn: the next group's double-float rows are copied into shared
// memory (cp.async) while the current group is sliced.
__global__ void __launch_bounds__(256)
    slice_panel_kernel(BatchView v, int kg, __nv_bfloat16* __restrict__ panel_sl, int32_t* __restrict__ panel_exp) {
  extern __shared__ float4 sl_smem[];
  __shared__ int s_e[SL_R];
  const int p = blockIdx.y;
  const Prob pr = v.prob[p];
  const int k = kg - pr.k_off;   // this problem's block step
  const int i = k + 1 + blockIdx.x / SL_CTAS;
  const int g0 = (blockIdx.x % SL_CTAS) * SL_GROUPS;   // first group of this CTA
  if (k < 0 || i >= pr.nt || prob_skipped(v.status[p])) return;
  if (!BEOR_INBOUNDS(v.flags, pr.ws_off + (tri_index(i, k) + 1) * BEOR_TILE_ELEMS <= v.ws_elems, BC_SLICE_ROW)) return;
  const float4* tile = reinterpret_cast<const float4*>(v.ws) + pr.ws_off + tri_index(i, k) * BEOR_TILE_ELEMS;
  auto load_group = [&](int grp) {   // rows 16 (g0 + grp) .. + 15, every column
    float4* buf = sl_smem + (grp & 1) * SL_BUF;
    for (int e = threadIdx.x; e < BEOR_TB * SL_R; e += 256) {
      const int c = e / SL_R, r = e % SL_R;
      cp_async16(buf + c * (SL_R + 1) + r, tile + c * BEOR_TB + (g0 + grp) * SL_R + r);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t rows = v.rows;
  // digit work: one 16-byte chunk of every plane per thread (one row, 8
  // consecutive columns); warp w takes K-chunk w and lane = (8-row group, K
  // half, row), so that a warp writes 512 contiguous bytes of each plane
  static_assert(SL_R == 16 && BEOR_TB / MX_KC == 8, "one warp per K-chunk, 32 chunks of 16 bytes per warp");
  const int rr = lane & 7, kh = (lane >> 3) & 1, hg = lane >> 4;
  const int r = hg * 8 + rr;
  const int c0 = warp * MX_KC + kh * 8;
  load_group(0);
  for (int grp = 0; grp < SL_GROUPS; ++grp) {
    if (grp + 1 < SL_GROUPS) {
      load_group(grp + 1);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();   // group grp is in shared memory
    const float4* buf = sl_smem + (grp & 1) * SL_BUF;
    const int r0 = (g0 + grp) * SL_R;
    // per-row exponent (one warp per row)
    for (int rw = warp; rw < SL_R; rw += 8) {
      float mx = 0.0f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 a = buf[(lane + 32 * q) * (SL_R + 1) + rw];
        mx = fmaxf(mx, fmaxf(fabsf(a.x), fabsf(a.z)));
      }
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      const int e = mx > 0.0f ? ilogbf(mx) + 1 : -1000;
      if (lane == 0) {
        s_e[rw] = e;
        if (BEOR_INBOUNDS(v.flags, pr.row_off + (int64_t)i * BEOR_TB + r0 + rw < rows, BC_SLICE_ROW))
          panel_exp[pr.row_off + (int64_t)i * BEOR_TB + r0 + rw] = e;
      }
    }
    __syncthreads();
    const int e = s_e[r];
    const int64_t grow = pr.row_off + (int64_t)i * BEOR_TB + r0 + r;
    uint32_t packed[BEOR_NPLANE][4];
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
      float val[2][BEOR_NPLANE];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const float4 a = buf[(c0 + q + u) * (SL_R + 1) + r];
#pragma unroll
        for (int part = 0; part < 2; ++part) {   // 0: real, 1: imaginary
          const float hi = part ? a.z : a.x, lo = part ? a.w : a.y;
          // balanced base-256 digits of the fixed-point number round(x * 2^(39 - e))
          float dv[BEOR_NSLICE];
          balanced_digits5(hi, lo, e, dv);
#pragma unroll
          for (int sl = 0; sl < BEOR_NSLICE; ++sl) {
            const float d = dv[sl];
            if (part == 0) {
              val[u][slice_plane(sl, BEOR_PART_RE)] = d;
            } else {
              val[u][slice_plane(sl, BEOR_PART_IM)] = d;
              val[u][slice_plane(sl, BEOR_PART_NEGIM)] = -d;
            }
          }
        }
      }
#pragma unroll
      for (int pl = 0; pl < BEOR_NPLANE; ++pl) {
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(val[0][pl], val[1][pl]);   // .x at the lower address
        packed[pl][q / 2] = *reinterpret_cast<const uint32_t*>(&h2);
      }
    }
    const int64_t off = slice_elem_off(grow, c0, rows);   // a multiple of 8 elements: 16-byte aligned
    if (BEOR_INBOUNDS(v.flags, grow < rows && off + 8 <= rows * BEOR_TB, BC_SLICE_OFF)) {
#pragma unroll
      for (int pl = 0; pl < BEOR_NPLANE; ++pl)
        *reinterpret_cast<uint4*>(panel_sl + (int64_t)pl * rows * BEOR_TB + off) =
            make_uint4(packed[pl][0], packed[pl][1], packed[pl][2], packed[pl][3]);
    }
    __syncthreads();   // buffer grp & 1 and s_e may be overwritten
  }
}

static __nv_bfloat16* slice_buf(const BatchView& v, int k) {
  return v.panel_sl + (size_t)(k & 1) * BEOR_NPLANE * v.rows * BEOR_TB;
}
static int32_t* exp_buf(const BatchView& v, int k) { return v.panel_exp + (size_t)(k & 1) * v.rows; }

cudaError_t launch_slice_panel(const BatchView& v, int k, cudaStream_t s, int prio) {
  const int nblk = SL_CTAS * (v.max_nt - 1 - k);   // block rows below block column k
  if (nblk <= 0) return cudaSuccess;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(slice_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SL_SMEM);
    attr = true;
  }
  return launch_prio(slice_panel_kernel, dim3(nblk, v.P), dim3(256), (size_t)SL_SMEM, s, prio, v, k,
                     slice_buf(v, k), exp_buf(v, k));
}

// ---------------------------------------------------------------------------
// host side: tensor maps, tile prefixes, launches
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// Slice planes in slice_elem_off order seen as a 5-D tensor: 256 elements
// (two 8-row groups, 512 contiguous bytes) x rows/16 x 8 K-chunks x 3 parts
// x 5 slices (plane = slice * 3 + part).  A box of box_rows rows of one
// K-chunk, `parts` consecutive parts from a given one and every slice is
// exactly the shared-memory operand image (no swizzle), fetched as 512-byte
// rows: [slice][part][rows] of 8-row x 16-byte core matrices.
static cudaError_t make_map(CUtensorMap* m, void* base, int64_t rows, int box_rows, int parts,
                            int slices = BEOR_NSLICE) {
  auto enc = get_encode();
  if (!enc) return cudaErrorNotSupported;
  if (rows % 16 || box_rows % 16) return cudaErrorInvalidValue;
  cuuint64_t dims[5] = {256, (cuuint64_t)(rows / 16), (cuuint64_t)(BEOR_TB / MX_KC), (cuuint64_t)BEOR_NPART,
                        (cuuint64_t)BEOR_NSLICE};
  cuuint64_t strides[4] = {512, (cuuint64_t)rows * MX_KC * 2, (cuuint64_t)rows * BEOR_TB * 2,
                           (cuuint64_t)rows * BEOR_TB * 2 * BEOR_NPART};
  cuuint32_t box[5] = {256, (cuuint32_t)(box_rows / 16), 1, (cuuint32_t)parts, (cuuint32_t)slices};
  cuuint32_t es[5] = {1, 1, 1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, base, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t mixed_maps_create(const BatchView& v, MixedMaps** out) {
  *out = nullptr;
  MixedMaps* m = new MixedMaps();
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    e = make_map(&m->panel_a[b], slice_buf(v, b), v.rows, MX_M, 1);
    if (e == cudaSuccess) e = make_map(&m->panel_b[b], slice_buf(v, b), v.rows, MX_N, 2);
    if (e == cudaSuccess) e = make_map(&m->panel_a4[b], slice_buf(v, b), v.rows, MX_M, 1, 4);
    if (e == cudaSuccess) e = make_map(&m->panel_b4[b], slice_buf(v, b), v.rows, MX_N, 2, 4);
  }
  if (e == cudaSuccess) e = make_map(&m->linv_b, v.linv_sl, (int64_t)v.P * BEOR_TB, MX_N, 2);
  if (e != cudaSuccess) {
    delete m;
    return e;
  }
  // tile prefix sums per step and kind (two 64-column sub-tiles per 128-tile)
  std::vector<Prob> hp(v.P);
  e = cudaMemcpy(hp.data(), v.prob, sizeof(Prob) * v.P, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    delete m;
    return e;
  }
  m->max_nt = v.max_nt;
  m->P = v.P;
  const int H = BEOR_TB / MX_N;
  std::vector<int64_t> pre((size_t)KIND_COUNT * v.max_nt * (v.P + 1), 0);
  for (int kind = 0; kind < KIND_COUNT; ++kind) m->h_total[kind].assign(v.max_nt, 0);
  for (int kind = 0; kind < KIND_COUNT; ++kind)
    for (int k = 0; k < v.max_nt; ++k) {
      int64_t* pk = pre.data() + ((size_t)kind * v.max_nt + k) * (v.P + 1);
      for (int p = 0; p < v.P; ++p) {
        const int kp = k - hp[p].k_off;                      // the problem's own block step
        const int T = kp < 0 ? 0 : std::max(0, hp[p].nt - kp - 1);   // block rows below the diagonal
        int64_t n = 0;
        switch (kind) {
          case KIND_PANEL: n = T; break;                          // i >= k + 1
          case KIND_COL: n = std::max(0, T - 1); break;           // i >= k + 2, j = k + 1
          case KIND_DCOL: n = T > 0 ? 1 : 0; break;               // (k + 1, k + 1)
          case KIND_REST: n = tri_count(std::max(0, T - 2)); break;   // i > j >= k + 2
          case KIND_DREST: n = std::max(0, T - 1); break;         // i = j >= k + 2
          case KIND_ALL: n = tri_count(std::max(0, T - 1)); break;    // i > j >= k + 1
          default: n = T; break;                                  // KIND_DALL: i = j >= k + 1
        }
        pk[p + 1] = pk[p] + n * H;
      }
      m->h_total[kind][k] = pk[v.P];
    }
  e = cudaMalloc(&m->d_prefix, sizeof(int64_t) * pre.size());
  if (e == cudaSuccess) e = cudaMemcpy(m->d_prefix, pre.data(), sizeof(int64_t) * pre.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&m->d_counter, sizeof(int) * KIND_COUNT * (size_t)v.max_nt);
  if (e != cudaSuccess) {
    mixed_maps_destroy(m);
    return e;
  }
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(slice_gemm_kernel<MODE_TRAIL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         Ring<MODE_TRAIL>::smem);
    cudaFuncSetAttribute(slice_gemm_kernel<MODE_TRAIL_DIAG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         Ring<MODE_TRAIL_DIAG>::smem);
    cudaFuncSetAttribute(slice_gemm_kernel<MODE_PANEL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         Ring<MODE_PANEL>::smem);
    attr = true;
  }
  *out = m;
  return cudaSuccess;
}

void mixed_maps_destroy(MixedMaps* m) {
  if (!m) return;
  if (m->d_prefix) cudaFree(m->d_prefix);
  if (m->d_counter) cudaFree(m->d_counter);
  delete m;
}

cudaError_t mixed_reset_counters(const MixedMaps* m, cudaStream_t s) {
  return cudaMemsetAsync(m->d_counter, 0, sizeof(int) * KIND_COUNT * (size_t)m->max_nt, s);
}

static int64_t mixed_tiles_kind(const MixedMaps* m, int kind, int k) {
  return k >= 0 && k < m->max_nt ? m->h_total[kind][k] : 0;
}

int64_t mixed_tiles(const MixedMaps* m, int kind, int k) {
  if (k < 0 || k >= m->max_nt) return 0;
  const int diag = kind == KIND_COL ? KIND_DCOL : kind == KIND_REST ? KIND_DREST : kind == KIND_ALL ? KIND_DALL : -1;
  return m->h_total[kind][k] + (diag >= 0 ? m->h_total[diag][k] : 0);
}

static int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

static cudaError_t launch_gemm(const BatchView& v, const MixedMaps* m, int k, int kind, cudaStream_t s, int prio,
                               int max_ctas = 0) {
  const int64_t nt = m->h_total[kind][k];
  if (nt <= 0) return cudaSuccess;
  int cap = (kind == KIND_REST || kind == KIND_DREST) ? v.grid_rest
            : (kind == KIND_COL || kind == KIND_DCOL || kind == KIND_PANEL) ? v.grid_col : 0;
  if (cap <= 0) cap = num_sms();
  if (max_ctas > 0) cap = std::min(cap, max_ctas);
  const int grid = (int)std::min<int64_t>(nt, cap);
  const int64_t* pre = m->d_prefix + ((size_t)kind * m->max_nt + k) * (m->P + 1);
  int* ctr = m->d_counter + (size_t)kind * m->max_nt + k;
  const int32_t* pexp = (const int32_t*)exp_buf(v, k);
  if (kind == KIND_PANEL)
    return launch_prio(slice_gemm_kernel<MODE_PANEL>, dim3(grid), dim3(MX_THREADS), (size_t)Ring<MODE_PANEL>::smem,
                       s, prio, m->panel_a[k & 1], m->linv_b, v, pre, nt, k, kind, ctr, pexp);
  if (kind == KIND_DCOL || kind == KIND_DREST || kind == KIND_DALL)
    return launch_prio(slice_gemm_kernel<MODE_TRAIL_DIAG>, dim3(grid), dim3(MX_THREADS),
                       (size_t)Ring<MODE_TRAIL_DIAG>::smem, s, prio, m->panel_a[k & 1], m->panel_b[k & 1], v, pre, nt,
                       k, kind, ctr, pexp);
  return launch_prio(slice_gemm_kernel<MODE_TRAIL>, dim3(grid), dim3(MX_THREADS), (size_t)Ring<MODE_TRAIL>::smem, s,
                     prio, m->panel_a4[k & 1], m->panel_b4[k & 1], v, pre, nt, k, kind, ctr, pexp);
}

cudaError_t launch_panel_mixed(const BatchView& v, const MixedMaps* m, int k, cudaStream_t s, int prio) {
  return launch_gemm(v, m, k, KIND_PANEL, s, prio);
}

// The off-diagonal tiles (reduced pair set), then the diagonal ones (full
// set), on the same stream.
cudaError_t launch_trail_mixed(const BatchView& v, const MixedMaps* m, int k, int part, cudaStream_t s, int prio,
                               int max_ctas) {
  const int kind = part == TRAIL_NEXT_COL ? KIND_COL : part == TRAIL_REST ? KIND_REST : KIND_ALL;
  const int diag = part == TRAIL_NEXT_COL ? KIND_DCOL : part == TRAIL_REST ? KIND_DREST : KIND_DALL;
  cudaError_t e = launch_gemm(v, m, k, kind, s, prio, max_ctas);
  if (e == cudaSuccess) e = launch_gemm(v, m, k, diag, s, prio, max_ctas);
  return e;
}

int trail_launch_count(const MixedMaps* m, int k, int part) {
  const int kind = part == TRAIL_NEXT_COL ? KIND_COL : part == TRAIL_REST ? KIND_REST : KIND_ALL;
  const int diag = part == TRAIL_NEXT_COL ? KIND_DCOL : part == TRAIL_REST ? KIND_DREST : KIND_DALL;
  return (mixed_tiles_kind(m, kind, k) > 0) + (mixed_tiles_kind(m, diag, k) > 0);
}

int device_sms() { return num_sms(); }

// ---------------------------------------------------------------------------
// float64 refinement: vec_r = dbar - (M + diag Phi^-1) x, x += vec_d
// ---------------------------------------------------------------------------
__global__ void resid_init_kernel(BatchView v) {
  const int p = blockIdx.y;
  const Prob pr = v.prob[p];
  const SetDesc sd = v.sets[pr.set];
  const int np = pr.nt * BEOR_TB;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < np; j += gridDim.x * blockDim.x) {
    double2 x = v.vec_x[pr.row_off + j], d = sd.dbar[j];
    double w = v.phi_inv[pr.row_off + j];
    v.vec_r[pr.row_off + j] = j < pr.n ? make_double2(d.x - w * x.x, d.y - w * x.y) : make_double2(0.0, 0.0);
  }
}

// x split exactly into three floats per component (hi, lo, t), for the
// float32-pipe residual below.
__global__ void xsplit_kernel(BatchView v) {
  const int p = blockIdx.y;
  const Prob pr = v.prob[p];
  const int np = pr.nt * BEOR_TB;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < np; j += gridDim.x * blockDim.x) {
    const double2 x = v.vec_x[pr.row_off + j];
    float* o = v.xtr + (pr.row_off + j) * 6;
    const float rh = (float)x.x, ih = (float)x.y;
    const double rd = x.x - (double)rh, id = x.y - (double)ih;
    const float rl = (float)rd, il = (float)id;
    o[0] = rh;
    o[1] = rl;
    o[2] = (float)(rd - (double)rl);
    o[3] = ih;
    o[4] = il;
    o[5] = (float)(id - (double)il);
  }
}

// hi + sm += (ah + al + at)(bh + bl + bt): the leading product split exactly
// (p + e, FMA), the terms down to 2^-48 of it added to e, p added to hi by an
// error-free two-sum whose error goes to sm (Ogita, Rump and Oishi, "Accurate
// sum and dot product", SIAM J. Sci. Comput. 26 (2005), Dot2).
__device__ __forceinline__ void dot2_mac(float& hi, float& sm, float ah, float al, float at, float bh, float bl,
                                         float bt) {
  const float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  e = fmaf(ah, bt, e);
  e = fmaf(al, bl, e);
  e = fmaf(at, bh, e);
  const float s = hi + p;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (p - bb);
  hi = s;
  sm += err + e;
}

// r_I -= sum_J M_IJ x_J for the problems of one work item, with float64-like
// accuracy on the float32 pipe: M and x as exact float triples, Dot2 products
// and sums within a 128-column tile, float64 totals across tiles and, across
// work items, float64 atomics.  Thread (row r, half h) serves 8 problems.
constexpr int RG = 16;   // problems per work item
__global__ void __launch_bounds__(256, 2) resid_df_kernel(BatchView v) {
  extern __shared__ float xs[];          // [RG][128][6]
  __shared__ int64_t roff[RG];
  const RWork w = v.rwork[blockIdx.x];
  const SetDesc sd = v.sets[w.set];
  const int r = threadIdx.x & (BEOR_TB - 1), half = threadIdx.x >> 7;
  if (threadIdx.x < RG) {
    const int q = threadIdx.x;
    roff[q] = q < w.nb && !prob_skipped(v.status[w.p0 + q]) ? v.prob[w.p0 + q].row_off : (int64_t)-1;
  }
  double tre[8], tim[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) tre[q] = tim[q] = 0.0;
  if (!BEOR_INBOUNDS(v.flags, w.I >= 0 && w.I < sd.nt && w.j0 >= 0 && w.j1 <= sd.nt, BC_RESID_M)) return;
  if (threadIdx.x < RG && roff[threadIdx.x] >= 0 &&
      !BEOR_INBOUNDS(v.flags, roff[threadIdx.x] + (int64_t)sd.nt * BEOR_TB <= v.rows, BC_RESID_X))
    roff[threadIdx.x] = -1;
  for (int J = w.j0; J < w.j1; ++J) {
    __syncthreads();
    for (int e = threadIdx.x; e < RG * BEOR_TB * 6; e += blockDim.x) {
      const int q = e / (BEOR_TB * 6), rem = e - q * (BEOR_TB * 6);
      xs[e] = roff[q] >= 0 ? v.xtr[(roff[q] + (int64_t)J * BEOR_TB) * 6 + rem] : 0.0f;
    }
    __syncthreads();
    const int64_t t0 = ((int64_t)w.I * sd.nt + J) * BEOR_TILE_ELEMS + r;
    const float4* __restrict__ T4 = sd.Mf + t0;
    const float2* __restrict__ T2 = sd.Mft + t0;
    float hr[8], sr[8], hi[8], si[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) hr[q] = sr[q] = hi[q] = si[q] = 0.0f;
#pragma unroll 2
    for (int c = 0; c < BEOR_TB; ++c) {
      const float4 m4 = __ldg(T4 + c * BEOR_TB);
      const float2 m2 = __ldg(T2 + c * BEOR_TB);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float* x = xs + ((half * 8 + q) * BEOR_TB + c) * 6;
        const float xrh = x[0], xrl = x[1], xrt = x[2], xih = x[3], xil = x[4], xit = x[5];
        // re += mr xr - mi xi, im += mr xi + mi xr
        dot2_mac(hr[q], sr[q], m4.x, m4.y, m2.x, xrh, xrl, xrt);
        dot2_mac(hr[q], sr[q], -m4.z, -m4.w, -m2.y, xih, xil, xit);
        dot2_mac(hi[q], si[q], m4.x, m4.y, m2.x, xih, xil, xit);
        dot2_mac(hi[q], si[q], m4.z, m4.w, m2.y, xrh, xrl, xrt);
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      tre[q] += (double)hr[q] + (double)sr[q];
      tim[q] += (double)hi[q] + (double)si[q];
    }
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int64_t ro = roff[half * 8 + q];
    if (ro < 0) continue;
    double2* dst = v.vec_r + ro + (int64_t)w.I * BEOR_TB + r;
    atomicAdd(&dst->x, -tre[q]);
    atomicAdd(&dst->y, -tim[q]);
  }
}

__global__ void resid_norm_kernel(BatchView v) {
  const int p = blockIdx.x;
  const Prob pr = v.prob[p];
  const SetDesc sd = v.sets[pr.set];
  __shared__ double red[2][32];
  double a = 0.0, b = 0.0;
  for (int j = threadIdx.x; j < pr.n; j += blockDim.x) {
    double2 r = v.vec_r[pr.row_off + j], d = sd.dbar[j];
    a += r.x * r.x + r.y * r.y;
    b += d.x * d.x + d.y * d.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = a;
    red[1][threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      sa += red[0][w];
      sb += red[1][w];
    }
    v.resid[p] = sb > 0.0 ? sqrt(sa / sb) : 0.0;
  }
}

cudaError_t launch_residual(const BatchView& v, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(resid_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(float) * RG * BEOR_TB * 6));
    attr = true;
  }
  resid_init_kernel<<<dim3(8, v.P), 256, 0, s>>>(v);
  xsplit_kernel<<<dim3(8, v.P), 256, 0, s>>>(v);
  resid_df_kernel<<<v.n_rwork, 256, sizeof(float) * RG * BEOR_TB * 6, s>>>(v);
  resid_norm_kernel<<<v.P, 256, 0, s>>>(v);
  return cudaGetLastError();
}

// x += d for every problem; one CTA per problem.  The relative size of the
// correction, ||d|| / ||x||, is the convergence measure: the error left after
// the step is about rho ||d||, with rho ~ kappa * 2^-39 << 1 the contraction
// of the refinement for the slice factor, so a correction below 1e-4 of x
// leaves an error far below every tolerance, while a failing factorisation
// (rho ~ 1) produces corrections of the size of x.  Larger -> status -1.
__global__ void refine_update_kernel(BatchView v) {
  const int p = blockIdx.x;
  const Prob pr = v.prob[p];
  if (prob_skipped(v.status[p])) return;
  __shared__ double red[2][32];
  const int np = pr.nt * BEOR_TB;
  double a = 0.0, b = 0.0;
  for (int j = threadIdx.x; j < np; j += blockDim.x) {
    const double2 x = v.vec_x[pr.row_off + j], d = v.vec_d[pr.row_off + j];
    const double2 y = make_double2(x.x + d.x, x.y + d.y);
    v.vec_x[pr.row_off + j] = y;
    a += d.x * d.x + d.y * d.y;
    b += y.x * y.x + y.y * y.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = a;
    red[1][threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      sa += red[0][w];
      sb += red[1][w];
    }
    const double rel = sb > 0.0 ? sqrt(sa / sb) : 0.0;
    v.resid[p] = rel;
    v.status[p] = rel <= 1e-4 ? 0 : -1;
  }
}

cudaError_t launch_refine_update(const BatchView& v, cudaStream_t s) {
  refine_update_kernel<<<v.P, 256, 0, s>>>(v);
  return cudaGetLastError();
}

int mixed_supported(int device) {
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
  if (major != 10 || minor != 3) return 0;
  return get_encode() != nullptr;
}

}  // namespace beor
