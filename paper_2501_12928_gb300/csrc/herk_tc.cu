// Tensor-core precompute of M = T^H N^-1 T for a dense instrument matrix
// (mixed-precision contexts).
//
// Sec. "Running BayesEoR": M is formed once per instrument; the likelihood's
// float64-accurate residual then uses it as exact, so M must carry float64
// accuracy.  With Y = (diag(sqrt(w)) T)^T (row j = model mode, K = the
// visibilities), M = conj(Y Y^H).  Y is cut into K-blocks of 128
// visibilities; every row of every block is scaled by its own power of two
// and rounded to seven balanced base-256 digits (56 bits, more than the 53
// of the float64 input), and each block's product is formed by tcgen05
// slice products with the pairs s + t <= 6: levels 0-2 exact in the fp32
// accumulators, the rest in a fourth, rounded about 2^-48 below the leading
// term (the same scheme as the factorisation's slice GEMM, two more digits).
// After each K-block the four levels are drained, scaled by the block's row
// exponents and added to a double-float accumulator in registers; the tile
// is written to M after the last block.  The visibilities are processed in
// passes of up to 64 K-blocks (one slicing launch and one product launch
// per pass, the product accumulating into M).
//
// Kernel structure as in the slice GEMM: one CTA per SM, persistent over the
// lower 128 x 64 tiles of M (tile counter), warp 0 issues TMA loads into a
// 3-slot ring of half-stages (one A part of 128 rows and its two-part B
// window of 64 rows, seven slices, one K-chunk of 16: 56 KB), warp 1 issues
// the tensor-core products, warps 2-17 drain and accumulate (16 columns each,
// so that the tile's double-float accumulators fit in registers).  Every wait is
// bounded; on expiry the kernel records an error code, drains what it issued
// and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "beor_common.cuh"
#include "beor_internal.h"
#include "tc_ptx.cuh"

namespace beor {

constexpr int HK_NS = 7;                                   // slices: 56-bit operands
constexpr int HK_NPLANE = HK_NS * BEOR_NPART;              // 21 planes (Im, Re, -Im per slice)
constexpr int HK_M = 128, HK_N = 64, HK_KC = 16;
constexpr int HK_A_BYTES = HK_NS * HK_M * HK_KC * 2;       // 28672
constexpr int HK_B_BYTES = HK_NS * 2 * HK_N * HK_KC * 2;   // 28672
constexpr int HK_HALF = HK_A_BYTES + HK_B_BYTES;           // 57344
constexpr int HK_SLICE = 4096;                             // one slice of the A part or of the B window
constexpr int HK_SLOTS = 3;
constexpr int HK_SMEM = HK_SLOTS * HK_HALF + 1024 + 256;   // 173312
constexpr int HK_EPI_WARPS = 16;   // four per TMEM lane quarter, 16 columns each
constexpr int HK_THREADS = 64 + 32 * HK_EPI_WARPS;
constexpr int HK_KB_PASS = 64;                             // K-blocks of 128 per pass
constexpr int HK_JOBS = 4;
enum { HK_ERR_TMA = 21, HK_ERR_MMA = 22, HK_ERR_ACC = 23, HK_ERR_EPI = 24 };

// ---------------------------------------------------------------------------
// slicing: Y[j][v] = sqrt(w_v) T[v][j] for the K-blocks of one pass; block
// (kb, 16 rows); digits of round(y 2^(55 - e_j)) for the row exponent e_j of
// the block (largest |re|, |im| below 2^e_j)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) herk_slice_kernel(const double2* __restrict__ T, int64_t ld,
                                                         const double* __restrict__ w, int64_t n_vis, int n,
                                                         int64_t v0, int64_t rows, int nkb_buf,
                                                         __nv_bfloat16* __restrict__ planes,
                                                         int32_t* __restrict__ exps) {
  constexpr int R = 16;
  __shared__ double2 s[BEOR_TB][R + 1];   // [visibility][row]
  __shared__ int s_e[R];
  const int kb = blockIdx.x;
  const int64_t j0 = (int64_t)blockIdx.y * R;
  const int64_t vb = v0 + (int64_t)kb * BEOR_TB;
  for (int e = threadIdx.x; e < BEOR_TB * R; e += 256) {
    const int vl = e / R, jj = e % R;
    const int64_t v = vb + vl, j = j0 + jj;
    double2 y = make_double2(0.0, 0.0);
    if (v < n_vis && j < n) {
      const double2 t = T[v * ld + j];
      const double sw = sqrt(w[v]);
      y = make_double2(t.x * sw, t.y * sw);
    }
    s[vl][jj] = y;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int r = warp; r < R; r += 8) {
    double mx = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double2 a = s[lane + 32 * q][r];
      mx = fmax(mx, fmax(fabs(a.x), fabs(a.y)));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int e = mx > 0.0 ? ilogb(mx) + 1 : -1000;
    if (lane == 0) {
      s_e[r] = e;
      exps[(int64_t)kb * rows + j0 + r] = e;
    }
  }
  __syncthreads();
  // warp = K-chunk of 16, lane = (8-row group, K half, row): 16-byte chunks of every plane
  const int rr = lane & 7, kh = (lane >> 3) & 1, g = lane >> 4;
  const int r = g * 8 + rr;
  const int c0 = warp * HK_KC + kh * 8;
  const int e = s_e[r];
  uint32_t packed[HK_NPLANE][4];
#pragma unroll
  for (int q = 0; q < 8; q += 2) {
    float val[2][HK_NPLANE];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const double2 a = s[c0 + q + u][r];
#pragma unroll
      for (int part = 0; part < 2; ++part) {   // 0: real, 1: imaginary
        long long X = 0;
        if (e > -1000) X = llrint(ldexp(part ? a.y : a.x, 55 - e));   // exact scaling; |X| < 2^55
        int dg[HK_NS];
#pragma unroll
        for (int sl = HK_NS - 1; sl >= 1; --sl) {
          const long long m = ((X + 128) & 255) - 128;
          dg[sl] = (int)m;
          X = (X - m) >> 8;
        }
        dg[0] = (int)X;
#pragma unroll
        for (int sl = 0; sl < HK_NS; ++sl) {
          const float d = ldexpf((float)dg[sl], -8 * sl);
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
    for (int pl = 0; pl < HK_NPLANE; ++pl) {
      const __nv_bfloat162 h2 = __floats2bfloat162_rn(val[0][pl], val[1][pl]);
      packed[pl][q / 2] = *reinterpret_cast<const uint32_t*>(&h2);
    }
  }
  const int64_t plane_elems = rows * BEOR_TB * nkb_buf;
  const int64_t off = slice_elem_off(j0 + r, kb * BEOR_TB + c0, rows);   // 16-byte aligned
#pragma unroll
  for (int pl = 0; pl < HK_NPLANE; ++pl)
    *reinterpret_cast<uint4*>(planes + (int64_t)pl * plane_elems + off) =
        make_uint4(packed[pl][0], packed[pl][1], packed[pl][2], packed[pl][3]);
}

// ---------------------------------------------------------------------------
// products
// ---------------------------------------------------------------------------
__device__ __forceinline__ void hk_issue_half_stage(uint32_t tmem, uint32_t a0, uint32_t b0, bool first) {
#pragma unroll
  for (int sa = 0; sa < HK_NS; ++sa) {
    const uint64_t ad = sdesc_kmajor(a0 + sa * HK_SLICE);
#pragma unroll
    for (int q = 0; q < slice_mma_count(sa, SLICE_PAIRS_FULL7); ++q) {
      const uint32_t acc = (first && sa == 0 && q < slice_mma_main(0)) ? 0u : 1u;
      tc_mma(tmem + (uint32_t)slice_mma_col(sa, q), ad,
             sdesc_kmajor(b0 + slice_mma_t(sa, q, SLICE_PAIRS_FULL7) * HK_SLICE),
             idesc_bf16(0, (uint32_t)slice_mma_n(sa, q)), acc);
    }
  }
}

struct HkJob {
  int i, j, h;   // tile (i, j) of M, column half h; i < 0: no more work
};

// M tile (i, j) columns h*64.. += conj(sum over the pass's K-blocks), or =
// when `accumulate` is 0.  Tiles from `counter` (zeroed before the launch).
// 576 threads: 18 warps over the SM's four register-file partitions (16,384
// registers each), five warps on some: at most 96 registers per thread
__global__ void __launch_bounds__(HK_THREADS, 1)
    herk_tc_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                   const int32_t* __restrict__ exps, int64_t rows, int nt, int nkb, int accumulate,
                   double2* __restrict__ Mt, int* __restrict__ counter, int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + HK_SLOTS * HK_HALF);
  // bars[0..2] full, [3..5] empty, [6] acc_full, [7] acc_empty, [8] drain,
  // [9..12] job_full, [13..16] job_empty; then the TMEM address, the abort flag, the jobs
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 17);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 18);
  HkJob* jobs = reinterpret_cast<HkJob*>(bars + 20);
  static_assert(20 * 8 + HK_JOBS * sizeof(HkJob) <= 256, "barrier area");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (HK_SLOTS + s); };
  const uint32_t acc_full = bar0 + 8u * 6, acc_empty = bar0 + 8u * 7, drain = bar0 + 8u * 8;
  auto job_full = [&](uint32_t q) { return bar0 + 8u * (9 + q); };
  auto job_empty = [&](uint32_t q) { return bar0 + 8u * (13 + q); };
  const unsigned long long wait_ns = TC_DRAIN_NS;
  const int64_t ntiles = tri_count(nt) * 2;

  if (threadIdx.x == 0) {
    for (int s = 0; s < HK_SLOTS; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, 32 * HK_EPI_WARPS);
    mbar_init(drain, 1);
    for (int q = 0; q < HK_JOBS; ++q) {
      mbar_init(job_full(q), 1);
      mbar_init(job_empty(q), 1 + HK_EPI_WARPS);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    prefetch_map(&map_a);
    prefetch_map(&map_b);
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      uint32_t it = 0;
      for (uint32_t n = 0;; ++n) {
        const uint32_t q = n % HK_JOBS;
        if (!mbar_wait(job_empty(q), ((n / HK_JOBS) & 1) ^ 1, abort_flag, wait_ns)) {
          atomicCAS(err, 0, HK_ERR_TMA);
          *abort_flag = 1;
          goto producer_done;
        }
        HkJob jb{-1, 0, 0};
        const int64_t t = atomicAdd(counter, 1);
        if (t < ntiles) {
          int a, b;
          int64_t u = t >> 1;
          a = (int)((sqrtf(8.0f * (float)u + 1.0f) - 1.0f) * 0.5f);
          while ((int64_t)a * (a + 1) / 2 > u) --a;
          while ((int64_t)(a + 1) * (a + 2) / 2 <= u) ++a;
          b = (int)(u - (int64_t)a * (a + 1) / 2);
          jb = HkJob{a, b, (int)(t & 1)};
        }
        jobs[q] = jb;
        mbar_arrive(job_full(q));
        if (jb.i < 0) break;
        const int a_row = jb.i * BEOR_TB, b_row = jb.j * BEOR_TB + jb.h * HK_N;
        for (int kk = 0; kk < nkb * (BEOR_TB / HK_KC); ++kk) {
          for (int h = 0; h < 2; ++h, ++it) {
            const int s = it % HK_SLOTS;
            const uint32_t ph = (it / HK_SLOTS) & 1;
            if (!mbar_wait(empty_bar(s), ph ^ 1, abort_flag, wait_ns)) {
              atomicCAS(err, 0, HK_ERR_TMA);
              *abort_flag = 1;
              goto producer_done;
            }
            mbar_expect_tx(full_bar(s), HK_HALF);
            const uint32_t dst = sbase + s * HK_HALF;
            tma_load_5d(dst, &map_a, 0, a_row / 16, kk, h, 0, full_bar(s));
            tma_load_5d(dst + HK_A_BYTES, &map_b, 0, b_row / 16, kk, h, 0, full_bar(s));
          }
        }
      }
    producer_done:
      for (uint32_t q = (it >= HK_SLOTS ? it - HK_SLOTS : 0); q < it; ++q)
        mbar_wait_deadline(full_bar(q % HK_SLOTS), (q / HK_SLOTS) & 1);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      uint32_t it = 0, acount = 0;
      bool bad = false;
      for (uint32_t n = 0; !bad; ++n) {
        const uint32_t q = n % HK_JOBS;
        if (!mbar_wait(job_full(q), (n / HK_JOBS) & 1, abort_flag, wait_ns)) {
          atomicCAS(err, 0, HK_ERR_MMA);
          *abort_flag = 1;
          break;
        }
        const HkJob jb = jobs[q];
        mbar_arrive(job_empty(q));
        if (jb.i < 0) break;
        for (int kb = 0; kb < nkb && !bad; ++kb, ++acount) {
          if (!mbar_wait(acc_empty, (acount & 1) ^ 1, abort_flag, wait_ns)) {
            atomicCAS(err, 0, HK_ERR_ACC);
            *abort_flag = 1;
            bad = true;
            break;
          }
          tc_fence_after();
          for (int kc = 0; kc < BEOR_TB / HK_KC && !bad; ++kc) {
            for (int h = 0; h < 2; ++h, ++it) {
              const int s = it % HK_SLOTS;
              const uint32_t ph = (it / HK_SLOTS) & 1;
              if (!mbar_wait(full_bar(s), ph, abort_flag, wait_ns)) {
                atomicCAS(err, 0, HK_ERR_MMA);
                *abort_flag = 1;
                bad = true;
                break;
              }
              tc_fence_after();
              const uint32_t a0 = sbase + s * HK_HALF;
              hk_issue_half_stage(tmem, a0, a0 + HK_A_BYTES, kc == 0 && h == 0);
              tc_commit(empty_bar(s));
            }
          }
          if (!bad) tc_commit(acc_full);
        }
      }
      tc_commit(drain);
      mbar_wait_deadline(drain, 0);
    }
  } else {
    // ---------------- epilogue (warps 2..17): drain and accumulate ----------------
    const int lane_base = 32 * (warp & 3);
    const int r = lane_base + lane;
    constexpr int NC = HK_N / 4;   // this warp's columns
    const int cbeg = ((warp - 2) >> 2) * NC;
    uint32_t acount = 0;
    bool bad = false;
    for (uint32_t n = 0; !bad; ++n) {
      const uint32_t q = n % HK_JOBS;
      if (!mbar_wait(job_full(q), (n / HK_JOBS) & 1, abort_flag, wait_ns)) {
        atomicCAS(err, 0, HK_ERR_EPI);
        *abort_flag = 1;
        break;
      }
      const HkJob jb = jobs[q];
      __syncwarp();
      if (lane == 0) mbar_arrive(job_empty(q));
      if (jb.i < 0) break;
      const uint32_t trow = tmem + ((uint32_t)lane_base << 16);
      float arh[NC], arl[NC], aih[NC], ail[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) arh[c] = arl[c] = aih[c] = ail[c] = 0.0f;
      for (int kb = 0; kb < nkb; ++kb, ++acount) {
        const int e_r = exps[(int64_t)kb * rows + jb.i * BEOR_TB + r];
        // the warp's 32 columns: lane q holds column cbeg + q's exponent
        const int ec_lane = lane < NC ? exps[(int64_t)kb * rows + jb.j * BEOR_TB + jb.h * HK_N + cbeg + lane] : 0;
        if (!mbar_wait(acc_full, acount & 1, abort_flag, wait_ns)) {
          atomicCAS(err, 0, HK_ERR_EPI);
          *abort_flag = 1;
          bad = true;
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int c0 = 0; c0 < NC; c0 += 2) {
          float lr[4][2], li[4][2];
#pragma unroll
          for (int l = 0; l < 4; ++l) {
            tmem_ld2(trow + (uint32_t)(l * 128 + cbeg + c0), lr[l]);
            tmem_ld2(trow + (uint32_t)(l * 128 + HK_N + cbeg + c0), li[l]);
          }
          tmem_ld_wait();
#pragma unroll
          for (int l = 0; l < 4; ++l) {
            reg_fence2(lr[l]);
            reg_fence2(li[l]);
          }
#pragma unroll
          for (int qq = 0; qq < 2; ++qq) {
            const int ec = __shfl_sync(0xffffffffu, ec_lane, c0 + qq);
            int ex = e_r + ec - 14;
            if (e_r <= -1000 || ec <= -1000) ex = 0;
            ex = max(-250, min(250, ex));
            const int e1 = ex >> 1, e2 = ex - e1;   // two exact power-of-two factors
            const float s1 = __int_as_float((e1 + 127) << 23), s2 = __int_as_float((e2 + 127) << 23);
            const dfl vr = levels_sum(lr[0][qq], lr[1][qq], lr[2][qq], lr[3][qq]);
            const dfl vi = levels_sum(li[0][qq], li[1][qq], li[2][qq], li[3][qq]);
            // one exact two-sum of the high parts, the low parts added in fp32
            // (about 2^-48 of the sum per K-block)
            const dfl tr = df_two_sum(arh[c0 + qq], vr.hi * s1 * s2);
            const dfl ti = df_two_sum(aih[c0 + qq], vi.hi * s1 * s2);
            const dfl ar = df_fast_two_sum(tr.hi, tr.lo + (arl[c0 + qq] + vr.lo * s1 * s2));
            const dfl ai = df_fast_two_sum(ti.hi, ti.lo + (ail[c0 + qq] + vi.lo * s1 * s2));
            arh[c0 + qq] = ar.hi;
            arl[c0 + qq] = ar.lo;
            aih[c0 + qq] = ai.hi;
            ail[c0 + qq] = ai.lo;
            // done before the next columns' tensor-memory loads are issued
            asm volatile("" : "+f"(arh[c0 + qq]), "+f"(arl[c0 + qq]), "+f"(aih[c0 + qq]), "+f"(ail[c0 + qq]));
          }
        }
        tc_fence_before();
        mbar_arrive(acc_empty);
      }
      if (bad) break;
      // M = conj(Y Y^H): tile (i, j), rows r, columns h*64 + cbeg.. (column-major tile)
      double2* Mtile = Mt + tri_index(jb.i, jb.j) * BEOR_TILE_ELEMS + (int64_t)(jb.h * HK_N) * BEOR_TB + r;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        // one column at a time: neither its conversion nor its load is
        // hoisted above the previous column's store (which would hold every
        // column's values at once)
        asm volatile("" : "+f"(arh[c]), "+f"(arl[c]), "+f"(aih[c]), "+f"(ail[c])::"memory");
        double re = (double)arh[c] + (double)arl[c];
        double im = -((double)aih[c] + (double)ail[c]);
        double2* p = Mtile + (int64_t)(cbeg + c) * BEOR_TB;
        if (accumulate) {
          const double2 o = *p;
          re += o.x;
          im += o.y;
        }
        if (jb.i == jb.j && r == jb.h * HK_N + cbeg + c) im = 0.0;   // diagonal: exactly real
        *p = make_double2(re, im);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 hk_encode() {
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

// 5-D view of the pass's planes: 256 elements x rows/16 x K-chunks x 3 parts x 7 slices
static cudaError_t hk_map(CUtensorMap* m, void* base, int64_t rows, int nkb_buf, int box_rows, int parts) {
  auto enc = hk_encode();
  if (!enc) return cudaErrorNotSupported;
  const uint64_t plane = (uint64_t)rows * BEOR_TB * nkb_buf * 2;
  cuuint64_t dims[5] = {256, (cuuint64_t)(rows / 16), (cuuint64_t)(nkb_buf * (BEOR_TB / HK_KC)), (cuuint64_t)BEOR_NPART,
                        (cuuint64_t)HK_NS};
  cuuint64_t strides[4] = {512, (cuuint64_t)rows * HK_KC * 2, plane, plane * BEOR_NPART};
  cuuint32_t box[5] = {256, (cuuint32_t)(box_rows / 16), 1, (cuuint32_t)parts, (cuuint32_t)HK_NS};
  cuuint32_t es[5] = {1, 1, 1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// M (packed float64 tiles, lower) = T^H diag(w) T on the tensor cores; the
// caller computes dbar.  Returns cudaErrorLaunchTimeout when a bounded wait
// gave up.
cudaError_t herk_dense_tc(const double2* T, int64_t n_vis, int n, int64_t ld, const double* w, int nt,
                          double2* Mt, cudaStream_t s) {
  const int64_t rows = (int64_t)nt * BEOR_TB;
  const int64_t nkb_total = (n_vis + BEOR_TB - 1) / BEOR_TB;
  const int nkb_buf = (int)std::min<int64_t>(HK_KB_PASS, nkb_total);
  const size_t plane_bytes = (size_t)rows * BEOR_TB * nkb_buf * 2;
  void *planes = nullptr, *exps = nullptr, *ctr = nullptr;
  cudaError_t e = cudaMalloc(&planes, plane_bytes * HK_NPLANE);
  if (e == cudaSuccess) e = cudaMalloc(&exps, sizeof(int32_t) * (size_t)rows * nkb_buf);
  if (e == cudaSuccess) e = cudaMalloc(&ctr, sizeof(int) * 2);   // tile counter, error word
  CUtensorMap ma, mb;
  if (e == cudaSuccess) e = hk_map(&ma, planes, rows, nkb_buf, HK_M, 1);
  if (e == cudaSuccess) e = hk_map(&mb, planes, rows, nkb_buf, HK_N, 2);
  static bool attr = false;
  if (e == cudaSuccess && !attr) {
    e = cudaFuncSetAttribute(herk_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, HK_SMEM);
    attr = e == cudaSuccess;
  }
  int nsm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t ntiles = tri_count(nt) * 2;
  const int grid = (int)std::min<int64_t>(ntiles, std::max(1, nsm));
  int* d_ctr = static_cast<int*>(ctr);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_ctr + 1, 0, sizeof(int), s);
  for (int64_t kb0 = 0; kb0 < nkb_total && e == cudaSuccess; kb0 += nkb_buf) {
    const int nkb = (int)std::min<int64_t>(nkb_buf, nkb_total - kb0);
    herk_slice_kernel<<<dim3(nkb, (unsigned)(rows / 16)), 256, 0, s>>>(
        T, ld, w, n_vis, n, kb0 * BEOR_TB, rows, nkb_buf, static_cast<__nv_bfloat16*>(planes),
        static_cast<int32_t*>(exps));
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(d_ctr, 0, sizeof(int), s);
    if (e == cudaSuccess) {
      herk_tc_kernel<<<grid, HK_THREADS, HK_SMEM, s>>>(ma, mb, static_cast<const int32_t*>(exps), rows, nt, nkb,
                                                       kb0 > 0 ? 1 : 0, Mt, d_ctr, d_ctr + 1);
      e = cudaGetLastError();
    }
  }
  int err = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err, d_ctr + 1, sizeof(int), cudaMemcpyDeviceToHost, s);
  const cudaError_t es = cudaStreamSynchronize(s);   // nothing may still use the buffers
  if (e == cudaSuccess) e = es;
  if (planes) cudaFree(planes);
  if (exps) cudaFree(exps);
  if (ctr) cudaFree(ctr);
  if (e == cudaSuccess && err) e = cudaErrorLaunchTimeout;
  return e;
}

}  // namespace beor
