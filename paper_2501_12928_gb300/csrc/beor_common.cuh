// Shared definitions of the GB300 likelihood library (device and host side).
//
// Matrix storage used by every factorisation kernel ("packed tiles"):
//   an N x N Hermitian matrix is padded to Np = nt*128 and stored as its
//   lower-triangular 128 x 128 tiles (i >= j), tile (i, j) at tile index
//   i*(i+1)/2 + j, each tile column-major (element (r, c) at c*128 + r) so
//   that 32 lanes handling 32 consecutive rows touch 32 consecutive elements.
// Element types: double2 {re, im} (float64 path) or float4
//   {re_hi, re_lo, im_hi, im_lo} (double-float pair per real number; the
//   mixed path's working matrix).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#define BEOR_TB 128                       // tile edge (complex rows / cols)
#define BEOR_TILE_ELEMS (BEOR_TB * BEOR_TB)
#define BEOR_NSLICE 5                     // bf16 slices per real value (mixed path)
#define BEOR_NPART 3                      // parts per slice: imaginary, real, negated imaginary
#define BEOR_NPLANE (BEOR_NPART * BEOR_NSLICE)
// Part order within a slice.  Windows of two consecutive parts are the
// tensor cores' B operands of a complex product C += A B^H computed as real
// products into [re | im] accumulator pairs: (im, re) multiplies Im A
// (re += Ai Bi, im += Ai Br) and (re, -im) multiplies Re A (re += Ar Br,
// im -= Ar Bi).
#define BEOR_PART_IM 0
#define BEOR_PART_RE 1
#define BEOR_PART_NEGIM 2
__host__ __device__ __forceinline__ int slice_plane(int slice, int part) { return slice * BEOR_NPART + part; }

// Tensor-core products of one A slice sa with a two-part B window in the
// slice GEMMs.  Slice pair (sa, t) belongs to level min(sa + t, 3); the
// accumulators are four levels of 128 TMEM columns, each a [re | im] pair of
// 64.  The window's slices t = 0..3-sa feed levels sa..3, contiguous in TMEM
// and in the window, so they take one product per two levels (N = 256 or
// 128, the `main` products); every other pair of the set adds into level 3
// with a product of its own (N = 128, the `extra` products).  Pair sets:
//  * SLICE_PAIRS_FULL5 (5 slices): every pair with sa + t <= 4;
//  * SLICE_PAIRS_REDUCED (5 slices, slice 4 unread): the pairs sa + t <= 3
//    and (2, 2).  The pairs dropped, (0, 4), (1, 3), (3, 1), (4, 0), lie 2^-32
//    below the leading term and have no sign bias off the diagonal; (2, 2)
//    is kept, and tiles on the diagonal of a Hermitian product (P P^H, where
//    |sigma_2|^2 >= 0 would bias the diagonal) use the full set;
//  * SLICE_PAIRS_FULL7 (7 slices, 56-bit operands): every pair with
//    sa + t <= 6; level 3 then rounds about 2^-48 below the leading term.
// Product q < slice_mma_count(sa, set) reads the window from slice
// slice_mma_t(sa, q, set) on and writes N = slice_mma_n(sa, q) columns from
// TMEM column slice_mma_col(sa, q).
enum { SLICE_PAIRS_REDUCED = 0, SLICE_PAIRS_FULL5 = 1, SLICE_PAIRS_FULL7 = 2 };
__host__ __device__ __forceinline__ int slice_mma_main(int sa) { return sa <= 3 ? (5 - sa) / 2 : 0; }
__host__ __device__ __forceinline__ int slice_mma_extra_first(int sa, int set) {
  return set == SLICE_PAIRS_REDUCED ? 2 : (4 - sa > 0 ? 4 - sa : 0);
}
__host__ __device__ __forceinline__ int slice_mma_extras(int sa, int set) {
  if (set == SLICE_PAIRS_REDUCED) return sa == 2 ? 1 : 0;
  if (set == SLICE_PAIRS_FULL5) return sa <= 4 ? 1 : 0;
  return sa <= 3 ? 3 : (sa <= 6 ? 7 - sa : 0);
}
__host__ __device__ __forceinline__ int slice_mma_count(int sa, int set) {
  return slice_mma_main(sa) + slice_mma_extras(sa, set);
}
__host__ __device__ __forceinline__ int slice_mma_t(int sa, int q, int set) {
  return q < slice_mma_main(sa) ? 2 * q : slice_mma_extra_first(sa, set) + (q - slice_mma_main(sa));
}
__host__ __device__ __forceinline__ int slice_mma_col(int sa, int q) {
  return q < slice_mma_main(sa) ? 128 * (sa + 2 * q) : 384;
}
__host__ __device__ __forceinline__ int slice_mma_n(int sa, int q) {
  if (q >= slice_mma_main(sa)) return 128;
  const int left = 4 - sa - 2 * q;   // levels still to cover
  return 128 * (left < 2 ? left : 2);
}

// Element (row, col) of one bf16 slice plane of `rows` rows x 128 columns
// (col = the GEMM's K index).  The plane is stored in the order in which the
// tensor cores read it from shared memory, so that one K-chunk of 16 columns
// for a block of rows is a contiguous range:
//   [K-chunk col/16][8-row group row/8][K half (col/8)%2][row%8][col%8],
// i.e. the canonical K-major layout without swizzle, 8 x 16-byte core
// matrices, the two K halves 128 bytes apart, row groups 256 bytes apart.
__host__ __device__ __forceinline__ int64_t slice_elem_off(int64_t row, int col, int64_t rows) {
  return (int64_t)(col >> 4) * rows * 16 + (row >> 3) * 128 + ((col >> 3) & 1) * 64 + (row & 7) * 8 + (col & 7);
}

namespace beor {

__host__ __device__ inline int64_t tri_index(int i, int j) { return (int64_t)i * (i + 1) / 2 + j; }
__host__ __device__ inline int64_t tri_count(int nt) { return (int64_t)nt * (nt + 1) / 2; }

// One matrix to factorise: prior point b of instrument set s.
struct Prob {
  int n;              // model dimension
  int nt;             // tiles per side
  int set;            // instrument set index
  int b;              // index within the set's batch
  int64_t ws_off;     // element offset of tile (0,0) in the workspace
  int64_t dinv_off;   // element offset (double2) of this problem's inverse diagonal blocks
  int64_t row_off;    // row offset of this problem in the panel-slice and vector buffers
  int k_off;          // block step of the batch at which this problem's step 0 runs (mixed:
                      // max nt - nt, so that all problems end together); kernels given the
                      // batch's step kg work on the problem's step kg - k_off
};

// One instrument (shared by all prior points of the set).
struct SetDesc {
  int n, nt, n_k;
  double lssm_prior_var;
  const double2* M;       // packed tiles (float64), lower
  const float4* Mdf;      // the same as double-float pairs (mixed contexts), or null
  const float4* Mf;       // mixed: all nt x nt tiles (upper ones as conjugate transposes), each
                          // element split exactly m = hi + lo + t: {re hi, re lo, im hi, im lo}
  const float2* Mft;      // ... and {re t, im t}
  const double2* dbar;    // Np
  const int32_t* kbin;    // n
  const double* phi;      // B x n_k (device staging)
};

// One CTA of the float64-accurate residual: row block I of set `set`
// against block columns [j0, j1), for problems p0 .. p0 + nb - 1.
struct RWork {
  int set, I, j0, j1, p0, nb;
};

// Bounds of the per-call device state shared by kernels.
struct Flags {
  int error;              // nonzero: a device-side bounded wait gave up (code)
  int bounds;             // bounds-checked builds: code of the first index check that failed
  int pad[30];
};

// Index checks of the bounds-checked build (-DBEOR_BOUNDS_CHECK), the
// stand-in for a memory checker: a failed check records its code in the
// batch's flags (first failure wins) and the access is skipped -- nothing
// traps.  In the regular build the checks compile away.
#ifdef BEOR_BOUNDS_CHECK
#define BEOR_INBOUNDS(flags, cond, code) \
  ((cond) ? true : (atomicCAS(&(flags)->bounds, 0, (code)), false))
#else
#define BEOR_INBOUNDS(flags, cond, code) true
#endif
// check codes
enum {
  BC_SLICE_ROW = 1, BC_SLICE_OFF = 2, BC_TMA_A = 3, BC_TMA_B = 4, BC_EPI_WS = 5, BC_EPI_EXP = 6,
  BC_DIAG_WS = 7, BC_DIAG_DINV = 8, BC_DIAG_LINV = 9, BC_SOLVE_VEC = 10, BC_RESID_M = 11, BC_RESID_X = 12,
  BC_INIT_WS = 13
};

// Per-problem status values besides 0 (ok), j > 0 (not positive definite at
// column j) and -1 (result outside its tolerance estimate, set at the end):
// -2 marks a prior point with a non-finite phi, found when the prior is
// formed; such a problem is skipped by every later kernel.
constexpr int STATUS_BAD_PHI = -2;
__host__ __device__ __forceinline__ bool prob_skipped(int st) { return st > 0 || st == STATUS_BAD_PHI; }

// ---------------------------------------------------------------------------
// double-float helpers (Dekker / Knuth error-free transformations, FMA based)
// ---------------------------------------------------------------------------
struct dfl { float hi, lo; };

__device__ __forceinline__ dfl df_two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
__device__ __forceinline__ dfl df_fast_two_sum(float a, float b) {
  float s = a + b;
  float e = b - (s - a);
  return {s, e};
}
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  dfl s = df_two_sum(a.hi, b.hi);
  dfl t = df_two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = df_fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return df_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
// a + b*c (b, c double-float)
__device__ __forceinline__ dfl df_fma(dfl a, dfl b, dfl c) { return df_add(a, df_mul(b, c)); }
__device__ __forceinline__ dfl df_from_double(double x) {
  float h = (float)x;
  float l = (float)(x - (double)h);
  return {h, l};
}
__device__ __forceinline__ double df_to_double(dfl a) { return (double)a.hi + (double)a.lo; }

// acc += (ah + al)(bh + bl) to about 2^-48 of the product: the leading
// product split exactly by FMA, first-order terms added to its error, the
// product summed by an error-free two-sum whose error goes to acc.lo (Dot2 of
// Ogita, Rump and Oishi, SIAM J. Sci. Comput. 26 (2005)).
__device__ __forceinline__ void dot2_acc(dfl& acc, float ah, float al, float bh, float bl) {
  const float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  const float s = acc.hi + p;
  const float bb = s - acc.hi;
  acc.lo += ((acc.hi - (s - bb)) + (p - bb)) + e;
  acc.hi = s;
}

// acc += (ah + al + at)(bh + bl): as dot2_acc, with the second-order terms
// al bl and at bh also added to the leading product's error.
__device__ __forceinline__ void dot2_acc3(dfl& acc, float ah, float al, float at, float bh, float bl) {
  const float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  e = fmaf(al, bl, e);
  e = fmaf(at, bh, e);
  const float s = acc.hi + p;
  const float bb = s - acc.hi;
  acc.lo += ((acc.hi - (s - bb)) + (p - bb)) + e;
  acc.hi = s;
}

// The five balanced base-256 digits of X = round((hi + lo) 2^(39 - e)) (a
// double-float with |hi + lo| < 2^e and lo at most half an ulp of hi;
// e <= -1000: all zero), returned as the values sigma_s 2^(-8 s) that the
// slice planes store (exact in bf16): sigma_4 .. sigma_1 in [-128, 127]
// taken from the bottom, sigma_0 the rest (|sigma_0| <= 128).  fp32 and
// 32-bit integer operations only, and no conversion instructions (they run
// on the FP64 pipe): with A, B the scaled parts (exact), A = 2^17 Ah + Al
// with Ah = rint(A 2^-17) (|Ah| < 2^22) and Al exact; round(Al + B) is the
// sum of the two parts' nearest integers, corrected by one step that the sum
// of their exact residuals decides; X = 2^17 Ah + xl.  Nearest integers of
// values below 2^22 and the digits' float values come from adding
// 1.5 * 2^23 (whose float bits then hold the integer in the low word).
__device__ __forceinline__ void balanced_digits5(float hi, float lo, int e, float* dv) {
  if (e <= -1000) {
#pragma unroll
    for (int sl = 0; sl < BEOR_NSLICE; ++sl) dv[sl] = 0.0f;
    return;
  }
  const float magic = 12582912.0f;   // 1.5 * 2^23, float bits 0x4B400000
  const int k = 39 - e, k1 = k >> 1, k2 = k - k1;   // 2^k as two exact factors
  const float f1 = __int_as_float((k1 + 127) << 23), f2 = __int_as_float((k2 + 127) << 23);
  const float A = __fmul_rn(__fmul_rn(hi, f1), f2), B = __fmul_rn(__fmul_rn(lo, f1), f2);
  const float t1 = __fmaf_rn(A, 0x1p-17f, magic);
  const int ah = __float_as_int(t1) - 0x4B400000;
  const float al = __fmaf_rn(-__fsub_rn(t1, magic), 131072.0f, A);   // A - 2^17 Ah, exact
  const float t2 = __fadd_rn(al, magic), t3 = __fadd_rn(B, magic);
  const float d = __fadd_rn(__fsub_rn(al, __fsub_rn(t2, magic)), __fsub_rn(B, __fsub_rn(t3, magic)));
  const int xl = (__float_as_int(t2) - 0x4B400000) + (__float_as_int(t3) - 0x4B400000) + (d > 0.5f ? 1 : 0) -
                 (d < -0.5f ? 1 : 0);
  // digits from the bottom: X mod 256 is xl mod 256, and after two digits
  // the rest fits 32 bits
  int dg[BEOR_NSLICE];
  dg[4] = ((xl + 128) & 255) - 128;
  const int y = (xl - dg[4]) >> 8;
  dg[3] = ((y + 128) & 255) - 128;
  int x = 2 * ah + ((y - dg[3]) >> 8);
  dg[2] = ((x + 128) & 255) - 128;
  x = (x - dg[2]) >> 8;
  dg[1] = ((x + 128) & 255) - 128;
  dg[0] = (x - dg[1]) >> 8;
#pragma unroll
  for (int sl = 0; sl < BEOR_NSLICE; ++sl)
    dv[sl] = __fmul_rn(__fsub_rn(__int_as_float(dg[sl] + 0x4B400000), magic),
                       __int_as_float((127 - 8 * sl) << 23));
}

}  // namespace beor
