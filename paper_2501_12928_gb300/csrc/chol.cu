// Blocked right-looking complex Cholesky of Sigma = M + Phi^-1 for a batch of
// problems, the triangular solves for abar = Sigma^-1 dbar, and the lnL
// assembly (lnL = -1/2 log|Phi| - 1/2 log|Sigma| + 1/2 dbar^H abar).
//
// Kernels here serve both precisions:
//  * prior / init:  Phi^-1 from phi (one amplitude per k bin, Eq. for P(k_i)),
//                   log|Phi|, and the working matrix W = M + diag(Phi^-1);
//  * diag:          float64 factorisation of the 128 x 128 diagonal block,
//                   log|Sigma| accumulation, status, and its inverse (float64;
//                   on the fp32 pipe, with bf16 slices, on the mixed path);
//  * panel/trail:   float64 tile GEMMs (the float64 comparator path);
//  * solve:         blocked forward / backward substitution;
//  * lnl:           q = Re(dbar^H abar), or its residual-corrected form, and lnL.
#include <algorithm>
#include <cmath>

#include "beor_common.cuh"
#include "beor_internal.h"

namespace beor {

// --------------------------------------------------------------------------
// workspace element access
// --------------------------------------------------------------------------
__device__ __forceinline__ double2 ws_load(const double2* p) { return *p; }
__device__ __forceinline__ double2 ws_load(const float4* p) {
  float4 v = *p;
  return make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
}
__device__ __forceinline__ void ws_store(double2* p, double2 v) { *p = v; }
__device__ __forceinline__ void ws_store(float4* p, double2 v) {
  float rh = (float)v.x, ih = (float)v.y;
  *p = make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
}

__device__ __forceinline__ void tile_of(int64_t t, int& I, int& J) {
  int i = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
  while ((int64_t)i * (i + 1) / 2 > t) --i;
  while ((int64_t)(i + 1) * (i + 2) / 2 <= t) ++i;
  I = i;
  J = (int)(t - (int64_t)i * (i + 1) / 2);
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    red[32] = s;
  }
  __syncthreads();
  return red[32];
}

// --------------------------------------------------------------------------
// prior: Phi^-1 per row, log|Phi| per problem, reset of the per-problem sums
// --------------------------------------------------------------------------
__global__ void prior_kernel(BatchView v) {
  const int p = blockIdx.x;
  const Prob pr = v.prob[p];
  const SetDesc sd = v.sets[pr.set];
  const double* phi = sd.phi + (int64_t)pr.b * sd.n_k;
  const double ln10 = 2.302585092994045684;
  __shared__ double red[33];
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  // a non-finite phi (possible only for device-memory input, which the host
  // does not read) marks the point; every later kernel skips it
  for (int i = threadIdx.x; i < sd.n_k; i += blockDim.x)
    if (!isfinite(phi[i])) s_bad = 1;
  double acc = 0.0;
  const int np = pr.nt * BEOR_TB;
  for (int j = threadIdx.x; j < np; j += blockDim.x) {
    double inv = 1.0;
    if (j < pr.n) {
      int kb = sd.kbin[j];
      if (kb >= 0) {
        double ph = phi[kb];
        inv = exp10(-ph);
        acc += ph * ln10;
      } else {
        inv = 1.0 / sd.lssm_prior_var;
        acc += log(sd.lssm_prior_var);
      }
    }
    v.phi_inv[pr.row_off + j] = inv;
  }
  double tot = block_sum(acc, red);   // its barriers also order the writes of s_bad
  if (threadIdx.x == 0) {
    v.logdet_phi[p] = tot;
    v.logdet_sigma[p] = 0.0;
    v.status[p] = s_bad ? STATUS_BAD_PHI : 0;
    v.resid[p] = 0.0;
  }
}

// grid (problem, tile): problems fastest, so the problems of one instrument
// read each tile of M from L2 rather than from HBM.  Float64 path: M as is.
__global__ void __launch_bounds__(256) init_ws_f64_kernel(BatchView v) {
  const int p = blockIdx.x;
  const Prob pr = v.prob[p];
  const SetDesc sd = v.sets[pr.set];
  const int64_t ntiles = tri_count(pr.nt);
  for (int64_t t = blockIdx.y; t < ntiles; t += gridDim.y) {
    int I, J;
    tile_of(t, I, J);
    if (!BEOR_INBOUNDS(v.flags, pr.ws_off + (t + 1) * BEOR_TILE_ELEMS <= v.ws_elems, BC_INIT_WS)) return;
    const double2* __restrict__ src = sd.M + t * BEOR_TILE_ELEMS;
    double2* __restrict__ dst = reinterpret_cast<double2*>(v.ws) + pr.ws_off + t * BEOR_TILE_ELEMS;
    const double* pinv = v.phi_inv + pr.row_off + (int64_t)I * BEOR_TB;
    for (int e = threadIdx.x; e < BEOR_TILE_ELEMS; e += blockDim.x) {
      double2 m = src[e];
      if (I == J && (e % BEOR_TB) == (e / BEOR_TB)) {
        m.x += pinv[e % BEOR_TB];
        m.y = 0.0;
      }
      dst[e] = m;
    }
  }
}

// Mixed path: copy the double-float M; the diagonal gets Phi^-1 in
// double-float arithmetic (no float64 instruction per element).
__global__ void __launch_bounds__(256) init_ws_df_kernel(BatchView v) {
  const int p = blockIdx.x;
  const Prob pr = v.prob[p];
  const SetDesc sd = v.sets[pr.set];
  const int64_t ntiles = tri_count(pr.nt);
  for (int64_t t = blockIdx.y; t < ntiles; t += gridDim.y) {
    int I, J;
    tile_of(t, I, J);
    if (!BEOR_INBOUNDS(v.flags, pr.ws_off + (t + 1) * BEOR_TILE_ELEMS <= v.ws_elems, BC_INIT_WS)) return;
    const float4* __restrict__ src = sd.Mdf + t * BEOR_TILE_ELEMS;
    float4* __restrict__ dst = reinterpret_cast<float4*>(v.ws) + pr.ws_off + t * BEOR_TILE_ELEMS;
    for (int e = threadIdx.x; e < BEOR_TILE_ELEMS; e += blockDim.x) dst[e] = src[e];
    if (I != J) continue;                 // uniform per CTA
    __syncthreads();                      // the copy of every diagonal element has landed
    if (threadIdx.x < BEOR_TB) {
      const int r = threadIdx.x;
      const int e = r * BEOR_TB + r;
      const float4 m = src[e];
      const dfl w = df_add(dfl{m.x, m.y}, df_from_double(v.phi_inv[pr.row_off + (int64_t)I * BEOR_TB + r]));
      dst[e] = make_float4(w.hi, w.lo, 0.0f, 0.0f);
    }
  }
}

cudaError_t launch_prior_init(const BatchView& v, bool mixed, cudaStream_t s) {
  prior_kernel<<<v.P, 256, 0, s>>>(v);
  dim3 g(v.P, (unsigned)std::min<int64_t>(tri_count(v.max_nt), 65535));
  if (mixed)
    init_ws_df_kernel<<<g, 256, 0, s>>>(v);
  else
    init_ws_f64_kernel<<<g, 256, 0, s>>>(v);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// diagonal block: float64 Cholesky, log-det, status, and the inverse of the
// block (float64; on the mixed path formed on the fp32 pipe) with, on the
// mixed path, the bf16 slices of its rows: value = 2^(e-7) sum_s sigma_s
// 2^(-8 s), sigma_s integers with |sigma_s| <= 128.
// --------------------------------------------------------------------------
#define DG_PACK (BEOR_TB * (BEOR_TB + 1) / 2)
__device__ __forceinline__ int pk(int i, int j) { return i * (i + 1) / 2 + j; }

// Complex Dot2 accumulation of a b into c (c[0] + c[1] the real part,
// c[2] + c[3] the imaginary part): a an element of L as double-float with
// its third terms at, b a double-float element.
__device__ __forceinline__ void cmac_l(dfl* c, float4 a, float2 at, float4 b) {
  dot2_acc3(c[0], a.x, a.y, at.x, b.x, b.y);
  dot2_acc3(c[1], -a.z, -a.w, -at.y, b.z, b.w);
  dot2_acc3(c[2], a.x, a.y, at.x, b.z, b.w);
  dot2_acc3(c[3], a.z, a.w, at.y, b.x, b.y);
}
__device__ __forceinline__ dfl df_add_quick(dfl x, dfl y) {
  const dfl t = df_two_sum(x.hi, y.hi);
  return dfl{t.hi, t.lo + (x.lo + y.lo)};
}
// Barrier of the 128 threads (four warps) of group id - 1.
__device__ __forceinline__ void group_sync(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }

// Block row I of the diagonal block's inverse, in place (512 threads): the
// rows 32 I .. 32 I + 31 of L (packed, double-float plus third terms Lt),
// every earlier block row and the diagonal block Linv_II already inverted.
// Output (J, r, c) of the block row goes to thread o % 512 (o = 1024 J +
// 32 r + c): lanes take consecutive columns, so a warp reads one element of
// L (a broadcast) and 32 consecutive elements of Linv per step.
template <int I>
__device__ __forceinline__ void inv_block_row(float4* Af, const float2* Lt, int tid) {
  constexpr int NQ = 2 * I;   // outputs per thread
  dfl xr[NQ], xi[NQ];
  // X_IJ = sum_{m = 32 J + c}^{32 I - 1} L[i][m] Linv[m][jj] (Linv_JJ is lower triangular)
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int o = tid + 512 * q, J = o >> 10, r = (o >> 5) & 31, c = o & 31;
    const int i = 32 * I + r, jj = 32 * J + c;
    dfl a[4] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
    for (int m = jj; m < 32 * I; ++m) cmac_l(a, Af[pk(i, m)], Lt[pk(i, m)], Af[pk(m, jj)]);
    xr[q] = df_add_quick(a[0], a[1]);
    xi[q] = df_add_quick(a[2], a[3]);
  }
  __syncthreads();   // every read of block row I (as L) is done
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int o = tid + 512 * q, J = o >> 10, r = (o >> 5) & 31, c = o & 31;
    const dfl ur = df_fast_two_sum(xr[q].hi, xr[q].lo), ui = df_fast_two_sum(xi[q].hi, xi[q].lo);
    Af[pk(32 * I + r, 32 * J + c)] = make_float4(ur.hi, ur.lo, ui.hi, ui.lo);
  }
  __syncthreads();   // X in place of L_IJ
  // Linv_IJ = -Linv_II X_IJ = -sum_{t <= r} Linv[i][32 I + t] X[32 I + t][jj]
  const float2 zero = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int o = tid + 512 * q, J = o >> 10, r = (o >> 5) & 31, c = o & 31;
    const int i = 32 * I + r, jj = 32 * J + c;
    dfl a[4] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
    for (int t = 0; t <= r; ++t) cmac_l(a, Af[pk(i, 32 * I + t)], zero, Af[pk(32 * I + t, jj)]);
    xr[q] = df_add_quick(a[0], a[1]);
    xi[q] = df_add_quick(a[2], a[3]);
  }
  __syncthreads();   // every read of X is done
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int o = tid + 512 * q, J = o >> 10, r = (o >> 5) & 31, c = o & 31;
    const dfl ur = df_fast_two_sum(xr[q].hi, xr[q].lo), ui = df_fast_two_sum(xi[q].hi, xi[q].lo);
    Af[pk(32 * I + r, 32 * J + c)] = make_float4(-ur.hi, -ur.lo, -ui.hi, -ui.lo);
  }
  __syncthreads();
}

template <typename WS>
__global__ void __launch_bounds__(512) diag_kernel(BatchView v, int kg, int mixed) {
  extern __shared__ double2 dsm[];
  double2* A = dsm;                    // packed lower 128x128
  double2* col = dsm + DG_PACK;        // 128
  __shared__ int s_fail;
  __shared__ double s_rinv;            // 1 / L_jj of the current column
  const int p = blockIdx.x;
  const Prob pr = v.prob[p];
  const int k = kg - pr.k_off;   // this problem's block step
  if (k < 0 || k >= pr.nt) return;
  if (v.status[p] != 0) return;
  if (!BEOR_INBOUNDS(v.flags, pr.ws_off + (tri_index(k, k) + 1) * BEOR_TILE_ELEMS <= v.ws_elems, BC_DIAG_WS) ||
      !BEOR_INBOUNDS(v.flags, pr.dinv_off + (int64_t)(k + 1) * DG_PACK <= v.dinv_elems, BC_DIAG_DINV) ||
      !BEOR_INBOUNDS(v.flags, !mixed || (int64_t)(p + 1) * BEOR_TB <= (int64_t)v.P * BEOR_TB, BC_DIAG_LINV))
    return;
  WS* ws = reinterpret_cast<WS*>(v.ws) + pr.ws_off + tri_index(k, k) * BEOR_TILE_ELEMS;
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int e = tid; e < BEOR_TILE_ELEMS; e += nthr) {
    int r = e % BEOR_TB, c = e / BEOR_TB;
    if (r >= c) A[pk(r, c)] = ws_load(ws + e);
  }
  if (tid == 0) s_fail = 0;
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31, nwarp = nthr >> 5;
  // Right-looking Cholesky, two columns per pass (rank-2 updates): half the
  // barriers and shared-memory round trips of one column per pass, with the
  // same operations in the same order as the rank-1 sequence (identical
  // results).  Thread 0 takes both pivots: L_jj, column j's element in row
  // j+1 and its update of a_{j+1,j+1}, then L_{j+1,j+1}.
  double2* col2 = col + BEOR_TB;   // column j+1 (this space later holds the mixed path's third terms of L)
  __shared__ double s_rinv2;
  for (int j = 0; j < BEOR_TB; j += 2) {
    if (tid == 0) {
      const double d = A[pk(j, j)].x;
      if (!(d > 0.0) || !isfinite(d)) {
        s_fail = k * BEOR_TB + j + 1;
      } else {
        const double l = sqrt(d);
        A[pk(j, j)] = make_double2(l, 0.0);
        const double rinv = 1.0 / l;
        s_rinv = rinv;
        double2 a = A[pk(j + 1, j)];
        a.x *= rinv;
        a.y *= rinv;
        A[pk(j + 1, j)] = a;
        col[j + 1] = a;
        double2 x = A[pk(j + 1, j + 1)];
        x.x = fma(-a.x, a.x, fma(-a.y, a.y, x.x));
        x.y = fma(-a.y, a.x, fma(a.x, a.y, x.y));
        const double d2 = x.x;
        if (!(d2 > 0.0) || !isfinite(d2)) {
          s_fail = k * BEOR_TB + j + 2;
        } else {
          const double l2 = sqrt(d2);
          A[pk(j + 1, j + 1)] = make_double2(l2, 0.0);
          s_rinv2 = 1.0 / l2;
        }
      }
    }
    __syncthreads();
    if (s_fail) break;
    const double inv = s_rinv, inv2 = s_rinv2;
    const double2 lj1 = col[j + 1];   // L_{j+1,j}
    // columns j and j+1 below the pair: scale column j, apply it to column
    // j+1 (the rank-1 step's update of those elements), scale column j+1
    for (int i = j + 2 + tid; i < BEOR_TB; i += nthr) {
      double2 a = A[pk(i, j)];
      a.x *= inv;
      a.y *= inv;
      A[pk(i, j)] = a;
      col[i] = a;
      double2 b = A[pk(i, j + 1)];
      b.x = fma(-a.x, lj1.x, fma(-a.y, lj1.y, b.x));
      b.y = fma(-a.y, lj1.x, fma(a.x, lj1.y, b.y));
      b.x *= inv2;
      b.y *= inv2;
      A[pk(i, j + 1)] = b;
      col2[i] = b;
    }
    __syncthreads();
    // rank-2 update of the trailing lower triangle (rows and columns >= j+2):
    // A_il -= L_ij conj(L_lj), then -= L_i,j+1 conj(L_l,j+1); the triangle's
    // elements are dealt out in order, so every lane has work
    {
      const int nt2 = BEOR_TB - 2 - j;
      const int total = nt2 * (nt2 + 1) / 2;
      for (int e = tid; e < total; e += nthr) {
        int a = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
        while (a * (a + 1) / 2 > e) --a;
        while ((a + 1) * (a + 2) / 2 <= e) ++a;
        const int i = j + 2 + a, l = j + 2 + (e - a * (a + 1) / 2);
        const double2 ai = col[i], al = col[l], bi = col2[i], bl = col2[l];
        double2 x = A[pk(i, l)];
        x.x = fma(-ai.x, al.x, fma(-ai.y, al.y, x.x));
        x.y = fma(-ai.y, al.x, fma(ai.x, al.y, x.y));
        x.x = fma(-bi.x, bl.x, fma(-bi.y, bl.y, x.x));
        x.y = fma(-bi.y, bl.x, fma(bi.x, bl.y, x.y));
        A[pk(i, l)] = x;
      }
    }
    __syncthreads();
  }
  if (s_fail) {
    if (tid == 0) v.status[p] = s_fail;
    return;
  }
  // log-determinant contribution, 2 sum ln L_jj over the real rows, in parallel
  {
    __shared__ double red[32];
    double ldp = 0.0;
    if (tid < BEOR_TB && k * BEOR_TB + tid < pr.n) ldp = 2.0 * log(A[pk(tid, tid)].x);
    for (int o = 16; o > 0; o >>= 1) ldp += __shfl_xor_sync(0xffffffffu, ldp, o);
    if (lane == 0) red[warp] = ldp;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < nwarp; ++w) s += red[w];
      v.logdet_sigma[p] += s;
    }
  }
  // L_kk back to the workspace tile (upper part zero)
  for (int e = tid; e < BEOR_TILE_ELEMS; e += nthr) {
    int r = e % BEOR_TB, c = e / BEOR_TB;
    ws_store(ws + e, r >= c ? A[pk(r, c)] : make_double2(0.0, 0.0));
  }
  __syncthreads();
  if (!mixed) {
    // in-place inverse, row by row: Linv[i][j] = -(sum_{m=j}^{i-1} L[i][m] Linv[m][j]) / L[i][i];
    // four threads share each dot product (thread = 4 j + part)
    const int jj = tid >> 2, part = tid & 3;
    for (int i = 0; i < BEOR_TB; ++i) {
      if (tid == 0) s_rinv = 1.0 / A[pk(i, i)].x;
      double sr = 0.0, si = 0.0;
      if (jj < i) {
        for (int m = jj + part; m < i; m += 4) {
          const double2 a = A[pk(i, m)], b = A[pk(m, jj)];
          sr = fma(a.x, b.x, fma(-a.y, b.y, sr));
          si = fma(a.x, b.y, fma(a.y, b.x, si));
        }
      }
      sr += __shfl_xor_sync(0xffffffffu, sr, 1);
      si += __shfl_xor_sync(0xffffffffu, si, 1);
      sr += __shfl_xor_sync(0xffffffffu, sr, 2);
      si += __shfl_xor_sync(0xffffffffu, si, 2);
      __syncthreads();
      if (jj < i && part == 0) {
        const double inv = s_rinv;
        A[pk(i, jj)] = make_double2(-sr * inv, -si * inv);
      }
      if (tid == 0) A[pk(i, i)] = make_double2(s_rinv, 0.0);
      __syncthreads();
    }
    double2* dinv = v.dinv + pr.dinv_off + (int64_t)k * DG_PACK;
    for (int e = tid; e < DG_PACK; e += nthr) dinv[e] = A[e];
    return;
  }
  // Mixed path: the inverse feeds the 40-bit panel slices and the
  // double-float solves only, so it is formed on the fp32 pipe instead of in
  // float64, whose rate on this GPU is 1/64 of fp32.  L is split exactly into
  // three floats per component: {re hi, re lo, im hi, im lo} in place (16
  // bytes per element either way) and the third terms in Lt.  Each product
  // L[i][m] Linv[m][j] keeps the terms down to 2^-48 of its leading part
  // (Dot2 accumulation); Linv itself is held as double-float.
  float4* Af = reinterpret_cast<float4*>(A);
  float2* Lt = reinterpret_cast<float2*>(col + BEOR_TB);
  for (int e = tid; e < DG_PACK; e += nthr) {
    const double2 a = A[e];
    const float rh = (float)a.x, ih = (float)a.y;
    const double rd = a.x - (double)rh, id = a.y - (double)ih;
    const float rl = (float)rd, il = (float)id;
    Af[e] = make_float4(rh, rl, ih, il);
    Lt[e] = make_float2((float)(rd - (double)rl), (float)(id - (double)il));
  }
  __shared__ dfl s_invs[BEOR_TB];      // 1 / L_ii for every row, formed in parallel
  __syncthreads();                     // the split of L is complete
  if (tid < BEOR_TB) {
    const float4 d = Af[pk(tid, tid)];
    s_invs[tid] = df_from_double(1.0 / ((double)d.x + (double)d.y + (double)Lt[pk(tid, tid)].x));
  }
  __syncthreads();
  // Blocked inverse (four 32-row blocks): the diagonal blocks are inverted
  // row by row, one block per 128 threads at once; then block row I = 1..3
  // takes X_IJ = sum_{M=J}^{I-1} L_IM Linv_MJ for every J < I and
  // Linv_IJ = -Linv_II X_IJ.  32 dependent row steps and 12 barriers instead
  // of 128 row steps with two barriers each; the operations per element are
  // those of the row recursion, with the division by L_ii of each step
  // replaced by the product with the inverted diagonal block.
  {
    const int g = tid >> 7, lt = tid & 127, jl = lt >> 2, part = lt & 3;
    const int jj = 32 * g + jl;
    for (int il = 0; il < 32; ++il) {
      const int i = 32 * g + il;
      dfl c[4] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
      if (jl < il)
        for (int m = jj + part; m < i; m += 4) cmac_l(c, Af[pk(i, m)], Lt[pk(i, m)], Af[pk(m, jj)]);
      dfl sr = df_add_quick(c[0], c[1]), si = df_add_quick(c[2], c[3]);
#pragma unroll
      for (int o = 1; o <= 2; o <<= 1) {
        sr = df_add_quick(sr, dfl{__shfl_xor_sync(0xffffffffu, sr.hi, o), __shfl_xor_sync(0xffffffffu, sr.lo, o)});
        si = df_add_quick(si, dfl{__shfl_xor_sync(0xffffffffu, si.hi, o), __shfl_xor_sync(0xffffffffu, si.lo, o)});
      }
      group_sync(1 + g);   // every read of row i (as L) is done
      if (jl < il && part == 0) {
        const dfl inv = s_invs[i];
        const dfl qr = df_mul(df_fast_two_sum(sr.hi, sr.lo), inv);
        const dfl qi = df_mul(df_fast_two_sum(si.hi, si.lo), inv);
        Af[pk(i, jj)] = make_float4(-qr.hi, -qr.lo, -qi.hi, -qi.lo);
      }
      if (lt == 0) Af[pk(i, i)] = make_float4(s_invs[i].hi, s_invs[i].lo, 0.0f, 0.0f);
      group_sync(1 + g);   // row i of Linv is complete
    }
  }
  __syncthreads();
  inv_block_row<1>(Af, Lt, tid);
  inv_block_row<2>(Af, Lt, tid);
  inv_block_row<3>(Af, Lt, tid);
  double2* dinv = v.dinv + pr.dinv_off + (int64_t)k * DG_PACK;
  for (int e = tid; e < DG_PACK; e += nthr) {
    const float4 f = Af[e];
    dinv[e] = make_double2((double)f.x + (double)f.y, (double)f.z + (double)f.w);
  }
  // slices of Linv rows (B operand of the panel product L_ik = A_ik Linv^H):
  // balanced base-256 digits of round(x * 2^(39 - e)), x = hi + lo (scaled
  // exactly by a power of two, rounded once)
  const int64_t lrows = (int64_t)v.P * BEOR_TB;
  const int64_t ps = lrows * BEOR_TB;   // one plane; plane index slice_plane(slice, part)
  for (int c = warp; c < BEOR_TB; c += nwarp) {
    float mx = 0.0f;
    for (int m = lane; m <= c; m += 32) {
      const float4 a = Af[pk(c, m)];
      mx = fmaxf(mx, fmaxf(fabsf(a.x), fabsf(a.z)));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int e = mx > 0.0f ? ilogbf(mx) + 1 : -1000;
    const int64_t row = (int64_t)p * BEOR_TB + c;
    if (lane == 0) v.linv_exp[row] = e;
    for (int m = lane; m < BEOR_TB; m += 32) {
      const float4 a = m <= c ? Af[pk(c, m)] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
      for (int part = 0; part < 2; ++part) {
        const float hi = part ? a.z : a.x, lo = part ? a.w : a.y;
        float dv[BEOR_NSLICE];
        balanced_digits5(hi, lo, e, dv);
        __nv_bfloat16* dst = v.linv_sl + slice_elem_off(row, m, lrows);
#pragma unroll
        for (int sl = 0; sl < BEOR_NSLICE; ++sl) {
          const float d = dv[sl];
          if (part == 0) {
            dst[slice_plane(sl, BEOR_PART_RE) * ps] = __float2bfloat16_rn(d);
          } else {
            dst[slice_plane(sl, BEOR_PART_IM) * ps] = __float2bfloat16_rn(d);
            dst[slice_plane(sl, BEOR_PART_NEGIM) * ps] = __float2bfloat16_rn(-d);
          }
        }
      }
    }
  }
}

cudaError_t launch_diag(const BatchView& v, int k, bool mixed, cudaStream_t s, int prio) {
  // packed block, one column, and (mixed) the third float terms of L
  const size_t smem = sizeof(double2) * (DG_PACK + BEOR_TB) + sizeof(float2) * DG_PACK;
  static bool init = false;
  if (!init) {
    cudaFuncSetAttribute(diag_kernel<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(diag_kernel<float4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    init = true;
  }
  if (mixed) return launch_prio(diag_kernel<float4>, dim3(v.P), dim3(512), smem, s, prio, v, k, 1);
  return launch_prio(diag_kernel<double2>, dim3(v.P), dim3(512), smem, s, prio, v, k, 0);
}

// --------------------------------------------------------------------------
// float64 panel: L_ik = A_ik Linv_kk^H for i > k (rows split in two halves)
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(256) panel_f64_kernel(BatchView v, int kg) {
  extern __shared__ double2 psm[];
  double2* xs = psm;                  // [128 m][64 r]
  double2* ys = psm + 128 * 64;       // [16 m][128 c]
  const int p = blockIdx.y;
  const Prob pr = v.prob[p];
  const int k = kg - pr.k_off;
  const int i = k + 1 + (blockIdx.x >> 1);
  if (k < 0 || i >= pr.nt || v.status[p] != 0) return;
  const int r0 = (blockIdx.x & 1) * 64;
  double2* tile = reinterpret_cast<double2*>(v.ws) + pr.ws_off + tri_index(i, k) * BEOR_TILE_ELEMS;
  const double2* linv = v.dinv + pr.dinv_off + (int64_t)k * DG_PACK;
  for (int e = threadIdx.x; e < 128 * 64; e += 256) {
    int m = e / 64, r = e % 64;
    xs[e] = tile[m * BEOR_TB + r0 + r];
  }
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double ar[4][8], ai[4][8];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) ar[a][b] = ai[a][b] = 0.0;
  for (int m0 = 0; m0 < BEOR_TB; m0 += 16) {
    __syncthreads();
    for (int e = threadIdx.x; e < 16 * 128; e += 256) {
      int mm = e / 128, c = e % 128, m = m0 + mm;
      ys[e] = m <= c ? linv[pk(c, m)] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    for (int mm = 0; mm < 16; ++mm) {
      double2 x[4], y[8];
#pragma unroll
      for (int a = 0; a < 4; ++a) x[a] = xs[(m0 + mm) * 64 + ty * 4 + a];
#pragma unroll
      for (int b = 0; b < 8; ++b) y[b] = ys[mm * 128 + tx * 8 + b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          // x * conj(y)
          ar[a][b] = fma(x[a].x, y[b].x, fma(x[a].y, y[b].y, ar[a][b]));
          ai[a][b] = fma(x[a].y, y[b].x, fma(-x[a].x, y[b].y, ai[a][b]));
        }
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      int r = r0 + ty * 4 + a, c = tx * 8 + b;
      tile[c * BEOR_TB + r] = make_double2(ar[a][b], ai[a][b]);
    }
}

cudaError_t launch_panel_f64(const BatchView& v, int k, cudaStream_t s) {
  int nblk = 2 * (v.max_nt - 1 - k);
  if (nblk <= 0) return cudaSuccess;
  const size_t smem = sizeof(double2) * (128 * 64 + 16 * 128);
  static bool init = false;
  if (!init) {
    cudaFuncSetAttribute(panel_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    init = true;
  }
  panel_f64_kernel<<<dim3(nblk, v.P), 256, smem, s>>>(v, k);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// float64 trailing update: A_ij -= L_ik L_jk^H, k < j <= i, 64 x 64 sub-tiles
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(256) trail_f64_kernel(BatchView v, int kg) {
  __shared__ double2 xs[16][64];
  __shared__ double2 ys[16][64];
  const int p = blockIdx.y;
  const Prob pr = v.prob[p];
  const int k = kg - pr.k_off;
  const int T = k < 0 ? 0 : pr.nt - k - 1;
  const int64_t t = blockIdx.x >> 2;
  if (T <= 0 || t >= tri_count(T) || v.status[p] != 0) return;
  const int si = (blockIdx.x >> 1) & 1, sj = blockIdx.x & 1;
  int a, b;
  tile_of(t, a, b);
  const int i = k + 1 + a, j = k + 1 + b;
  if (i == j && si < sj) return;   // upper part of a diagonal tile is never read
  double2* ws = reinterpret_cast<double2*>(v.ws) + pr.ws_off;
  const double2* X = ws + tri_index(i, k) * BEOR_TILE_ELEMS + si * 64;
  const double2* Y = ws + tri_index(j, k) * BEOR_TILE_ELEMS + sj * 64;
  double2* C = ws + tri_index(i, j) * BEOR_TILE_ELEMS;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double ar[4][4], ai[4][4];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int w = 0; w < 4; ++w) ar[q][w] = ai[q][w] = 0.0;
  for (int m0 = 0; m0 < BEOR_TB; m0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      int mm = e / 64, r = e % 64;
      xs[mm][r] = X[(m0 + mm) * BEOR_TB + r];
      ys[mm][r] = Y[(m0 + mm) * BEOR_TB + r];
    }
    __syncthreads();
#pragma unroll 4
    for (int mm = 0; mm < 16; ++mm) {
      double2 x[4], y[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        x[q] = xs[mm][ty * 4 + q];
        y[q] = ys[mm][tx * 4 + q];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          ar[q][w] = fma(x[q].x, y[w].x, fma(x[q].y, y[w].y, ar[q][w]));
          ai[q][w] = fma(x[q].y, y[w].x, fma(-x[q].x, y[w].y, ai[q][w]));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      int r = si * 64 + ty * 4 + q, c = sj * 64 + tx * 4 + w;
      double2 cv = C[c * BEOR_TB + r];
      cv.x -= ar[q][w];
      cv.y -= ai[q][w];
      C[c * BEOR_TB + r] = cv;
    }
}

cudaError_t launch_trail_f64(const BatchView& v, int k, cudaStream_t s) {
  int T = v.max_nt - k - 1;
  if (T <= 0) return cudaSuccess;
  int64_t nblk = tri_count(T) * 4;
  trail_f64_kernel<<<dim3((unsigned)nblk, v.P), 256, 0, s>>>(v, k);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// Triangular solves with the factor: out = L^-H L^-1 rhs, blocked by 128.
// One launch per block step covers every problem: CTA (i, p) applies the
// update of block row i with the block just solved; the CTA that completes
// the next block row also applies that block's float64 inverse, so a step's
// critical path is one tile update plus one 128 x 128 float64 matvec.
// Off-diagonal products: float64 for the float64 path, double-float (fp32
// pairs) for the mixed path's double-float factor.
// --------------------------------------------------------------------------
struct CAcc {          // complex accumulator
  double2 d;           // float64 path
  dfl re, im;          // double-float path: hi = error-free running sum, lo = its accumulated errors
};

__device__ __forceinline__ void cacc_zero(CAcc& a) {
  a.d = make_double2(0.0, 0.0);
  a.re = dfl{0.0f, 0.0f};
  a.im = dfl{0.0f, 0.0f};
}
// a += L * y (conj_l: a += conj(L) * y); y given as double2 and as double-float pairs
__device__ __forceinline__ void cacc_mac(CAcc& a, const double2* L, double2 y, dfl, dfl, bool conj_l) {
  const double2 l = *L;
  const double li = conj_l ? -l.y : l.y;
  a.d.x = fma(l.x, y.x, fma(-li, y.y, a.d.x));
  a.d.y = fma(l.x, y.y, fma(li, y.x, a.d.y));
}
__device__ __forceinline__ void cacc_mac(CAcc& a, const float4* L, double2, dfl yr, dfl yi, bool conj_l) {
  const float4 l = *L;
  const float lih = conj_l ? -l.z : l.z, lil = conj_l ? -l.w : l.w;
  // re += lr yr - li yi, im += lr yi + li yr
  dot2_acc(a.re, l.x, l.y, yr.hi, yr.lo);
  dot2_acc(a.re, -lih, -lil, yi.hi, yi.lo);
  dot2_acc(a.im, l.x, l.y, yi.hi, yi.lo);
  dot2_acc(a.im, lih, lil, yr.hi, yr.lo);
}
__device__ __forceinline__ double2 cacc_get(const CAcc& a, const double2*) { return a.d; }
__device__ __forceinline__ double2 cacc_get(const CAcc& a, const float4*) {
  return make_double2((double)a.re.hi + (double)a.re.lo, (double)a.im.hi + (double)a.im.lo);
}
__device__ __forceinline__ void cacc_add(CAcc& a, const CAcc& b) {
  a.d.x += b.d.x;
  a.d.y += b.d.y;
  dfl s = df_two_sum(a.re.hi, b.re.hi);
  a.re = dfl{s.hi, s.lo + (a.re.lo + b.re.lo)};
  s = df_two_sum(a.im.hi, b.im.hi);
  a.im = dfl{s.hi, s.lo + (a.im.lo + b.im.lo)};
}

// sum over the 8 lanes of an aligned lane octet (xor 1, 2, 4)
__device__ __forceinline__ void cacc_reduce8(CAcc& a, const double2*) {
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    a.d.x += __shfl_xor_sync(0xffffffffu, a.d.x, o);
    a.d.y += __shfl_xor_sync(0xffffffffu, a.d.y, o);
  }
}
__device__ __forceinline__ void cacc_reduce8(CAcc& a, const float4*) {
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    CAcc b;
    b.d = make_double2(0.0, 0.0);
    b.re.hi = __shfl_xor_sync(0xffffffffu, a.re.hi, o);
    b.re.lo = __shfl_xor_sync(0xffffffffu, a.re.lo, o);
    b.im.hi = __shfl_xor_sync(0xffffffffu, a.im.hi, o);
    b.im.lo = __shfl_xor_sync(0xffffffffu, a.im.lo, o);
    cacc_add(a, b);
  }
}

// y_blk = Linv (or Linv^H when herm) * r_blk, float64; 128 threads of the CTA
__device__ __forceinline__ void diag_apply(const double2* __restrict__ li, const double2* rk, double2* out,
                                           bool herm) {
  const int t = threadIdx.x;
  if (t >= BEOR_TB) return;
  double sr = 0.0, si = 0.0;
  if (!herm) {
    for (int m = 0; m <= t; ++m) {
      const double2 a = li[pk(t, m)], q = rk[m];
      sr = fma(a.x, q.x, fma(-a.y, q.y, sr));
      si = fma(a.x, q.y, fma(a.y, q.x, si));
    }
  } else {
    for (int m = t; m < BEOR_TB; ++m) {
      const double2 a = li[pk(m, t)], q = rk[m];
      sr = fma(a.x, q.x, fma(a.y, q.y, sr));
      si = fma(a.x, q.y, fma(-a.y, q.x, si));
    }
  }
  out[t] = make_double2(sr, si);
}

// Forward step k (k = -1: only y_0).  CTA (i, p), i = k+1 .. nt-1:
// r_i -= L_ik y_k; the CTA with i == k+1 then sets y_{k+1} = Linv r_{k+1}.
template <typename WS>
__global__ void __launch_bounds__(256) fwd_step_kernel(BatchView v, int kg, const double2* __restrict__ rhs) {
  __shared__ double2 yk[BEOR_TB];
  __shared__ dfl ykr[BEOR_TB], yki[BEOR_TB];
  __shared__ CAcc part[BEOR_TB];
  __shared__ double2 rk[BEOR_TB];
  const int p = blockIdx.y;
  const Prob pr = v.prob[p];
  const int k = kg - pr.k_off;   // this problem's step (-1: start)
  if (k < -1) return;
  const int i = k + 1 + blockIdx.x;
  if (i >= pr.nt || prob_skipped(v.status[p])) return;
  if (!BEOR_INBOUNDS(v.flags, pr.row_off + (int64_t)pr.nt * BEOR_TB <= v.rows, BC_SOLVE_VEC) ||
      !BEOR_INBOUNDS(v.flags, k < 0 || pr.ws_off + (tri_index(i, k) + 1) * BEOR_TILE_ELEMS <= v.ws_elems, BC_SOLVE_VEC))
    return;
  const int tid = threadIdx.x;
  double2* r = v.vec_t + pr.row_off;
  double2* y = v.vec_y + pr.row_off;
  if (k < 0) {
    // initial step: r = rhs for all rows of block 0 handled here, other rows by their own CTAs
    if (tid < BEOR_TB) r[i * BEOR_TB + tid] = rhs[pr.row_off + i * BEOR_TB + tid];
    if (i != 0) return;
    __syncthreads();
    if (tid < BEOR_TB) rk[tid] = r[tid];
    __syncthreads();
    diag_apply(v.dinv + pr.dinv_off, rk, yk, false);
    __syncthreads();
    if (tid < BEOR_TB) y[tid] = yk[tid];
    return;
  }
  if (tid < BEOR_TB) {
    const double2 q = y[k * BEOR_TB + tid];
    yk[tid] = q;
    ykr[tid] = df_from_double(q.x);
    yki[tid] = df_from_double(q.y);
  }
  __syncthreads();
  const WS* t = reinterpret_cast<const WS*>(v.ws) + pr.ws_off + tri_index(i, k) * BEOR_TILE_ELEMS;
  const int row = tid & 127, half = tid >> 7;
  CAcc a;
  cacc_zero(a);
#pragma unroll 4
  for (int m = half * 64; m < half * 64 + 64; ++m)
    cacc_mac(a, t + m * BEOR_TB + row, yk[m], ykr[m], yki[m], false);
  if (half) part[row] = a;
  __syncthreads();
  if (!half) {
    cacc_add(a, part[row]);
    const double2 s = cacc_get(a, t);
    double2 cur = r[i * BEOR_TB + row];
    cur.x -= s.x;
    cur.y -= s.y;
    r[i * BEOR_TB + row] = cur;
    rk[row] = cur;
  }
  if (i != k + 1) return;
  __syncthreads();
  diag_apply(v.dinv + pr.dinv_off + (int64_t)i * DG_PACK, rk, yk, false);
  __syncthreads();
  if (tid < BEOR_TB) y[i * BEOR_TB + tid] = yk[tid];
}

// Backward step k (k = nt: only x_{nt-1} for each problem).  CTA (i, p),
// i = 0 .. k-1: r_i -= L_ki^H x_k; the CTA with i == k-1 then sets
// x_{k-1} = Linv^H r_{k-1}.  Steps run from the largest nt down; problems
// with fewer tiles join when k < their nt.
template <typename WS>
__global__ void __launch_bounds__(256) bwd_step_kernel(BatchView v, int k, double2* __restrict__ out) {
  __shared__ double2 xk[BEOR_TB];
  __shared__ dfl xkr[BEOR_TB], xki[BEOR_TB];
  __shared__ double2 rk[BEOR_TB];
  const int p = blockIdx.y;
  const Prob pr = v.prob[p];
  if (prob_skipped(v.status[p])) return;
  if (!BEOR_INBOUNDS(v.flags, pr.row_off + (int64_t)pr.nt * BEOR_TB <= v.rows, BC_SOLVE_VEC)) return;
  const int tid = threadIdx.x;
  double2* r = v.vec_t + pr.row_off;
  double2* x = out + pr.row_off;
  const double2* y = v.vec_y + pr.row_off;
  if (k >= pr.nt) {
    // start: r = y; the CTA for the last block applies Linv^H
    const int i = blockIdx.x;
    if (i >= pr.nt) return;
    if (tid < BEOR_TB) r[i * BEOR_TB + tid] = y[i * BEOR_TB + tid];
    if (k != pr.nt || i != pr.nt - 1) return;
    __syncthreads();
    if (tid < BEOR_TB) rk[tid] = r[i * BEOR_TB + tid];
    __syncthreads();
    diag_apply(v.dinv + pr.dinv_off + (int64_t)i * DG_PACK, rk, xk, true);
    __syncthreads();
    if (tid < BEOR_TB) x[i * BEOR_TB + tid] = xk[tid];
    return;
  }
  const int i = blockIdx.x;
  if (i >= k) return;
  if (tid < BEOR_TB) {
    const double2 q = x[k * BEOR_TB + tid];
    xk[tid] = q;
    xkr[tid] = df_from_double(q.x);
    xki[tid] = df_from_double(q.y);
  }
  __syncthreads();
  // r_i[c] -= sum_m conj(L_ki[m][c]) x_k[m]: tile (k, i) is column-major, so
  // column c is 128 contiguous elements.  A warp takes 4 columns at a time,
  // 8 lanes per column on interleaved m (each load instruction reads four
  // 128-byte segments), and sums the 8 partials by shuffles.
  const WS* t = reinterpret_cast<const WS*>(v.ws) + pr.ws_off + tri_index(k, i) * BEOR_TILE_ELEMS;
  const int warp = tid >> 5, lane = tid & 31, cl = lane >> 3, mo = lane & 7;
#pragma unroll 1
  for (int it = 0; it < 4; ++it) {
    const int c = warp * 16 + it * 4 + cl;
    CAcc a;
    cacc_zero(a);
#pragma unroll 4
    for (int u = 0; u < 16; ++u) {
      const int m = mo + 8 * u;
      cacc_mac(a, t + c * BEOR_TB + m, xk[m], xkr[m], xki[m], true);
    }
    cacc_reduce8(a, t);
    if (mo == 0) {
      const double2 sv = cacc_get(a, t);
      double2 cur = r[i * BEOR_TB + c];
      cur.x -= sv.x;
      cur.y -= sv.y;
      r[i * BEOR_TB + c] = cur;
      rk[c] = cur;
    }
  }
  if (i != k - 1) return;
  __syncthreads();
  diag_apply(v.dinv + pr.dinv_off + (int64_t)i * DG_PACK, rk, xk, true);
  __syncthreads();
  if (tid < BEOR_TB) x[i * BEOR_TB + tid] = xk[tid];
}


// Forward step k of y = L^-1 rhs (k = -1: r = rhs and y_0), every problem.
cudaError_t launch_fwd_step(const BatchView& v, bool mixed, const double2* rhs, int k, cudaStream_t s, int prio) {
  const int nb = k < 0 ? v.max_nt : v.max_nt - k - 1;
  if (nb <= 0) return cudaSuccess;
  if (mixed) return launch_prio(fwd_step_kernel<float4>, dim3(nb, v.P), dim3(256), 0, s, prio, v, k, rhs);
  return launch_prio(fwd_step_kernel<double2>, dim3(nb, v.P), dim3(256), 0, s, prio, v, k, rhs);
}

// out = L^-H y (y in vec_y), every problem.
template <typename WS>
static cudaError_t bwd_impl(const BatchView& v, double2* out, cudaStream_t s) {
  const int nt = v.max_nt;
  bwd_step_kernel<WS><<<dim3(nt, v.P), 256, 0, s>>>(v, nt, out);
  for (int k = nt - 1; k >= 1; --k) {
    // problems whose last block is k-1 (nt_p == k) start here
    bwd_step_kernel<WS><<<dim3(k, v.P), 256, 0, s>>>(v, k, out);
  }
  return cudaGetLastError();
}

cudaError_t launch_bwd(const BatchView& v, bool mixed, double2* out, cudaStream_t s) {
  return mixed ? bwd_impl<float4>(v, out, s) : bwd_impl<double2>(v, out, s);
}

cudaError_t launch_solve_fwd(const BatchView& v, bool mixed, const double2* rhs, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  for (int k = -1; k + 1 < v.max_nt && e == cudaSuccess; ++k) e = launch_fwd_step(v, mixed, rhs, k, s, 0);
  return e;
}

cudaError_t launch_solve(const BatchView& v, bool mixed, const double2* rhs, double2* out, cudaStream_t s) {
  cudaError_t e = launch_solve_fwd(v, mixed, rhs, s);
  return e == cudaSuccess ? launch_bwd(v, mixed, out, s) : e;
}

int solve_launch_count(int max_nt) { return 2 * max_nt; }

// --------------------------------------------------------------------------
// dbar of each problem's set into the right-hand-side vector
// --------------------------------------------------------------------------
__global__ void copy_dbar_kernel(BatchView v) {
  const int p = blockIdx.x;
  const Prob pr = v.prob[p];
  const SetDesc sd = v.sets[pr.set];
  const int np = pr.nt * BEOR_TB;
  for (int j = threadIdx.x; j < np; j += blockDim.x) v.vec_b[pr.row_off + j] = sd.dbar[j];
}

cudaError_t launch_copy_dbar(const BatchView& v, cudaStream_t s) {
  copy_dbar_kernel<<<v.P, 256, 0, s>>>(v);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// lnL = -1/2 log|Phi| - 1/2 log|Sigma| + 1/2 Re(dbar^H x)
// --------------------------------------------------------------------------
// lnL = -1/2 log|Phi| - 1/2 log|Sigma| + 1/2 q (Eq. for the marginal
// likelihood of the power spectrum).  corr = 0: q = Re(dbar^H x), x the
// (refined) solution.  corr = 1: q from the first solution x~ of the
// approximate factor, corrected with the float64 residual r = dbar - Sigma x~
// (vec_r) and y = L~^-1 r (vec_y):
//   q = dbar^H x~ + x~^H r + r^H Sigma^-1 r,  r^H Sigma^-1 r ~ |y|^2,
// exact but for the last term's factor error, about eta |y|^2 with
// eta ~ sqrt(|y|^2 / q) the relative error of x~ in the Sigma norm.
__global__ void lnl_kernel(BatchView v, int corr) {
  const int p = blockIdx.x;
  const Prob pr = v.prob[p];
  const SetDesc sd = v.sets[pr.set];
  __shared__ double red[33];
  double acc = 0.0, t = 0.0;
  for (int j = threadIdx.x; j < pr.n; j += blockDim.x) {
    double2 d = sd.dbar[j], x = v.vec_x[pr.row_off + j];
    acc += d.x * x.x + d.y * x.y;
    if (corr) {
      const double2 r = v.vec_r[pr.row_off + j], y = v.vec_y[pr.row_off + j];
      acc += x.x * r.x + x.y * r.y;
      t += y.x * y.x + y.y * y.y;
    }
  }
  double q = block_sum(acc, red);
  __syncthreads();
  if (corr) t = block_sum(t, red);
  if (threadIdx.x == 0) {
    if (corr) {
      q += t;
      const double eta = q > 0.0 ? sqrt(t / q) : INFINITY;
      v.resid[p] = eta;
      // estimated remaining error of q above 1e-2 (5e-3 in lnL): flag
      if (v.status[p] == 0 && !(eta * t <= 1e-2)) v.status[p] = -1;
    }
    v.q[p] = q;
    if (v.status[p] == STATUS_BAD_PHI)
      v.lnl[p] = __longlong_as_double(0x7ff8000000000000ll);   // NaN: no likelihood for a non-finite phi
    else if (v.status[p] > 0)
      v.lnl[p] = -INFINITY;
    else
      v.lnl[p] = -0.5 * v.logdet_phi[p] - 0.5 * v.logdet_sigma[p] + 0.5 * q;
  }
}

cudaError_t launch_lnl(const BatchView& v, cudaStream_t s, int corr) {
  lnl_kernel<<<v.P, 256, 0, s>>>(v, corr);
  return cudaGetLastError();
}

}  // namespace beor
