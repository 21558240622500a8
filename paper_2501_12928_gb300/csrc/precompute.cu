// One-off precompute of M = T^H N^-1 T and dbar = T^H N^-1 d in float64.
//
// Sec. "Running BayesEoR": the instrument model forward-models the data; the
// likelihood needs the data-space products T^H N^-1 T and T^H N^-1 d once
// per instrument, after which every prior point only changes a diagonal.
// Two routes:
//  * dense:    M = T^H diag(w) T directly from T (n_vis x n row-major): on
//              the FP64 pipe (float64 contexts) or as seven-digit bf16 slice
//              products on the tensor cores (mixed contexts, herk_tc.cu),
//  * factored: T[(f,tb),(c,x)] = A_f[tb,c] W[f,x] gives
//              G_f = A_f^H diag(w_f) A_f and
//              M[(c,x),(c',x')] = sum_f conj(W[f,x]) W[f,x'] G_f[c,c'],
//    which never forms T.
// Both are float64 throughout (the refinement of the solve and the
// log-determinant need an M accurate far beyond float32).
#include "beor_common.cuh"
#include "beor_internal.h"

namespace beor {

// ---------------------------------------------------------------------------
// C = X^H diag(w) X, X: K x n complex (row-major, leading dimension ldx),
// batched over blockIdx.z with element strides.  Each CTA computes one
// 64 x 64 sub-tile of a lower 128-tile.  mode 0: write packed tiles (the
// factorisation layout); mode 1: write a dense row-major Hermitian matrix.
// ---------------------------------------------------------------------------
constexpr int HK_T = 64;   // sub-tile edge
constexpr int HK_K = 16;   // K rows per smem stage

__global__ void __launch_bounds__(256) herk_f64_kernel(const double2* __restrict__ X, int64_t ldx,
                                                       int64_t x_batch_stride, const double* __restrict__ w,
                                                       int64_t w_batch_stride, int64_t K, int n, int nt,
                                                       double2* __restrict__ C, int64_t ldc,
                                                       int64_t c_batch_stride, int mode) {
  __shared__ double2 sa[HK_K][HK_T];
  __shared__ double2 sb[HK_K][HK_T];
  const int bz = blockIdx.z;
  X += bz * x_batch_stride;
  w += bz * w_batch_stride;
  C += bz * c_batch_stride;
  // which 128-tile (I, J), I >= J, and which 64 sub-tile
  int t = blockIdx.x >> 2, sub = blockIdx.x & 3;
  int I = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((int64_t)I * (I + 1) / 2 > t) --I;
  while ((int64_t)(I + 1) * (I + 2) / 2 <= t) ++I;
  int J = t - I * (I + 1) / 2;
  const int si = sub >> 1, sj = sub & 1;
  const int r0 = I * BEOR_TB + si * HK_T;     // rows of C  <- columns of X (conj side)
  const int c0 = J * BEOR_TB + sj * HK_T;     // cols of C  <- columns of X
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double ar[4][4], ai[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) ar[a][b] = ai[a][b] = 0.0;
  const bool skip = (r0 >= n) || (c0 >= n);
  if (!skip) {
    for (int64_t k0 = 0; k0 < K; k0 += HK_K) {
      for (int e = threadIdx.x; e < HK_K * HK_T; e += 256) {
        int kk = e / HK_T, cc = e % HK_T;
        int64_t k = k0 + kk;
        double2 va = make_double2(0.0, 0.0), vb = make_double2(0.0, 0.0);
        if (k < K) {
          if (r0 + cc < n) va = X[k * ldx + r0 + cc];
          if (c0 + cc < n) {
            vb = X[k * ldx + c0 + cc];
            double ww = w[k];
            vb.x *= ww;
            vb.y *= ww;
          }
        }
        sa[kk][cc] = va;
        sb[kk][cc] = vb;
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < HK_K; ++kk) {
        double2 a[4], b[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          a[q] = sa[kk][ty * 4 + q];
          b[q] = sb[kk][tx * 4 + q];
        }
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            // conj(a) * b
            ar[p][q] = fma(a[p].x, b[q].x, fma(a[p].y, b[q].y, ar[p][q]));
            ai[p][q] = fma(a[p].x, b[q].y, fma(-a[p].y, b[q].x, ai[p][q]));
          }
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int r = r0 + ty * 4 + p, c = c0 + tx * 4 + q;
      double vr = ar[p][q], vi = ai[p][q];
      if (r >= n || c >= n) { vr = 0.0; vi = 0.0; }
      if (r == c) vi = 0.0;
      if (mode == 0) {
        int64_t off = tri_index(I, J) * BEOR_TILE_ELEMS + (int64_t)(c - J * BEOR_TB) * BEOR_TB + (r - I * BEOR_TB);
        C[off] = make_double2(vr, vi);
      } else if (r < n && c < n) {
        C[(int64_t)r * ldc + c] = make_double2(vr, vi);
        if (I != J) C[(int64_t)c * ldc + r] = make_double2(vr, -vi);
      }
    }
}

// u[b][j] = sum_k conj(X_b[k, j]) w_b[k] d_b[k]  (atomic accumulation over K chunks)
__global__ void xh_w_d_kernel(const double2* __restrict__ X, int64_t ldx, int64_t x_batch_stride,
                              const double* __restrict__ w, const double2* __restrict__ d,
                              int64_t vec_batch_stride, int64_t K, int n, int64_t kchunk,
                              double2* __restrict__ u, int64_t u_batch_stride) {
  const int bz = blockIdx.z;
  X += bz * x_batch_stride;
  w += bz * vec_batch_stride;
  d += bz * vec_batch_stride;
  u += bz * u_batch_stride;
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  int64_t k0 = blockIdx.y * kchunk, k1 = min(K, k0 + kchunk);
  double sr = 0.0, si = 0.0;
  for (int64_t k = k0; k < k1; ++k) {
    double2 x = X[k * ldx + j];
    double2 dd = d[k];
    double ww = w[k];
    double dr = dd.x * ww, di = dd.y * ww;
    sr = fma(x.x, dr, fma(x.y, di, sr));
    si = fma(x.x, di, fma(-x.y, dr, si));
  }
  atomicAdd(&u[j].x, sr);
  atomicAdd(&u[j].y, si);
}

// Structured M: M[(c,x),(c',x')] = sum_f conj(W[f,x]) W[f,x'] G[f][c][c'] into packed tiles.
__global__ void assemble_M_kernel(const double2* __restrict__ G, const double2* __restrict__ W, int nf,
                                  int ncells, int nx, int n, int nt, double2* __restrict__ Mt) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t total = tri_count(nt) * BEOR_TILE_ELEMS;
  if (e >= total) return;
  int64_t t = e / BEOR_TILE_ELEMS;
  int w_in = (int)(e % BEOR_TILE_ELEMS);
  int I = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((int64_t)I * (I + 1) / 2 > t) --I;
  while ((int64_t)(I + 1) * (I + 2) / 2 <= t) ++I;
  int J = (int)(t - (int64_t)I * (I + 1) / 2);
  int r = I * BEOR_TB + (w_in % BEOR_TB);
  int c = J * BEOR_TB + (w_in / BEOR_TB);
  double vr = 0.0, vi = 0.0;
  if (r < n && c < n) {
    int cr = r / nx, xr = r % nx, cc = c / nx, xc = c % nx;
    for (int f = 0; f < nf; ++f) {
      double2 wa = W[f * nx + xr], wb = W[f * nx + xc];
      // conj(wa) * wb
      double pr = wa.x * wb.x + wa.y * wb.y;
      double pi = wa.x * wb.y - wa.y * wb.x;
      double2 g = G[((int64_t)f * ncells + cr) * ncells + cc];
      vr = fma(pr, g.x, fma(-pi, g.y, vr));
      vi = fma(pr, g.y, fma(pi, g.x, vi));
    }
    if (r == c) vi = 0.0;
  }
  Mt[e] = make_double2(vr, vi);
}

// dbar[(c,x)] = sum_f conj(W[f,x]) u[f][c]
__global__ void assemble_dbar_kernel(const double2* __restrict__ u, const double2* __restrict__ W, int nf,
                                     int ncells, int nx, int n, int np, double2* __restrict__ dbar) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= np) return;
  double vr = 0.0, vi = 0.0;
  if (j < n) {
    int c = j / nx, x = j % nx;
    for (int f = 0; f < nf; ++f) {
      double2 ww = W[f * nx + x], uu = u[(int64_t)f * ncells + c];
      vr = fma(ww.x, uu.x, fma(ww.y, uu.y, vr));
      vi = fma(ww.x, uu.y, fma(-ww.y, uu.x, vi));
    }
  }
  dbar[j] = make_double2(vr, vi);
}

// x -> (hi, lo) float pairs with hi + lo = x to ~48 bits (once per precompute)
__global__ void split_df_kernel(const double2* __restrict__ M, int64_t n, float4* __restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = M[e];
    const float rh = (float)v.x, ih = (float)v.y;
    out[e] = make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
  }
}

// ---------------------------------------------------------------------------
// host launchers
// Tile (I, J) of the full square, element (r, c) column-major: M_IJ for
// I > J, conj(M_JI)^T for I < J, the Hermitian mirror of the stored lower
// part inside diagonal tiles; entries beyond n are zero.  Each component
// is split m = hi + lo + t exactly (hi = fl(m), lo = fl(m - hi), and the
// remainder has at most 53 - 48 bits).
__global__ void split_full_kernel(const double2* __restrict__ M, int n, int nt, float4* __restrict__ hl,
                                  float2* __restrict__ tt) {
  const int I = blockIdx.x / nt, J = blockIdx.x % nt;
  const int64_t out0 = (int64_t)blockIdx.x * BEOR_TILE_ELEMS;
  for (int e = threadIdx.x; e < BEOR_TILE_ELEMS; e += blockDim.x) {
    const int c = e / BEOR_TB, r = e % BEOR_TB;
    const int gr = I * BEOR_TB + r, gc = J * BEOR_TB + c;
    double2 m = make_double2(0.0, 0.0);
    if (gr < n && gc < n) {
      if (gr >= gc) {
        m = M[tri_index(I, J) * BEOR_TILE_ELEMS + (int64_t)c * BEOR_TB + r];
      } else {
        const double2 u = M[tri_index(J, I) * BEOR_TILE_ELEMS + (int64_t)r * BEOR_TB + c];
        m = make_double2(u.x, -u.y);
      }
    }
    const float rh = (float)m.x, ih = (float)m.y;
    const double rd = m.x - (double)rh, id = m.y - (double)ih;
    const float rl = (float)rd, il = (float)id;
    hl[out0 + e] = make_float4(rh, rl, ih, il);
    tt[out0 + e] = make_float2((float)(rd - (double)rl), (float)(id - (double)il));
  }
}

cudaError_t split_full_triple(const double2* M, int n, int nt, float4* hl, float2* t, cudaStream_t s) {
  split_full_kernel<<<nt * nt, 256, 0, s>>>(M, n, nt, hl, t);
  return cudaGetLastError();
}

cudaError_t split_double_float(const double2* M, int64_t n, float4* out, cudaStream_t s) {
  split_df_kernel<<<1024, 256, 0, s>>>(M, n, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
cudaError_t precompute_dense(const double2* T, int64_t n_vis, int n, int64_t ld, const double* w,
                             const double2* d, int nt, double2* Mt, double2* dbar, cudaStream_t s, bool tc) {
  cudaError_t e;
  if (tc) {
    e = herk_dense_tc(T, n_vis, n, ld, w, nt, Mt, s);   // seven-digit slice products (herk_tc.cu)
  } else {
    dim3 grid((unsigned)(tri_count(nt) * 4), 1, 1);
    herk_f64_kernel<<<grid, 256, 0, s>>>(T, ld, 0, w, 0, n_vis, n, nt, Mt, 0, 0, 0);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  cudaMemsetAsync(dbar, 0, sizeof(double2) * (size_t)nt * BEOR_TB, s);
  int64_t kchunk = 4096;
  dim3 g2((n + 255) / 256, (unsigned)((n_vis + kchunk - 1) / kchunk), 1);
  xh_w_d_kernel<<<g2, 256, 0, s>>>(T, ld, 0, w, d, 0, n_vis, n, kchunk, dbar, 0);
  return cudaGetLastError();
}

cudaError_t precompute_factored(const double2* A, const double2* W, int nf, int64_t ntb, int ncells,
                                int nx, const double* w, const double2* d, int n, int nt,
                                double2* G_scratch, double2* u_scratch, double2* Mt, double2* dbar,
                                cudaStream_t s) {
  int ntc = (ncells + BEOR_TB - 1) / BEOR_TB;
  dim3 grid((unsigned)(tri_count(ntc) * 4), 1, (unsigned)nf);
  herk_f64_kernel<<<grid, 256, 0, s>>>(A, ncells, ntb * ncells, w, ntb, ntb, ncells, ntc, G_scratch,
                                        ncells, (int64_t)ncells * ncells, 1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int64_t total = tri_count(nt) * BEOR_TILE_ELEMS;
  assemble_M_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(G_scratch, W, nf, ncells, nx, n, nt, Mt);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  cudaMemsetAsync(u_scratch, 0, sizeof(double2) * (size_t)nf * ncells, s);
  int64_t kchunk = 2048;
  dim3 g2((ncells + 255) / 256, (unsigned)((ntb + kchunk - 1) / kchunk), (unsigned)nf);
  xh_w_d_kernel<<<g2, 256, 0, s>>>(A, ncells, ntb * ncells, w, d, ntb, ntb, ncells, kchunk, u_scratch, ncells);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int np = nt * BEOR_TB;
  assemble_dbar_kernel<<<(np + 255) / 256, 256, 0, s>>>(u_scratch, W, nf, ncells, nx, n, np, dbar);
  return cudaGetLastError();
}

}  // namespace beor
