// Instrument model from its geometry (beor_set_instrument_desc).
//
// Sec. "Running BayesEoR": the instrument model is the primary beam and the
// uv sampling of each baseline.  It is built here in the factored form the
// precompute uses, T[(f, tb), (c, x)] = A_f[tb, c] W[f, x]:
//  * A_f = NUDFT_f . diag(beam) . F_uv: the model's uv cells (i_u, i_v), the
//    (0, 0) cell removed, mapped to an n_pix x n_pix sky grid by the unitary
//    inverse 2-D DFT F_uv, weighted by an achromatic Gaussian beam, and
//    observed by each baseline / time sample at frequency f
//    (exp(-2 pi i (u l + v m)), uv in wavelengths at f);
//  * W = [E | S]: the unitary inverse eta-DFT over the channels (eta index
//    -nf/2 .. nf/2 - 1) and the foreground power laws (f / f0)^-beta, each
//    column scaled to unit 2-norm;
//  * the k-bin map: |k| = sqrt(i_u^2 + i_v^2 + eta^2) in grid units for the
//    EoR modes, n_k log-spaced shells between their smallest and largest
//    |k| (the maximum goes to the last shell), -1 for foreground modes.
// The uv cell size is set so that the longest baseline reaches the grid
// edge at the top channel of nf_grid channels (sub-bands of one band share
// the band's grid), and the sky grid spans one field of view, 1 / du.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/beor.h"

namespace {

constexpr double kC = 299792458.0;
constexpr double kTwoPi = 6.283185307179586476925;

// BF[p][c] = beam(l_p, m_p) exp(2 pi i (px_p i_u + py_p i_v) / n_pix) / n_pix,
// pixel p = py * n_pix + px.
__global__ void beam_uvdft_kernel(int npx, const int* __restrict__ cells, int ncells, double dl, double two_s2,
                                  double2* __restrict__ BF) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)npx * npx * ncells) return;
  const int c = (int)(e % ncells);
  const int p = (int)(e / ncells);
  const int py = p / npx, px = p % npx;
  const double x = px - npx / 2.0, y = py - npx / 2.0;
  const double l = x * dl, m = y * dl;
  const double beam = exp(-(l * l + m * m) / two_s2);
  double s, co;
  sincospi(2.0 * (x * cells[2 * c] + y * cells[2 * c + 1]) / npx, &s, &co);
  BF[e] = make_double2(beam * co / npx, beam * s / npx);
}

// A[f][tb][c] = sum_p exp(-2 pi i (u l_p + v m_p)) BF[p][c]: one CTA per
// (f, tb) row, the row's phase factors in shared memory, threads over c.
__global__ void __launch_bounds__(256) nudft_kernel(int npx, int ncells, int64_t ntb, const double* __restrict__ uv_m,
                                                    const double* __restrict__ freqs, double dl,
                                                    const double2* __restrict__ BF, double2* __restrict__ A) {
  extern __shared__ double2 ph[];   // npx * npx
  const int64_t row = blockIdx.x;   // f * ntb + tb
  const int f = (int)(row / ntb);
  const int64_t tb = row % ntb;
  const double scale = freqs[f] / kC;
  const double u = uv_m[2 * tb] * scale, v = uv_m[2 * tb + 1] * scale;
  const int np = npx * npx;
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    const double l = (p % npx - npx / 2.0) * dl, m = (p / npx - npx / 2.0) * dl;
    double s, co;
    sincospi(-2.0 * (u * l + v * m), &s, &co);
    ph[p] = make_double2(co, s);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < ncells; c += blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int p = 0; p < np; ++p) {
      const double2 a = ph[p], b = BF[(int64_t)p * ncells + c];
      re = fma(a.x, b.x, fma(-a.y, b.y, re));
      im = fma(a.x, b.y, fma(a.y, b.x, im));
    }
    A[row * ncells + c] = make_double2(re, im);
  }
}

struct DevArr {
  void* p = nullptr;
  ~DevArr() {
    if (p) cudaFree(p);
  }
};

int fail(cudaError_t e) {
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? BEOR_ENOMEM : BEOR_ECUDA;
}

}  // namespace

extern "C" int beor_set_instrument_desc(beor_ctx* ctx, const beor_instrument_desc* d) {
  if (!ctx || !d) return BEOR_EINVAL;
  if (d->nu < 3 || d->nu % 2 == 0 || d->nu > 255 || d->nf < 1 || d->n_pix < 2 || d->n_pix > 256 || d->n_bl < 1 ||
      d->n_t < 1 || d->n_k < 1 || d->n_lssm < 0 || d->n_lssm > 8 || d->nf_grid < 0)
    return BEOR_EINVAL;
  if (!d->bl_enu_m || !d->hour_angle_rad || (d->n_lssm > 0 && !d->lssm_beta)) return BEOR_EINVAL;
  if (!(d->f0_hz > 0.0) || !(d->df_hz >= 0.0) || (d->nf > 1 && !(d->df_hz > 0.0)) || !(d->beam_fwhm_rad > 0.0) ||
      !std::isfinite(d->latitude_rad) || !(d->lssm_prior_var > 0.0))
    return BEOR_EINVAL;
  const int h = (d->nu - 1) / 2;
  const int nf = d->nf, npx = d->n_pix, nx = d->nf + d->n_lssm;
  const int nf_grid = d->nf_grid ? d->nf_grid : nf;
  const int64_t ntb = (int64_t)d->n_t * d->n_bl;
  // cells: i_v outer, i_u inner, (0, 0) removed
  std::vector<int> cells;
  for (int iv = -h; iv <= h; ++iv)
    for (int iu = -h; iu <= h; ++iu)
      if (iu || iv) {
        cells.push_back(iu);
        cells.push_back(iv);
      }
  const int ncells = (int)cells.size() / 2;
  // uv cell from the longest baseline at the grid's top channel; sky grid = one field of view
  double bmax = 0.0;
  for (int b = 0; b < d->n_bl; ++b) bmax = std::max(bmax, std::hypot(d->bl_enu_m[3 * b], d->bl_enu_m[3 * b + 1]));
  const double f_top = d->f0_hz + d->df_hz * (nf_grid - 1);
  const double du = bmax * f_top / kC / h;
  if (!(du > 0.0) || !std::isfinite(du)) return BEOR_EINVAL;
  const double fov = 1.0 / du, dl = fov / npx;
  const double sig = d->beam_fwhm_rad / (2.0 * std::sqrt(2.0 * std::log(2.0)));
  // baseline uv (metres) per time sample of a drift scan pointed at the zenith at transit
  const double sl = std::sin(d->latitude_rad), cl = std::cos(d->latitude_rad);
  std::vector<double> uv((size_t)ntb * 2), freqs(nf);
  for (int t = 0; t < d->n_t; ++t) {
    const double H = d->hour_angle_rad[t], sh = std::sin(H), ch = std::cos(H);
    for (int b = 0; b < d->n_bl; ++b) {
      const double E = d->bl_enu_m[3 * b], N = d->bl_enu_m[3 * b + 1], U = d->bl_enu_m[3 * b + 2];
      const double X = -sl * N + cl * U, Y = E, Z = cl * N + sl * U;
      const size_t r = (size_t)t * d->n_bl + b;
      uv[2 * r] = sh * X + ch * Y;
      uv[2 * r + 1] = -sl * ch * X + sl * sh * Y + cl * Z;
    }
  }
  for (int f = 0; f < nf; ++f) freqs[f] = d->f0_hz + d->df_hz * f;
  // spectral basis W = [E | S]
  std::vector<beor_c128> W((size_t)nf * nx);
  for (int f = 0; f < nf; ++f)
    for (int x = 0; x < nf; ++x) {
      const double eta = x - nf / 2;
      const double arg = kTwoPi * (f * eta) / nf;
      W[(size_t)f * nx + x] = beor_c128{std::cos(arg) / std::sqrt((double)nf), std::sin(arg) / std::sqrt((double)nf)};
    }
  for (int q = 0; q < d->n_lssm; ++q) {
    double nrm = 0.0;
    for (int f = 0; f < nf; ++f) nrm += std::pow(freqs[f] / d->f0_hz, -2.0 * d->lssm_beta[q]);
    nrm = std::sqrt(nrm);
    for (int f = 0; f < nf; ++f)
      W[(size_t)f * nx + nf + q] = beor_c128{std::pow(freqs[f] / d->f0_hz, -d->lssm_beta[q]) / nrm, 0.0};
  }
  // k bins
  const int64_t n = (int64_t)ncells * nx;
  std::vector<double> kmag(n, 0.0);
  std::vector<int32_t> kbin(n, -1);
  double kmin = INFINITY, kmax = 0.0;
  for (int c = 0; c < ncells; ++c)
    for (int x = 0; x < nf; ++x) {
      const double eta = x - nf / 2, iu = cells[2 * c], iv = cells[2 * c + 1];
      const double k = std::sqrt(iu * iu + iv * iv + eta * eta);
      kmag[(size_t)c * nx + x] = k;
      kmin = std::min(kmin, k);
      kmax = std::max(kmax, k);
    }
  std::vector<double> edges(d->n_k + 1);
  for (int i = 0; i <= d->n_k; ++i) edges[i] = kmin * std::pow(kmax / kmin, (double)i / d->n_k);
  for (int c = 0; c < ncells; ++c)
    for (int x = 0; x < nf; ++x) {
      const double k = kmag[(size_t)c * nx + x];
      // the shell k_i <= |k| < k_(i+1); the largest |k| in the last shell
      const int b = (int)(std::upper_bound(edges.begin(), edges.end(), k) - edges.begin()) - 1;
      kbin[(size_t)c * nx + x] = std::min(std::max(b, 0), d->n_k - 1);
    }
  // A on the device
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(cudaErrorUnknown);
  DevArr dcells, dBF, duv, dfreq, dA;
  cudaError_t e;
  const size_t nbf = (size_t)npx * npx * ncells;
  if ((e = cudaMalloc(&dcells.p, sizeof(int) * cells.size())) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&dBF.p, sizeof(double2) * nbf)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&duv.p, sizeof(double) * uv.size())) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&dfreq.p, sizeof(double) * nf)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&dA.p, sizeof(double2) * (size_t)nf * ntb * ncells)) != cudaSuccess) return fail(e);
  if ((e = cudaMemcpy(dcells.p, cells.data(), sizeof(int) * cells.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(duv.p, uv.data(), sizeof(double) * uv.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(dfreq.p, freqs.data(), sizeof(double) * nf, cudaMemcpyHostToDevice)) != cudaSuccess)
    return fail(e);
  beam_uvdft_kernel<<<(unsigned)((nbf + 255) / 256), 256>>>(npx, (const int*)dcells.p, ncells, dl, 2.0 * sig * sig,
                                                             (double2*)dBF.p);
  const size_t smem = sizeof(double2) * npx * npx;
  if (smem > 48 * 1024 &&
      (e = cudaFuncSetAttribute(nudft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return fail(e);
  nudft_kernel<<<(unsigned)(nf * ntb), 256, smem>>>(npx, ncells, ntb, (const double*)duv.p,
                                                      (const double*)dfreq.p, dl, (const double2*)dBF.p,
                                                      (double2*)dA.p);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(e);
  return beor_set_instrument(ctx, (const beor_c128*)dA.p, W.data(), nf, ntb, ncells, nx, kbin.data(), d->n_k,
                             d->lssm_prior_var);
}
