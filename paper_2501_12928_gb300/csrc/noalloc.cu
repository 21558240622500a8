// dbar = T^H N^-1 d of a factored instrument, computed without allocating
// any device memory.
//
// Who needs this: callers that may not, or must not, call cudaMalloc --
// for instance code running inside another framework that has already
// reserved all device memory in its own pool (a fresh cudaMalloc would fail
// or fragment that pool), or a loop that must never stall on the device
// allocator (cudaMalloc / cudaFree can synchronise the whole device).  The
// regular precompute allocates its per-frequency partial sums; this variant
// keeps them in a fixed file-scope device array instead, so the caller only
// provides inputs and the output.
//
// The partial sums u[f][c] = sum_tb conj(A_f[tb, c]) d[f, tb] / sigma^2 live
// in g_noalloc_u, at most kNoallocMaxU = 65536 complex values (1 MiB),
// which every GPU that loads the library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/beor.h"

namespace {

constexpr int64_t kNoallocMaxU = 65536;     // nf * ncells limit
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double2 g_noalloc_u[kNoallocMaxU];

__global__ void noalloc_zero_kernel(double2* u, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    u[i] = make_double2(0.0, 0.0);
}

// u[f][c] += sum over a chunk of tb of conj(A[f][tb][c]) d[f][tb] / noise_var[f][tb]
__global__ void noalloc_partial_kernel(const double2* __restrict__ A, const double* __restrict__ noise_var,
                                       const double2* __restrict__ d, int64_t ntb, int ncells, int64_t chunk,
                                       double2* __restrict__ u) {
  const int f = blockIdx.z;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  const int64_t t0 = (int64_t)blockIdx.y * chunk, t1 = min(ntb, t0 + chunk);
  const double2* Af = A + (int64_t)f * ntb * ncells;
  double sr = 0.0, si = 0.0;
  for (int64_t tb = t0; tb < t1; ++tb) {
    const double2 a = Af[tb * ncells + c];
    const double2 dd = d[(int64_t)f * ntb + tb];
    const double w = 1.0 / noise_var[(int64_t)f * ntb + tb];
    const double dr = dd.x * w, di = dd.y * w;
    sr = fma(a.x, dr, fma(a.y, di, sr));
    si = fma(a.x, di, fma(-a.y, dr, si));
  }
  atomicAdd(&u[(int64_t)f * ncells + c].x, sr);
  atomicAdd(&u[(int64_t)f * ncells + c].y, si);
}

// dbar[(c, x)] = sum_f conj(W[f][x]) u[f][c]
__global__ void noalloc_assemble_kernel(const double2* __restrict__ u, const double2* __restrict__ W, int nf,
                                        int ncells, int nx, double2* __restrict__ dbar) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= (int64_t)ncells * nx) return;
  const int c = (int)(j / nx), x = (int)(j % nx);
  double vr = 0.0, vi = 0.0;
  for (int f = 0; f < nf; ++f) {
    const double2 w = W[f * nx + x], q = u[(int64_t)f * ncells + c];
    vr = fma(w.x, q.x, fma(w.y, q.y, vr));
    vi = fma(w.x, q.y, fma(-w.y, q.x, vi));
  }
  dbar[j] = make_double2(vr, vi);
}

std::mutex g_noalloc_mu;
double2* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up
// once per device (host code cannot use the array's name as an address).
int noalloc_scratch(double2** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return BEOR_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return BEOR_ENOTSUP;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    double2* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_noalloc_u);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return BEOR_ECUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return BEOR_OK;
}

// Device memory of device `dev` (the current one), or managed memory: a
// pointer to another GPU's memory is refused, since the kernels run on `dev`
// and would read it over a peer mapping that may not exist.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" int beor_dbar_factored_noalloc(const beor_c128* A, const beor_c128* W, int nf, int64_t ntb, int ncells,
                                          int nx, const double* noise_var, const beor_c128* d, beor_c128* dbar_out,
                                          void* stream) {
  if (!A || !W || !noise_var || !d || !dbar_out) return BEOR_EINVAL;
  if (nf <= 0 || ntb <= 0 || ncells <= 0 || nx <= 0) return BEOR_EINVAL;
  if ((int64_t)nf * ncells > kNoallocMaxU || nf > 65535) return BEOR_EINVAL;   // beyond the fixed scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return BEOR_ECUDA;
  }
  if (!on_device(A, dev) || !on_device(W, dev) || !on_device(noise_var, dev) || !on_device(d, dev) ||
      !on_device(dbar_out, dev))
    return BEOR_EINVAL;
  double2* u = nullptr;
  int r = noalloc_scratch(&u);
  if (r) return r;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t nu = (int64_t)nf * ncells;
  noalloc_zero_kernel<<<(unsigned)((nu + 255) / 256), 256, 0, s>>>(u, nu);
  const int64_t chunk = 2048;
  dim3 g((ncells + 127) / 128, (unsigned)((ntb + chunk - 1) / chunk), (unsigned)nf);
  noalloc_partial_kernel<<<g, 128, 0, s>>>(reinterpret_cast<const double2*>(A), noise_var,
                                           reinterpret_cast<const double2*>(d), ntb, ncells, chunk, u);
  const int64_t n = (int64_t)ncells * nx;
  noalloc_assemble_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
      u, reinterpret_cast<const double2*>(W), nf, ncells, nx, reinterpret_cast<double2*>(dbar_out));
  if (cudaGetLastError() != cudaSuccess) return BEOR_ECUDA;
  return BEOR_OK;
}
