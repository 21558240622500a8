// Learned emulator of lnL(phi): a multilayer perceptron n_in -> depth x width
// (GELU) -> 1, trained and evaluated by the library's own kernels.
//
// Numbers: bf16 weights and activations feed the tensor cores
// (mma.sync m16n8k16, fp32 accumulation); pre-activations, gradients of the
// loss, master weights and the Adam moments are fp32.  The emulator only
// pre-screens candidate prior points for the nested sampler; every accepted
// point is evaluated exactly.
//
// Kernels: one tiled bf16 GEMM with fused epilogues (bias + GELU for hidden
// layers, bias for the output, GELU-derivative for the backward data product,
// plain store for weight gradients), a loss/seed-gradient kernel, a column-sum
// kernel for bias gradients and one fused Adam update over every parameter.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/beor.h"

namespace {

constexpr int kMaxLayers = 9;
constexpr int kGT = 64;     // GEMM CTA tile (M and N)
constexpr int kGK = 16;     // K step
constexpr int kPad = 8;     // smem row padding (bf16 elements)

enum { EPI_HIDDEN = 0, EPI_OUT = 1, EPI_DX = 2, EPI_DW = 3 };

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

struct GemmArgs {
  // C[m][n] = sum_k A(m, k) B(n, k); A(m,k) = A[m*am + k*ak], B(n,k) = B[n*bn + k*bk]
  const __nv_bfloat16* A;
  int64_t am, ak;
  const __nv_bfloat16* B;
  int64_t bn, bk;
  int M, N, K;
  // epilogue
  const float* bias;        // [N] (HIDDEN, OUT)
  float* Z;                 // [M][ldz] pre-activation out (HIDDEN) / input (DX)
  int64_t ldz;
  __nv_bfloat16* H;         // [M][ldh] bf16 output (HIDDEN: GELU(z); DX: dZ of previous layer)
  int64_t ldh;
  float* F;                 // fp32 output: OUT y[m]; DX dZ fp32 [M][ldh]; DW grad [M][ldf]
  int64_t ldf;
  int n_valid;              // columns written (N may be padded)
};

template <int EPI>
__global__ void __launch_bounds__(128) gemm_bf16_kernel(GemmArgs g) {
  __shared__ __align__(16) __nv_bfloat16 sA[kGT][kGK + kPad];
  __shared__ __align__(16) __nv_bfloat16 sB[kGT][kGK + kPad];
  const int m0 = blockIdx.y * kGT, n0 = blockIdx.x * kGT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int gq = lane >> 2, tq = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.0f;
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
  for (int k0 = 0; k0 < g.K; k0 += kGK) {
    for (int e = threadIdx.x; e < kGT * kGK; e += 128) {
      const int r = e / kGK, k = e % kGK;
      const int gm = m0 + r, gn = n0 + r, gk = k0 + k;
      sA[r][k] = (gm < g.M && gk < g.K) ? g.A[gm * g.am + gk * g.ak] : zero;
      sB[r][k] = (gn < g.N && gk < g.K) ? g.B[gn * g.bn + gk * g.bk] : zero;
    }
    __syncthreads();
    uint32_t af[2][4], bf[4][2];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int r = wm + mt * 16 + gq;
      af[mt][0] = *reinterpret_cast<const uint32_t*>(&sA[r][2 * tq]);
      af[mt][1] = *reinterpret_cast<const uint32_t*>(&sA[r + 8][2 * tq]);
      af[mt][2] = *reinterpret_cast<const uint32_t*>(&sA[r][2 * tq + 8]);
      af[mt][3] = *reinterpret_cast<const uint32_t*>(&sA[r + 8][2 * tq + 8]);
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int c = wn + nt * 8 + gq;
      bf[nt][0] = *reinterpret_cast<const uint32_t*>(&sB[c][2 * tq]);
      bf[nt][1] = *reinterpret_cast<const uint32_t*>(&sB[c][2 * tq + 8]);
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        float* d = acc[mt][nt];
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(af[mt][0]), "r"(af[mt][1]), "r"(af[mt][2]), "r"(af[mt][3]), "r"(bf[nt][0]), "r"(bf[nt][1]));
      }
    __syncthreads();
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = m0 + wm + mt * 16 + gq + ((q & 2) ? 8 : 0);
        const int n = n0 + wn + nt * 8 + 2 * tq + (q & 1);
        if (m >= g.M || n >= g.n_valid) continue;
        const float v = acc[mt][nt][q];
        if (EPI == EPI_HIDDEN) {
          const float z = v + g.bias[n];
          g.Z[m * g.ldz + n] = z;
          g.H[m * g.ldh + n] = __float2bfloat16_rn(gelu(z));
        } else if (EPI == EPI_OUT) {
          g.F[m] = v + g.bias[n];
        } else if (EPI == EPI_DX) {
          const float dz = v * gelu_grad(g.Z[m * g.ldz + n]);
          g.F[m * g.ldf + n] = dz;
          g.H[m * g.ldh + n] = __float2bfloat16_rn(dz);
        } else {
          g.F[m * g.ldf + n] = v;
        }
      }
}

template <int EPI>
cudaError_t gemm(const GemmArgs& a, cudaStream_t s) {
  dim3 grid((a.N + kGT - 1) / kGT, (a.M + kGT - 1) / kGT);
  gemm_bf16_kernel<EPI><<<grid, 128, 0, s>>>(a);
  return cudaGetLastError();
}

// normalised, zero-padded bf16 input rows
__global__ void input_kernel(const float* __restrict__ x, int n, int n_in, int ld, const float* __restrict__ shift,
                             const float* __restrict__ scale, __nv_bfloat16* __restrict__ H0) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * ld) return;
  const int m = (int)(e / ld), i = (int)(e % ld);
  const float v = i < n_in ? (x[(int64_t)m * n_in + i] - shift[i]) * scale[i] : 0.0f;
  H0[e] = __float2bfloat16_rn(v);
}

// loss = mean (y - t)^2 in normalised units; seed gradient dZ_out = 2 (y - t) / n
__global__ void loss_kernel(const float* __restrict__ y, const float* __restrict__ t, int n, float y_shift,
                            float y_scale, float* __restrict__ dz, int ldz, __nv_bfloat16* __restrict__ dzb,
                            float* __restrict__ loss) {
  __shared__ float red[32];
  float acc = 0.0f;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
    const float target = (t[m] - y_shift) / y_scale;
    const float r = y[m] - target;
    acc += r * r;
    const float gdz = 2.0f * r / (float)n;
    for (int c = 0; c < ldz; ++c) {
      dz[(int64_t)m * ldz + c] = c == 0 ? gdz : 0.0f;
      dzb[(int64_t)m * ldz + c] = __float2bfloat16_rn(c == 0 ? gdz : 0.0f);
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    atomicAdd(loss, s / (float)n);
  }
}

// db[o] = sum_m dz[m][o]
__global__ void colsum_kernel(const float* __restrict__ dz, int n, int ld, int cols, float* __restrict__ db) {
  const int o = blockIdx.x;
  if (o >= cols) return;
  __shared__ float red[32];
  float acc = 0.0f;
  for (int m = threadIdx.x; m < n; m += blockDim.x) acc += dz[(int64_t)m * ld + o];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    db[o] = s;
  }
}

// Adam on one flat parameter array with its bf16 working copy (optional)
struct AdamSeg {
  float* p;
  float* g;
  float* m;
  float* v;
  __nv_bfloat16* pb;    // bf16 copy (weights) or null (biases)
  int64_t n;
  int rows, cols, ldb;  // layout of the bf16 copy (padded)
};
struct AdamArgs {
  AdamSeg seg[2 * kMaxLayers];
  int nseg;
  float lr, b1, b2, eps, c1, c2;   // c1 = 1 - b1^t, c2 = 1 - b2^t
};

__global__ void adam_kernel(AdamArgs a) {
  const AdamSeg sg = a.seg[blockIdx.y];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < sg.n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gr = sg.g[i];
    const float m = a.b1 * sg.m[i] + (1.0f - a.b1) * gr;
    const float v = a.b2 * sg.v[i] + (1.0f - a.b2) * gr * gr;
    sg.m[i] = m;
    sg.v[i] = v;
    const float p = sg.p[i] - a.lr * (m / a.c1) / (sqrtf(v / a.c2) + a.eps);
    sg.p[i] = p;
    if (sg.pb) {
      const int r = (int)(i / sg.cols), c = (int)(i % sg.cols);
      sg.pb[(int64_t)r * sg.ldb + c] = __float2bfloat16_rn(p);
    }
  }
}

// He-uniform initial weights from a counter-based generator (SplitMix64 of
// seed, layer and index): W ~ U(-sqrt(6 / fan_in), sqrt(6 / fan_in)).
__global__ void init_kernel(float* W, int64_t n, int fan_in, uint64_t seed, int layer) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1) + ((uint64_t)layer << 48);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);   // [0, 1)
    const double lim = sqrt(6.0 / (double)fan_in);
    W[i] = (float)((2.0 * u - 1.0) * lim);
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ W, int rows, int cols, int ldb, __nv_bfloat16* __restrict__ Wb) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)rows * cols) return;
  const int r = (int)(e / cols), c = (int)(e % cols);
  Wb[(int64_t)r * ldb + c] = __float2bfloat16_rn(W[e]);
}

// y = y_net * scale + shift (the network's output units to lnL units)
__global__ void affine_kernel(float* y, int n, float scale, float shift) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = y[i] * scale + shift;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int pad16(int x) { return (x + 15) / 16 * 16; }

}  // namespace

struct beor_mlp {
  int device = 0, n_in = 0, width = 0, depth = 0, L = 0;
  int fin[kMaxLayers], fout[kMaxLayers];      // logical sizes
  int kin[kMaxLayers], kout[kMaxLayers];      // padded sizes (bf16 copies, activations)
  float *W[kMaxLayers] = {}, *b[kMaxLayers] = {}, *gW[kMaxLayers] = {}, *gb[kMaxLayers] = {};
  float *mW[kMaxLayers] = {}, *vW[kMaxLayers] = {}, *mb[kMaxLayers] = {}, *vb[kMaxLayers] = {};
  __nv_bfloat16* Wb[kMaxLayers] = {};
  float *x_shift = nullptr, *x_scale = nullptr;
  float y_shift = 0.0f, y_scale = 1.0f;
  int64_t step = 0;
  // batch workspace
  int cap = 0;
  __nv_bfloat16* H[kMaxLayers + 1] = {};      // activations (H[0] = normalised input)
  float* Z[kMaxLayers] = {};                  // pre-activations of hidden layers
  float* dZ = nullptr;                        // fp32 gradient of the current layer's pre-activation
  float* dZ2 = nullptr;
  __nv_bfloat16* dZb = nullptr;
  __nv_bfloat16* dZb2 = nullptr;
  float *xin = nullptr, *tin = nullptr, *yout = nullptr, *loss = nullptr;
  std::vector<void*> owned;
};

namespace {

cudaError_t dalloc(beor_mlp* m, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) {
    m->owned.push_back(*p);
    cudaMemset(*p, 0, bytes);
  }
  return e;
}

cudaError_t ensure_cap(beor_mlp* m, int n) {
  if (n <= m->cap) return cudaSuccess;
  // release the old batch workspace
  auto rel = [&](void* p) {
    if (!p) return;
    for (auto& q : m->owned)
      if (q == p) q = nullptr;
    cudaFree(p);
  };
  for (int l = 0; l <= m->L; ++l) rel(m->H[l]);
  for (int l = 0; l < m->L; ++l) rel(m->Z[l]);
  rel(m->dZ);
  rel(m->dZ2);
  rel(m->dZb);
  rel(m->dZb2);
  rel(m->xin);
  rel(m->tin);
  rel(m->yout);
  int cap = 1024;
  while (cap < n) cap *= 2;
  const int wmax = std::max(m->width, 16);
  cudaError_t e = cudaSuccess;
  for (int l = 0; l <= m->L && e == cudaSuccess; ++l) {
    const int w = l == 0 ? m->kin[0] : (l < m->L ? m->kout[l - 1] : 16);
    e = dalloc(m, (void**)&m->H[l], sizeof(__nv_bfloat16) * (size_t)cap * w);
  }
  for (int l = 0; l < m->L && e == cudaSuccess; ++l)
    e = dalloc(m, (void**)&m->Z[l], sizeof(float) * (size_t)cap * std::max(m->kout[l], 16));
  if (e == cudaSuccess) e = dalloc(m, (void**)&m->dZ, sizeof(float) * (size_t)cap * wmax);
  if (e == cudaSuccess) e = dalloc(m, (void**)&m->dZ2, sizeof(float) * (size_t)cap * wmax);
  if (e == cudaSuccess) e = dalloc(m, (void**)&m->dZb, sizeof(__nv_bfloat16) * (size_t)cap * wmax);
  if (e == cudaSuccess) e = dalloc(m, (void**)&m->dZb2, sizeof(__nv_bfloat16) * (size_t)cap * wmax);
  if (e == cudaSuccess) e = dalloc(m, (void**)&m->xin, sizeof(float) * (size_t)cap * m->n_in);
  if (e == cudaSuccess) e = dalloc(m, (void**)&m->tin, sizeof(float) * (size_t)cap);
  if (e == cudaSuccess) e = dalloc(m, (void**)&m->yout, sizeof(float) * (size_t)cap);
  if (e == cudaSuccess) m->cap = cap;
  return e;
}

cudaError_t copy_in(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  return cudaMemcpyAsync(dst, src, bytes, on_device(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
}

// forward pass over n rows already in m->xin; output y in m->yout
cudaError_t forward(beor_mlp* m, int n, cudaStream_t s) {
  const int ld0 = m->kin[0];
  input_kernel<<<(unsigned)(((int64_t)n * ld0 + 255) / 256), 256, 0, s>>>(m->xin, n, m->n_in, ld0, m->x_shift,
                                                                           m->x_scale, m->H[0]);
  for (int l = 0; l < m->L; ++l) {
    GemmArgs g{};
    g.A = m->H[l];
    g.am = m->kin[l];
    g.ak = 1;
    g.B = m->Wb[l];
    g.bn = m->kin[l];
    g.bk = 1;
    g.M = n;
    g.N = m->kout[l];
    g.K = m->kin[l];
    g.bias = m->b[l];
    if (l + 1 < m->L) {
      g.Z = m->Z[l];
      g.ldz = m->kout[l];
      g.H = m->H[l + 1];
      g.ldh = m->kout[l];
      g.n_valid = m->fout[l];
      cudaError_t e = gemm<EPI_HIDDEN>(g, s);
      if (e != cudaSuccess) return e;
    } else {
      g.F = m->yout;
      g.n_valid = 1;
      cudaError_t e = gemm<EPI_OUT>(g, s);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// loss and gradients of every parameter for n rows (targets in m->tin)
cudaError_t backward(beor_mlp* m, int n, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(m->loss, 0, sizeof(float), s);
  if (e != cudaSuccess) return e;
  const int lo = m->L - 1;
  // dZ of the output layer: n x kout[lo] (only column 0 nonzero)
  loss_kernel<<<std::min(1024, (n + 255) / 256), 256, 0, s>>>(m->yout, m->tin, n, m->y_shift, m->y_scale, m->dZ,
                                                              m->kout[lo], m->dZb, m->loss);
  float* dz = m->dZ;
  __nv_bfloat16* dzb = m->dZb;
  float* dz2 = m->dZ2;
  __nv_bfloat16* dzb2 = m->dZb2;
  for (int l = lo; l >= 0; --l) {
    const int ldz = m->kout[l];
    // weight gradient: gW[o][i] = sum_m dZ[m][o] H_l[m][i]
    GemmArgs gw{};
    gw.A = dzb;
    gw.am = 1;
    gw.ak = ldz;
    gw.B = m->H[l];
    gw.bn = 1;
    gw.bk = m->kin[l];
    gw.M = m->fout[l];
    gw.N = m->fin[l];
    gw.K = n;
    gw.F = m->gW[l];
    gw.ldf = m->fin[l];
    gw.n_valid = m->fin[l];
    e = gemm<EPI_DW>(gw, s);
    if (e != cudaSuccess) return e;
    colsum_kernel<<<m->fout[l], 256, 0, s>>>(dz, n, ldz, m->fout[l], m->gb[l]);
    if (l > 0) {
      // dZ_{l-1} = (dZ_l W_l) * gelu'(Z_{l-1})
      GemmArgs gx{};
      gx.A = dzb;
      gx.am = ldz;
      gx.ak = 1;
      gx.B = m->Wb[l];
      gx.bn = 1;
      gx.bk = m->kin[l];
      gx.M = n;
      gx.N = m->kin[l];
      gx.K = m->kout[l];
      gx.Z = m->Z[l - 1];
      gx.ldz = m->kout[l - 1];
      gx.F = dz2;
      gx.ldf = m->kout[l - 1];
      gx.H = dzb2;
      gx.ldh = m->kout[l - 1];
      gx.n_valid = m->fout[l - 1];
      e = gemm<EPI_DX>(gx, s);
      if (e != cudaSuccess) return e;
      std::swap(dz, dz2);
      std::swap(dzb, dzb2);
    }
  }
  return cudaGetLastError();
}

}  // namespace

extern "C" {

int beor_mlp_create(beor_mlp** out, int device, int n_in, int width, int depth, uint64_t seed) {
  if (!out || n_in < 1 || n_in > 16 || width < 16 || width > 256 || width % 16 || depth < 1 || depth > 8)
    return BEOR_EINVAL;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return BEOR_EINVAL;
  }
  beor_mlp* m = new beor_mlp();
  m->device = device;
  m->n_in = n_in;
  m->width = width;
  m->depth = depth;
  m->L = depth + 1;
  for (int l = 0; l < m->L; ++l) {
    m->fin[l] = l == 0 ? n_in : width;
    m->fout[l] = l == m->L - 1 ? 1 : width;
    m->kin[l] = pad16(m->fin[l]);
    m->kout[l] = l == m->L - 1 ? 16 : width;
  }
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < m->L && e == cudaSuccess; ++l) {
    const size_t nw = (size_t)m->fout[l] * m->fin[l];
    e = dalloc(m, (void**)&m->W[l], sizeof(float) * nw);
    if (e == cudaSuccess) e = dalloc(m, (void**)&m->gW[l], sizeof(float) * nw);
    if (e == cudaSuccess) e = dalloc(m, (void**)&m->mW[l], sizeof(float) * nw);
    if (e == cudaSuccess) e = dalloc(m, (void**)&m->vW[l], sizeof(float) * nw);
    if (e == cudaSuccess) e = dalloc(m, (void**)&m->b[l], sizeof(float) * m->fout[l]);
    if (e == cudaSuccess) e = dalloc(m, (void**)&m->gb[l], sizeof(float) * m->fout[l]);
    if (e == cudaSuccess) e = dalloc(m, (void**)&m->mb[l], sizeof(float) * m->fout[l]);
    if (e == cudaSuccess) e = dalloc(m, (void**)&m->vb[l], sizeof(float) * m->fout[l]);
    if (e == cudaSuccess)
      e = dalloc(m, (void**)&m->Wb[l], sizeof(__nv_bfloat16) * (size_t)m->kout[l] * m->kin[l]);
    if (e == cudaSuccess) {
      init_kernel<<<256, 256>>>(m->W[l], (int64_t)nw, m->fin[l], seed, l);
      to_bf16_kernel<<<(unsigned)((nw + 255) / 256), 256>>>(m->W[l], m->fout[l], m->fin[l], m->kin[l], m->Wb[l]);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = dalloc(m, (void**)&m->x_shift, sizeof(float) * n_in);
  if (e == cudaSuccess) e = dalloc(m, (void**)&m->x_scale, sizeof(float) * n_in);
  if (e == cudaSuccess) e = dalloc(m, (void**)&m->loss, sizeof(float));
  if (e == cudaSuccess) {
    std::vector<float> one(n_in, 1.0f);
    e = cudaMemcpy(m->x_scale, one.data(), sizeof(float) * n_in, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = ensure_cap(m, 1024);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    for (void* p : m->owned)
      if (p) cudaFree(p);
    delete m;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? BEOR_ENOMEM : BEOR_ECUDA;
  }
  *out = m;
  return BEOR_OK;
}

int beor_mlp_destroy(beor_mlp* m) {
  if (!m) return BEOR_EINVAL;
  cudaSetDevice(m->device);
  cudaDeviceSynchronize();
  for (void* p : m->owned)
    if (p) cudaFree(p);
  delete m;
  return BEOR_OK;
}

int beor_mlp_set_norm(beor_mlp* m, const float* x_shift, const float* x_scale, float y_shift, float y_scale) {
  if (!m || !x_shift || !x_scale || !(y_scale != 0.0f)) return BEOR_EINVAL;
  cudaSetDevice(m->device);
  if (copy_in(m->x_shift, x_shift, sizeof(float) * m->n_in, 0) != cudaSuccess ||
      copy_in(m->x_scale, x_scale, sizeof(float) * m->n_in, 0) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess)
    return BEOR_ECUDA;
  m->y_shift = y_shift;
  m->y_scale = y_scale;
  return BEOR_OK;
}

int beor_mlp_infer(beor_mlp* m, const float* x, int n, float* y_out, void* stream) {
  if (!m || !x || !y_out || n <= 0) return BEOR_EINVAL;
  cudaSetDevice(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int chunk = 65536;
  if (ensure_cap(m, std::min(n, chunk)) != cudaSuccess) return BEOR_ENOMEM;
  const bool dev_out = on_device(y_out);
  for (int off = 0; off < n; off += chunk) {
    const int c = std::min(chunk, n - off);
    if (copy_in(m->xin, x + (int64_t)off * m->n_in, sizeof(float) * (size_t)c * m->n_in, s) != cudaSuccess)
      return BEOR_ECUDA;
    if (forward(m, c, s) != cudaSuccess) return BEOR_ECUDA;
    affine_kernel<<<(c + 255) / 256, 256, 0, s>>>(m->yout, c, m->y_scale, m->y_shift);
    if (cudaMemcpyAsync(y_out + off, m->yout, sizeof(float) * c,
                        dev_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return BEOR_ECUDA;
  }
  if (!dev_out && cudaStreamSynchronize(s) != cudaSuccess) return BEOR_ECUDA;
  return cudaGetLastError() == cudaSuccess ? BEOR_OK : BEOR_ECUDA;
}

static int mlp_grads(beor_mlp* m, const float* x, const float* y, int n, float* loss_out, cudaStream_t s) {
  if (ensure_cap(m, n) != cudaSuccess) return BEOR_ENOMEM;
  if (copy_in(m->xin, x, sizeof(float) * (size_t)n * m->n_in, s) != cudaSuccess) return BEOR_ECUDA;
  if (copy_in(m->tin, y, sizeof(float) * (size_t)n, s) != cudaSuccess) return BEOR_ECUDA;
  if (forward(m, n, s) != cudaSuccess) return BEOR_ECUDA;
  if (backward(m, n, s) != cudaSuccess) return BEOR_ECUDA;
  if (loss_out) {
    if (cudaMemcpyAsync(loss_out, m->loss, sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess) return BEOR_ECUDA;
  }
  return BEOR_OK;
}

int beor_mlp_train_step(beor_mlp* m, const float* x, const float* y, int n, float lr, float beta1, float beta2,
                        float eps, float* loss_out, void* stream) {
  if (!m || !x || !y || n <= 0 || !(lr > 0.0f)) return BEOR_EINVAL;
  cudaSetDevice(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  int r = mlp_grads(m, x, y, n, loss_out, s);
  if (r) return r;
  m->step += 1;
  AdamArgs a{};
  a.lr = lr;
  a.b1 = beta1;
  a.b2 = beta2;
  a.eps = eps;
  a.c1 = 1.0f - powf(beta1, (float)m->step);
  a.c2 = 1.0f - powf(beta2, (float)m->step);
  for (int l = 0; l < m->L; ++l) {
    a.seg[a.nseg++] = AdamSeg{m->W[l], m->gW[l], m->mW[l], m->vW[l], m->Wb[l], (int64_t)m->fout[l] * m->fin[l],
                              m->fout[l], m->fin[l], m->kin[l]};
    a.seg[a.nseg++] = AdamSeg{m->b[l], m->gb[l], m->mb[l], m->vb[l], nullptr, (int64_t)m->fout[l], 1, m->fout[l], 0};
  }
  adam_kernel<<<dim3(64, a.nseg), 256, 0, s>>>(a);
  if (cudaGetLastError() != cudaSuccess) return BEOR_ECUDA;
  if (loss_out && cudaStreamSynchronize(s) != cudaSuccess) return BEOR_ECUDA;
  return BEOR_OK;
}

int beor_mlp_grad(beor_mlp* m, const float* x, const float* y, int n, int layer, float* dW, float* db,
                  float* loss_out) {
  if (!m || !x || !y || n <= 0 || layer < 0 || layer >= m->L) return BEOR_EINVAL;
  cudaSetDevice(m->device);
  int r = mlp_grads(m, x, y, n, loss_out, 0);
  if (r) return r;
  if (cudaDeviceSynchronize() != cudaSuccess) return BEOR_ECUDA;
  if (dW && cudaMemcpy(dW, m->gW[layer], sizeof(float) * (size_t)m->fout[layer] * m->fin[layer],
                       cudaMemcpyDeviceToHost) != cudaSuccess)
    return BEOR_ECUDA;
  if (db && cudaMemcpy(db, m->gb[layer], sizeof(float) * m->fout[layer], cudaMemcpyDeviceToHost) != cudaSuccess)
    return BEOR_ECUDA;
  return BEOR_OK;
}

int beor_mlp_get_params(beor_mlp* m, int layer, float* W, float* b) {
  if (!m || layer < 0 || layer >= m->L) return BEOR_EINVAL;
  cudaSetDevice(m->device);
  if (W && cudaMemcpy(W, m->W[layer], sizeof(float) * (size_t)m->fout[layer] * m->fin[layer],
                      cudaMemcpyDeviceToHost) != cudaSuccess)
    return BEOR_ECUDA;
  if (b && cudaMemcpy(b, m->b[layer], sizeof(float) * m->fout[layer], cudaMemcpyDeviceToHost) != cudaSuccess)
    return BEOR_ECUDA;
  return BEOR_OK;
}

int beor_mlp_set_params(beor_mlp* m, int layer, const float* W, const float* b) {
  if (!m || layer < 0 || layer >= m->L) return BEOR_EINVAL;
  cudaSetDevice(m->device);
  const size_t nw = (size_t)m->fout[layer] * m->fin[layer];
  if (W) {
    if (copy_in(m->W[layer], W, sizeof(float) * nw, 0) != cudaSuccess) return BEOR_ECUDA;
    to_bf16_kernel<<<(unsigned)((nw + 255) / 256), 256>>>(m->W[layer], m->fout[layer], m->fin[layer], m->kin[layer],
                                                          m->Wb[layer]);
  }
  if (b && copy_in(m->b[layer], b, sizeof(float) * m->fout[layer], 0) != cudaSuccess) return BEOR_ECUDA;
  return cudaDeviceSynchronize() == cudaSuccess ? BEOR_OK : BEOR_ECUDA;
}

}  // extern "C"
