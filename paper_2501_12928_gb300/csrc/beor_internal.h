// Host-side launchers shared between the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "beor_common.cuh"

namespace beor {

// precompute.cu
cudaError_t split_double_float(const double2* M, int64_t n, float4* out, cudaStream_t s);
// Full nt x nt tile square of the packed lower M (n x n, padding zero), each
// element split exactly into three floats per component.
cudaError_t split_full_triple(const double2* M, int n, int nt, float4* hl, float2* t, cudaStream_t s);
cudaError_t precompute_dense(const double2* T, int64_t n_vis, int n, int64_t ld, const double* w,
                             const double2* d, int nt, double2* Mt, double2* dbar, cudaStream_t s, bool tc);
// herk_tc.cu: M (packed lower float64 tiles) = T^H diag(w) T on the tensor cores
cudaError_t herk_dense_tc(const double2* T, int64_t n_vis, int n, int64_t ld, const double* w, int nt,
                          double2* Mt, cudaStream_t s);
cudaError_t precompute_factored(const double2* A, const double2* W, int nf, int64_t ntb, int ncells,
                                int nx, const double* w, const double2* d, int n, int nt,
                                double2* G_scratch, double2* u_scratch, double2* Mt, double2* dbar,
                                cudaStream_t s);

// Device-side view of one batched evaluation (all problems of all sets).
struct BatchView {
  int P;                     // problems
  int nsets;
  const Prob* prob;          // [P]
  const SetDesc* sets;       // [nsets]
  int max_nt;
  // workspaces
  void* ws;                  // packed tiles of every problem (double2 or float4)
  double2* dinv;             // inverse diagonal blocks, packed lower 128x128 per block
  double* phi_inv;           // [rows] prior inverse per problem row (padded rows = 1)
  double2* vec_b;            // [rows] right-hand side / residual
  double2* vec_y;            // [rows] forward-solve result
  double2* vec_x;            // [rows] solution
  double2* vec_t;            // [rows] solve scratch
  double2* vec_r;            // [rows] residual dbar - Sigma x (lnL correction or refinement)
  double2* vec_d;            // [rows] refinement correction
  double* logdet_phi;        // [P]
  double* logdet_sigma;      // [P]
  double* q;                 // [P]
  double* lnl;               // [P]
  int32_t* status;           // [P]
  double* resid;             // [P] accuracy indicator (see beor_stats.resid_rel_max)
  Flags* flags;
  // mixed path slice buffers
  __nv_bfloat16* panel_sl;   // 2 buffers (block step parity) of NPLANE planes of rows x 128 (slice_elem_off order), plane = slice_plane(slice, part)
  int32_t* panel_exp;        // 2 buffers of [rows]
  __nv_bfloat16* linv_sl;    // NPLANE planes of (P*128) x 128, slice_elem_off order
  int32_t* linv_exp;         // [P*128]
  // float64-accurate residual on the float32 pipe (mixed path)
  float* xtr;                // [rows][6]: x re (hi, lo, t), im (hi, lo, t)
  const RWork* rwork;        // CTA work items
  int n_rwork;
  int64_t rows;              // sum of padded dimensions
  int64_t ws_elems;          // elements of ws (bounds checks)
  int64_t dinv_elems;        // elements of dinv (bounds checks)
  // bounded waits of the tensor-core kernels: limit of a role's wait on
  // another role (ns), and a test switch (nonzero: the first trailing-update
  // CTA of the evaluation withholds one operand copy, so that the wait on it
  // runs out and the error path is taken)
  unsigned long long wait_ns;
  int test_skip_copy;
  // schedule: CTAs of the trailing launches for columns j >= k + 2 and of the
  // next-column / panel launches (0: one per SM)
  int grid_rest, grid_col;
};

// Launch with an explicit scheduling priority (0: the stream's own); the
// attribute is kept by stream capture, so graph nodes carry it too.
template <typename... Exp, typename... Act>
static cudaError_t launch_prio(void (*kern)(Exp...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, int prio,
                               Act&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributePriority;
  at[0].val.priority = prio;
  cfg.attrs = at;
  cfg.numAttrs = prio != 0 ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Act>(args)...);
}

// chol.cu (both precisions)
cudaError_t launch_prior_init(const BatchView& v, bool mixed, cudaStream_t s);
cudaError_t launch_diag(const BatchView& v, int k, bool mixed, cudaStream_t s, int prio = 0);
cudaError_t launch_panel_f64(const BatchView& v, int k, cudaStream_t s);
cudaError_t launch_trail_f64(const BatchView& v, int k, cudaStream_t s);
cudaError_t launch_solve(const BatchView& v, bool mixed, const double2* rhs, double2* out, cudaStream_t s);
// The solve's two halves: forward step k (k = -1: start) of vec_y = L^-1 rhs,
// and the whole backward pass out = L^-H vec_y.
cudaError_t launch_fwd_step(const BatchView& v, bool mixed, const double2* rhs, int k, cudaStream_t s, int prio = 0);
cudaError_t launch_bwd(const BatchView& v, bool mixed, double2* out, cudaStream_t s);
int solve_launch_count(int max_nt);
cudaError_t launch_lnl(const BatchView& v, cudaStream_t s, int corr);   // corr: residual-corrected q
cudaError_t launch_solve_fwd(const BatchView& v, bool mixed, const double2* rhs, cudaStream_t s);   // vec_y = L^-1 rhs
cudaError_t launch_copy_dbar(const BatchView& v, cudaStream_t s);

// mixed.cu
struct MixedMaps;  // opaque TMA descriptors of one batch
cudaError_t mixed_maps_create(const BatchView& v, MixedMaps** out);
void mixed_maps_destroy(MixedMaps* m);
// Block step k of the mixed factorisation: slicing of the panel column (buffer k % 2),
// the panel product, and the trailing update, whole or split into the next block
// column (j = k + 1) and the rest (j >= k + 2) so that step k + 1 can start early.
// prio: launch priority (0: the stream's).
enum { TRAIL_ALL = 0, TRAIL_NEXT_COL = 1, TRAIL_REST = 2 };
cudaError_t mixed_reset_counters(const MixedMaps* m, cudaStream_t s);   // before every evaluation
int64_t mixed_tiles(const MixedMaps* m, int kind, int k);               // kind 0 next col, 1 rest, 2 panel, 3 all
cudaError_t launch_slice_panel(const BatchView& v, int k, cudaStream_t s, int prio = 0);
cudaError_t launch_panel_mixed(const BatchView& v, const MixedMaps* m, int k, cudaStream_t s, int prio = 0);
// The trailing update is two launches: its off-diagonal tiles (reduced slice
// pair set) and its diagonal tiles (full set).  max_ctas > 0 caps each
// launch's CTAs further (below the schedule's cap).
cudaError_t launch_trail_mixed(const BatchView& v, const MixedMaps* m, int k, int part, cudaStream_t s,
                               int prio = 0, int max_ctas = 0);
int trail_launch_count(const MixedMaps* m, int k, int part);   // kernels launch_trail_mixed launches
int device_sms();   // SMs of the current device
cudaError_t launch_residual(const BatchView& v, cudaStream_t s);      // vec_r = dbar - Sigma x (float64)
cudaError_t launch_refine_update(const BatchView& v, cudaStream_t s); // x += vec_d; residual norm
int mixed_supported(int device);

}  // namespace beor
