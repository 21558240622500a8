// C ABI of the library: contexts (one instrument each), the precompute, and
// batched likelihood evaluations driven through captured CUDA graphs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <mutex>
#include <vector>

#include "../../include/beor.h"
#include "beor_common.cuh"
#include "beor_internal.h"

using namespace beor;

namespace {

constexpr int kRefineIters = 2;   // refinement steps of the mixed solve (fixed: graph-captured)
constexpr int kClasses = 8;       // kernel classes timed when profiling is on
enum { KC_INIT = 0, KC_DIAG, KC_SLICE, KC_PANEL, KC_TRAIL, KC_SOLVE, KC_REFINE, KC_LNL };
bool g_profiling = false;
bool g_lookahead = true;      // default schedule of shapes without one of their own
// bounded-wait test switch (beor_set_wait_test): role-wait limit (0 = the
// kernels' own 2 s) and whether one operand copy is withheld
unsigned long long g_wait_ns = 0;
int g_skip_copy = 0;

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// copy n bytes from a host-or-device source to device memory
cudaError_t to_device(void* dst, const void* src, size_t n, cudaStream_t s) {
  return cudaMemcpyAsync(dst, src, n, is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
}
cudaError_t from_device(void* dst, const void* src, size_t n, cudaStream_t s) {
  return cudaMemcpyAsync(dst, src, n, is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
}

struct DevBuf {
  void* p = nullptr;
  size_t n = 0;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  cudaError_t alloc(size_t bytes) {
    release();
    if (bytes == 0) return cudaSuccess;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      p = nullptr;
      return e;
    }
    n = bytes;
    return cudaSuccess;
  }
  template <typename T>
  T* as() const { return reinterpret_cast<T*>(p); }
};

struct Plan;

}  // namespace

struct beor_ctx {
  int device = 0;
  int precision = BEOR_PREC_FP64;
  bool poisoned = false;
  // model
  int model_kind = 0;   // 0 none, 1 dense T, 2 factored
  int64_t n_vis = 0;
  int n = 0, nt = 0, n_k = 0;
  double lssm_prior_var = 1.0;
  int nf = 0, ncells = 0, nx = 0;
  int64_t ntb = 0, ld = 0;
  DevBuf T, A, W, kbin;
  // data
  bool have_data = false;
  DevBuf d, w;
  // precompute
  bool have_pre = false;
  DevBuf M, dbar, Mdf, Mf, Mft;
  // bookkeeping
  beor_stats stats{};
  Plan* last_plan = nullptr;
  int last_first = 0;
  std::vector<double> last_ldphi, last_ldsig, last_q;
};

namespace {

std::mutex g_mu;
std::vector<Plan*> g_plans;

struct Plan {
  std::vector<beor_ctx*> ctxs;
  std::vector<int> Bs;
  int device = 0;
  bool mixed = false;
  int P = 0, max_nt = 0;
  int64_t rows = 0;
  std::vector<Prob> h_prob;
  std::vector<SetDesc> h_sets;
  std::vector<int> first;   // first problem index of each set
  DevBuf d_prob, d_sets, ws, dinv, phi_inv, vecs, scal, flags, phis, panel_sl, panel_exp, linv_sl, linv_exp;
  DevBuf xtr, rwork;                // float32-pipe residual: x triples, work items
  int n_rwork = 0;
  std::vector<int64_t> phi_off;
  BatchView view{};
  MixedMaps* maps = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  int64_t launches = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool prof = false;
  bool refine_x = false;            // mixed: refine the solution (posterior mean) rather than correct q
  int slot = 0;                     // independent copies of one batch shape (asynchronous calls)
  bool lookahead = true;            // schedule of the mixed factorisation captured in the graph
  beor_schedule sch{};              // the shape's schedule when the plan was built
  unsigned long long wait_ns = 0;   // bounded-wait settings captured in the graph
  int skip_copy = 0;
  int prio_hi = 0;                  // greatest stream priority of the device
  std::vector<cudaEvent_t> pev;     // boundary events (profiling)
  std::vector<int> pcls;            // class of the launch after each boundary event
  std::vector<int> pstr;            // its stream: 0 main, 1 side (rest of the trailing update), 2 forward steps
  cudaStream_t side = nullptr;      // second stream of the look-ahead schedule (rest of the trailing update)
  cudaStream_t side2 = nullptr;     // third stream: forward substitution of dbar, step by step
  cudaEvent_t ev_col = nullptr, ev_rest = nullptr, ev_diag = nullptr, ev_fwd = nullptr;
  ~Plan() {
    for (cudaEvent_t e : pev) cudaEventDestroy(e);
    for (cudaEvent_t e : {ev_col, ev_rest, ev_diag, ev_fwd})
      if (e) cudaEventDestroy(e);
    if (side) cudaStreamDestroy(side);
    if (side2) cudaStreamDestroy(side2);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (maps) mixed_maps_destroy(maps);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
  }
};

thread_local cudaError_t g_last_cuda = cudaSuccess;   // the last CUDA failure seen by this thread

int fail_cuda(beor_ctx* c, cudaError_t e) {
  if (e == cudaSuccess) return BEOR_OK;
  g_last_cuda = e;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return BEOR_ENOMEM;
  }
  if (c) c->poisoned = true;
  return BEOR_ECUDA;
}

#define CKC(ctx, expr)                              \
  do {                                              \
    cudaError_t _e = (expr);                        \
    if (_e != cudaSuccess) return fail_cuda(ctx, _e); \
  } while (0)

// The sequence of kernels of one batched evaluation.  With `mark` set, an
// externally visible event is recorded on the launching stream before and
// after every launch, so that each kernel class can be timed inside the graph
// (launches on the two streams of the look-ahead schedule overlap, so the
// class times add up to more than the evaluation's wall time).
cudaError_t run_sequence(Plan& pl, cudaStream_t s, int64_t* nlaunch, bool mark) {
  const BatchView& v = pl.view;
  int64_t L = 0;
  size_t ev_i = 0;
  cudaError_t e;
  if (mark) {
    pl.pcls.clear();
    pl.pstr.clear();
  }
  auto tick = [&](cudaStream_t on) -> cudaError_t {
    if (!mark) return cudaSuccess;
    if (ev_i >= pl.pev.size()) {
      cudaEvent_t ev;
      cudaError_t x = cudaEventCreate(&ev);
      if (x != cudaSuccess) return x;
      pl.pev.push_back(ev);
    }
    return cudaEventRecordWithFlags(pl.pev[ev_i++], on, cudaEventRecordExternal);
  };
#define RUN_ON(cls, on, x)            \
  do {                                \
    if (mark) {                       \
      pl.pcls.push_back(cls);         \
      pl.pstr.push_back(on == s ? 0 : on == pl.side ? 1 : 2); \
    }                                 \
    e = tick(on);                     \
    if (e != cudaSuccess) return e;   \
    e = (x);                          \
    if (e != cudaSuccess) return e;   \
    e = tick(on);                     \
    if (e != cudaSuccess) return e;   \
  } while (0)
#define RUN(cls, x) RUN_ON(cls, s, x)
  if (pl.mixed) {
    e = mixed_reset_counters(pl.maps, s);
    if (e != cudaSuccess) return e;
  }
  RUN(KC_INIT, launch_prior_init(v, pl.mixed, s));
  L += 2;
  RUN(KC_INIT, launch_copy_dbar(v, s));
  L += 1;
  const bool la = pl.mixed && pl.lookahead;
  if (la) {
    // Look-ahead schedule of the mixed factorisation (three streams):
    //   main:  col(k) -> diag(k+1) -> slice(k+1) -> panel(k+1) -> slice(k+1) -> [rest(k)] col(k+1) ...
    //   side:  [col(k)] rest(k)
    //   side2: [diag(k+1)] forward substitution step k of y = L^-1 dbar
    // col(k) updates block column k+1 only, rest(k) the columns j >= k+2, so
    // the float64 diagonal factorisation and the panel of step k+1 run at high
    // priority on the SMs that rest(k) leaves free; rest(k) takes its tiles
    // from a counter, so its CTAs that start late (after the high-priority
    // kernels) just take fewer.  Forward step k needs only block column k
    // (final after panel(k)) and the inverse diagonal block k+1.
    const int hi = pl.prio_hi;
    auto fwd_after_diag = [&]() -> cudaError_t {
      cudaError_t x = cudaEventRecord(pl.ev_diag, s);
      if (x == cudaSuccess) x = cudaStreamWaitEvent(pl.side2, pl.ev_diag, 0);
      return x;
    };
    RUN(KC_DIAG, launch_diag(v, 0, true, s, hi));
    L += 1;
    if ((e = fwd_after_diag()) != cudaSuccess) return e;
    RUN_ON(KC_SOLVE, pl.side2, launch_fwd_step(v, true, v.vec_b, -1, pl.side2));
    L += 1;
    if (pl.max_nt > 1) {
      RUN(KC_SLICE, launch_slice_panel(v, 0, s, hi));
      RUN(KC_PANEL, launch_panel_mixed(v, pl.maps, 0, s, hi));
      RUN(KC_SLICE, launch_slice_panel(v, 0, s, hi));
      L += 3;
    }
    for (int k = 0; k + 1 < pl.max_nt; ++k) {
      RUN(KC_TRAIL, launch_trail_mixed(v, pl.maps, k, TRAIL_NEXT_COL, s, hi));
      L += trail_launch_count(pl.maps, k, TRAIL_NEXT_COL);
      if ((e = cudaEventRecord(pl.ev_col, s)) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(pl.side, pl.ev_col, 0)) != cudaSuccess) return e;
      RUN(KC_DIAG, launch_diag(v, k + 1, true, s, hi));
      L += 1;
      if ((e = fwd_after_diag()) != cudaSuccess) return e;
      RUN_ON(KC_SOLVE, pl.side2, launch_fwd_step(v, true, v.vec_b, k, pl.side2));
      L += 1;
      if (mixed_tiles(pl.maps, 1, k) > 0) {
        // reserve_diag: leave free the SMs that step k + 1's diagonal blocks
        // (one CTA each, running beside this launch) need
        int cap = 0;
        if (pl.sch.reserve_diag) {
          int active = 0;
          for (const Prob& pr : pl.h_prob) {
            const int kp = k + 1 - pr.k_off;
            active += kp >= 0 && kp < pr.nt && pr.n > 0;
          }
          cap = std::max(8, device_sms() - active);
        }
        RUN_ON(KC_TRAIL, pl.side, launch_trail_mixed(v, pl.maps, k, TRAIL_REST, pl.side, 0, cap));
        L += trail_launch_count(pl.maps, k, TRAIL_REST);
      }
      if ((e = cudaEventRecord(pl.ev_rest, pl.side)) != cudaSuccess) return e;
      if (k + 2 < pl.max_nt) {
        RUN(KC_SLICE, launch_slice_panel(v, k + 1, s, hi));
        RUN(KC_PANEL, launch_panel_mixed(v, pl.maps, k + 1, s, hi));
        RUN(KC_SLICE, launch_slice_panel(v, k + 1, s, hi));
        L += 3;
      }
      if ((e = cudaStreamWaitEvent(s, pl.ev_rest, 0)) != cudaSuccess) return e;
    }
    if ((e = cudaEventRecord(pl.ev_fwd, pl.side2)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(s, pl.ev_fwd, 0)) != cudaSuccess) return e;
  } else {
    for (int k = 0; k < pl.max_nt; ++k) {
      RUN(KC_DIAG, launch_diag(v, k, pl.mixed, s));
      L += 1;
      if (k + 1 < pl.max_nt) {
        if (pl.mixed) {
          RUN(KC_SLICE, launch_slice_panel(v, k, s));
          RUN(KC_PANEL, launch_panel_mixed(v, pl.maps, k, s));
          RUN(KC_SLICE, launch_slice_panel(v, k, s));
          RUN(KC_TRAIL, launch_trail_mixed(v, pl.maps, k, TRAIL_ALL, s));
          L += 3 + trail_launch_count(pl.maps, k, TRAIL_ALL);
        } else {
          RUN(KC_PANEL, launch_panel_f64(v, k, s));
          RUN(KC_TRAIL, launch_trail_f64(v, k, s));
          L += 2;
        }
      }
    }
  }
  if (la) {
    RUN(KC_SOLVE, launch_bwd(v, true, v.vec_x, s));   // the forward half ran during the factorisation
    L += pl.max_nt;
  } else {
    RUN(KC_SOLVE, launch_solve(v, pl.mixed, v.vec_b, v.vec_x, s));
    L += solve_launch_count(pl.max_nt);
  }
  const bool corr = pl.mixed && !pl.refine_x;
  if (pl.mixed && pl.refine_x) {
    // the solution itself is wanted (posterior mean): float64 iterative refinement
    for (int it = 0; it < kRefineIters; ++it) {
      RUN(KC_REFINE, launch_residual(v, s));
      RUN(KC_SOLVE, launch_solve(v, true, v.vec_r, v.vec_d, s));
      RUN(KC_REFINE, launch_refine_update(v, s));
      L += 5 + solve_launch_count(pl.max_nt);
    }
  } else if (corr) {
    // lnL only: one float64 residual r = dbar - Sigma x~ and y = L~^-1 r
    // correct the quadratic form (see lnl_kernel)
    RUN(KC_REFINE, launch_residual(v, s));
    RUN(KC_SOLVE, launch_solve_fwd(v, true, v.vec_r, s));
    L += 4 + pl.max_nt;
  }
  RUN(KC_LNL, launch_lnl(v, s, corr ? 1 : 0));
  L += 1;
#undef RUN
#undef RUN_ON
  if (nlaunch) *nlaunch = L;
  return cudaSuccess;
}

// Schedules per batch shape: precision, lnL or posterior mean, and the
// (model dimension, B) of every set in order.
std::map<std::string, beor_schedule> g_schedules;

std::string shape_key(beor_ctx* const* ctxs, int nsets, const int* Bs, bool need_x) {
  std::string k = "p" + std::to_string(ctxs[0]->precision) + (need_x ? "x1:" : "x0:");
  for (int s = 0; s < nsets; ++s) k += std::to_string(ctxs[s]->n) + "x" + std::to_string(Bs[s]) + ",";
  return k;
}

beor_schedule default_schedule() {
  beor_schedule d{};
  d.lookahead = g_lookahead ? 1 : 0;
  d.rest_ctas = 0;
  d.col_ctas = 0;
  d.align_ends = 1;
  d.reserve_diag = 0;
  return d;
}

beor_schedule schedule_of(const std::string& key) {
  auto it = g_schedules.find(key);
  return it == g_schedules.end() ? default_schedule() : it->second;
}

bool same_schedule(const beor_schedule& a, const beor_schedule& b) {
  return a.lookahead == b.lookahead && a.rest_ctas == b.rest_ctas && a.col_ctas == b.col_ctas &&
         a.align_ends == b.align_ends && a.reserve_diag == b.reserve_diag;
}

int build_plan(beor_ctx* const* ctxs, int nsets, const int* Bs, bool need_x, int slot, Plan** out) {
  Plan* pl = new Plan();
  pl->refine_x = need_x;
  pl->slot = slot;
  pl->device = ctxs[0]->device;
  pl->mixed = ctxs[0]->precision == BEOR_PREC_MIXED;
  int64_t ws_elems = 0, dinv_elems = 0, rows = 0;
  int64_t phi_total = 0;
  for (int s = 0; s < nsets; ++s) {
    beor_ctx* c = ctxs[s];
    pl->ctxs.push_back(c);
    pl->Bs.push_back(Bs[s]);
    pl->first.push_back((int)pl->h_prob.size());
    SetDesc sd{};
    sd.n = c->n;
    sd.nt = c->nt;
    sd.n_k = c->n_k;
    sd.lssm_prior_var = c->lssm_prior_var;
    sd.M = c->M.as<double2>();
    sd.Mdf = c->Mdf.as<float4>();
    sd.Mf = c->Mf.as<float4>();
    sd.Mft = c->Mft.as<float2>();
    sd.dbar = c->dbar.as<double2>();
    sd.kbin = c->kbin.as<int32_t>();
    pl->phi_off.push_back(phi_total);
    phi_total += (int64_t)Bs[s] * c->n_k;
    pl->h_sets.push_back(sd);
    for (int b = 0; b < Bs[s]; ++b) {
      Prob pr{};
      pr.n = c->n;
      pr.nt = c->nt;
      pr.set = s;
      pr.b = b;
      pr.ws_off = ws_elems;
      pr.dinv_off = dinv_elems;
      pr.row_off = rows;
      ws_elems += tri_count(c->nt) * BEOR_TILE_ELEMS;
      dinv_elems += (int64_t)c->nt * (BEOR_TB * (BEOR_TB + 1) / 2);
      rows += (int64_t)c->nt * BEOR_TB;
      pl->max_nt = std::max(pl->max_nt, c->nt);
      pl->h_prob.push_back(pr);
    }
  }
  pl->P = (int)pl->h_prob.size();
  pl->rows = rows;
  pl->sch = schedule_of(shape_key(ctxs, nsets, Bs, need_x));
  // mixed batches of uneven sizes: each problem starts max_nt - nt block steps
  // late, so that all end on the last step and the light late steps of the
  // largest problems overlap the heavy early steps of the smaller ones
  for (Prob& pr : pl->h_prob) pr.k_off = pl->mixed && pl->sch.align_ends ? pl->max_nt - pr.nt : 0;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) {
    if (x != cudaSuccess && e == cudaSuccess) e = x;
  };
  chk(pl->phis.alloc(sizeof(double) * std::max<int64_t>(1, phi_total)));
  for (int s = 0; s < nsets; ++s) pl->h_sets[s].phi = pl->phis.as<double>() + pl->phi_off[s];
  chk(pl->d_prob.alloc(sizeof(Prob) * pl->P));
  chk(pl->d_sets.alloc(sizeof(SetDesc) * nsets));
  chk(pl->ws.alloc((pl->mixed ? sizeof(float4) : sizeof(double2)) * (size_t)ws_elems));
  chk(pl->dinv.alloc(sizeof(double2) * (size_t)dinv_elems));
  chk(pl->phi_inv.alloc(sizeof(double) * (size_t)rows));
  chk(pl->vecs.alloc(sizeof(double2) * (size_t)rows * 6));
  chk(pl->scal.alloc(sizeof(double) * (size_t)pl->P * 6 + sizeof(int32_t) * pl->P));
  chk(pl->flags.alloc(sizeof(Flags)));
  if (pl->mixed) {
    chk(pl->panel_sl.alloc(sizeof(__nv_bfloat16) * 2 * (size_t)BEOR_NPLANE * rows * BEOR_TB));
    chk(pl->panel_exp.alloc(sizeof(int32_t) * 2 * (size_t)rows));
    chk(pl->linv_sl.alloc(sizeof(__nv_bfloat16) * (size_t)BEOR_NPLANE * pl->P * BEOR_TB * BEOR_TB));
    chk(pl->linv_exp.alloc(sizeof(int32_t) * (size_t)pl->P * BEOR_TB));
    chk(pl->xtr.alloc(sizeof(float) * 6 * (size_t)rows));
    // residual work items: row block x 16 block columns x 16 problems
    std::vector<RWork> wk;
    for (int s = 0; s < nsets; ++s) {
      const int nt = ctxs[s]->nt;
      for (int I = 0; I < nt; ++I)
        for (int j0 = 0; j0 < nt; j0 += 16)
          for (int g = 0; g < Bs[s]; g += 16)
            wk.push_back(RWork{s, I, j0, std::min(nt, j0 + 16), pl->first[s] + g, std::min(16, Bs[s] - g)});
    }
    pl->n_rwork = (int)wk.size();
    chk(pl->rwork.alloc(sizeof(RWork) * wk.size()));
    if (e == cudaSuccess) chk(cudaMemcpy(pl->rwork.p, wk.data(), sizeof(RWork) * wk.size(), cudaMemcpyHostToDevice));
  }
  if (e != cudaSuccess) {
    delete pl;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? BEOR_ENOMEM : BEOR_ECUDA;
  }
  chk(cudaMemcpy(pl->d_prob.p, pl->h_prob.data(), sizeof(Prob) * pl->P, cudaMemcpyHostToDevice));
  chk(cudaMemcpy(pl->d_sets.p, pl->h_sets.data(), sizeof(SetDesc) * nsets, cudaMemcpyHostToDevice));
  chk(cudaMemset(pl->flags.p, 0, sizeof(Flags)));
  BatchView& v = pl->view;
  v.P = pl->P;
  v.nsets = nsets;
  v.prob = pl->d_prob.as<Prob>();
  v.sets = pl->d_sets.as<SetDesc>();
  v.max_nt = pl->max_nt;
  v.ws = pl->ws.p;
  v.dinv = pl->dinv.as<double2>();
  v.phi_inv = pl->phi_inv.as<double>();
  double2* vb = pl->vecs.as<double2>();
  v.vec_b = vb;
  v.vec_y = vb + rows;
  v.vec_x = vb + 2 * rows;
  v.vec_t = vb + 3 * rows;
  v.vec_r = vb + 4 * rows;
  v.vec_d = vb + 5 * rows;
  double* sc = pl->scal.as<double>();
  v.logdet_phi = sc;
  v.logdet_sigma = sc + pl->P;
  v.q = sc + 2 * pl->P;
  v.lnl = sc + 3 * pl->P;
  v.resid = sc + 4 * pl->P;
  v.status = reinterpret_cast<int32_t*>(sc + 6 * pl->P);
  v.flags = pl->flags.as<Flags>();
  v.panel_sl = pl->panel_sl.as<__nv_bfloat16>();
  v.panel_exp = pl->panel_exp.as<int32_t>();
  v.linv_sl = pl->linv_sl.as<__nv_bfloat16>();
  v.linv_exp = pl->linv_exp.as<int32_t>();
  v.xtr = pl->xtr.as<float>();
  v.rwork = pl->rwork.as<RWork>();
  v.n_rwork = pl->n_rwork;
  v.rows = rows;
  v.ws_elems = ws_elems;
  v.dinv_elems = dinv_elems;
  v.grid_rest = pl->sch.rest_ctas;
  v.grid_col = pl->sch.col_ctas;
  if (pl->mixed) {
    chk(mixed_maps_create(v, &pl->maps));
    int lo = 0, hi = 0;
    chk(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    pl->prio_hi = hi;
    chk(cudaStreamCreateWithPriority(&pl->side, cudaStreamNonBlocking, lo));
    chk(cudaStreamCreateWithPriority(&pl->side2, cudaStreamNonBlocking, lo));
    for (cudaEvent_t* ev : {&pl->ev_col, &pl->ev_rest, &pl->ev_diag, &pl->ev_fwd})
      chk(cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
  }
  chk(cudaEventCreate(&pl->ev0));
  chk(cudaEventCreate(&pl->ev1));
  if (e != cudaSuccess) {
    delete pl;
    return BEOR_ECUDA;
  }
  *out = pl;
  return BEOR_OK;
}

Plan* find_plan(beor_ctx* const* ctxs, int nsets, const int* Bs, bool need_x, int slot) {
  for (Plan* p : g_plans) {
    if ((int)p->ctxs.size() != nsets || p->refine_x != need_x || p->slot != slot) continue;
    bool same = true;
    for (int s = 0; s < nsets && same; ++s) same = p->ctxs[s] == ctxs[s] && p->Bs[s] == Bs[s];
    if (same) return p;
  }
  return nullptr;
}

// Plans whose schedule is no longer their shape's (after beor_set_schedule or
// beor_set_lookahead) are released; the next call rebuilds them.
void drop_plans_with_stale_schedule() {
  std::vector<Plan*> keep;
  bool synced = false;
  for (Plan* p : g_plans) {
    const beor_schedule cur = schedule_of(shape_key(p->ctxs.data(), (int)p->ctxs.size(), p->Bs.data(), p->refine_x));
    if (!same_schedule(cur, p->sch)) {
      if (!synced) {   // no evaluation of the plan may still be running
        cudaSetDevice(p->device);
        cudaDeviceSynchronize();
        synced = true;
      }
      for (beor_ctx* o : p->ctxs)
        if (o->last_plan == p) o->last_plan = nullptr;
      delete p;
    } else {
      keep.push_back(p);
    }
  }
  g_plans.swap(keep);
}

void drop_plans_of(beor_ctx* c) {
  std::lock_guard<std::mutex> lk(g_mu);
  std::vector<Plan*> keep;
  for (Plan* p : g_plans) {
    if (std::find(p->ctxs.begin(), p->ctxs.end(), c) != p->ctxs.end()) {
      // the other contexts of a multi-context batch may still name this plan
      // as their last one (diagnostics); every context in a kept plan is
      // alive, since destroying a context drops its plans first
      for (beor_ctx* o : p->ctxs)
        if (o->last_plan == p) o->last_plan = nullptr;
      delete p;
    } else {
      keep.push_back(p);
    }
  }
  g_plans.swap(keep);
}

int check_ready(const beor_ctx* c) {
  if (!c) return BEOR_EINVAL;
  if (c->poisoned) return BEOR_ESTATE;
  return BEOR_OK;
}

int validate_kbin(const int32_t* kbin_host, int64_t n, int n_k) {
  std::vector<int64_t> cnt(n_k, 0);
  for (int64_t j = 0; j < n; ++j) {
    int b = kbin_host[j];
    if (b < -1 || b >= n_k) return BEOR_EINVAL;
    if (b >= 0) cnt[b]++;
  }
  for (int i = 0; i < n_k; ++i)
    if (cnt[i] == 0) return BEOR_EINVAL;
  return BEOR_OK;
}

int set_kbin(beor_ctx* c, const int32_t* kbin, int64_t n, int n_k, double lssm) {
  if (!kbin || n_k < 1 || !(lssm > 0.0) || !std::isfinite(lssm)) return BEOR_EINVAL;
  std::vector<int32_t> h(n);
  if (is_device_ptr(kbin)) {
    CKC(c, cudaMemcpy(h.data(), kbin, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(h.data(), kbin, sizeof(int32_t) * n);
  }
  int r = validate_kbin(h.data(), n, n_k);
  if (r) return r;
  CKC(c, c->kbin.alloc(sizeof(int32_t) * n));
  CKC(c, cudaMemcpy(c->kbin.p, h.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice));
  c->n_k = n_k;
  c->lssm_prior_var = lssm;
  return BEOR_OK;
}

}  // namespace

namespace beor {
// Shape key and precision of a batch, for the autotuner (autotune.cu).
std::string shape_key_of(beor_ctx* const* ctxs, int nsets, const int* B) {
  return shape_key(ctxs, nsets, B, false);
}
bool is_mixed(const beor_ctx* c) { return c && c->precision == BEOR_PREC_MIXED; }
}  // namespace beor

extern "C" {

const char* beor_last_cuda_error(void) { return cudaGetErrorName(g_last_cuda); }

int beor_build_info(void) {
#ifdef BEOR_BOUNDS_CHECK
  return 1;
#else
  return 0;
#endif
}

const char* beor_strerror(int code) {
  switch (code) {
    case BEOR_OK: return "ok";
    case BEOR_EINVAL: return "invalid argument";
    case BEOR_ENOMEM: return "out of memory";
    case BEOR_ECUDA: return "CUDA error";
    case BEOR_ETIMEOUT: return "device-side wait timed out";
    case BEOR_ESTATE: return "call out of order or context poisoned";
    case BEOR_ENOTSUP: return "not supported on this device";
    default: return "unknown error";
  }
}

int beor_create(beor_ctx** out, int device, int precision) {
  if (!out || (precision != BEOR_PREC_FP64 && precision != BEOR_PREC_MIXED)) return BEOR_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return BEOR_EINVAL;
  }
  if (cudaSetDevice(device) != cudaSuccess) return BEOR_ECUDA;
  if (precision == BEOR_PREC_MIXED && !mixed_supported(device)) return BEOR_ENOTSUP;
  beor_ctx* c = new beor_ctx();
  c->device = device;
  c->precision = precision;
  *out = c;
  return BEOR_OK;
}

int beor_destroy(beor_ctx* c) {
  if (!c) return BEOR_EINVAL;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  drop_plans_of(c);
  delete c;
  return BEOR_OK;
}

int beor_set_T(beor_ctx* c, const beor_c128* T, int64_t n_vis, int64_t n_model, int64_t ld,
               const int32_t* kbin, int n_k, double lssm_prior_var) {
  int r = check_ready(c);
  if (r) return r;
  if (!T || n_vis <= 0 || n_model <= 0 || ld < n_model || n_model > (1 << 20)) return BEOR_EINVAL;
  cudaSetDevice(c->device);
  drop_plans_of(c);
  r = set_kbin(c, kbin, n_model, n_k, lssm_prior_var);
  if (r) return r;
  c->model_kind = 1;
  c->n_vis = n_vis;
  c->n = (int)n_model;
  c->nt = (int)((n_model + BEOR_TB - 1) / BEOR_TB);
  c->ld = n_model;
  c->A.release();
  c->W.release();
  CKC(c, c->T.alloc(sizeof(double2) * (size_t)n_vis * n_model));
  if (ld == n_model) {
    CKC(c, to_device(c->T.p, T, sizeof(double2) * (size_t)n_vis * n_model, 0));
  } else {
    CKC(c, cudaMemcpy2D(c->T.p, sizeof(double2) * n_model, T, sizeof(double2) * ld, sizeof(double2) * n_model,
                        n_vis, is_device_ptr(T) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
  }
  CKC(c, cudaDeviceSynchronize());
  c->have_data = false;
  c->have_pre = false;
  return BEOR_OK;
}

int beor_set_instrument(beor_ctx* c, const beor_c128* A, const beor_c128* W, int nf, int64_t ntb, int ncells,
                        int nx, const int32_t* kbin, int n_k, double lssm_prior_var) {
  int r = check_ready(c);
  if (r) return r;
  if (!A || !W || nf <= 0 || ntb <= 0 || ncells <= 0 || nx <= 0) return BEOR_EINVAL;
  int64_t n = (int64_t)ncells * nx;
  if (n > (1 << 20)) return BEOR_EINVAL;
  cudaSetDevice(c->device);
  drop_plans_of(c);
  r = set_kbin(c, kbin, n, n_k, lssm_prior_var);
  if (r) return r;
  c->model_kind = 2;
  c->nf = nf;
  c->ntb = ntb;
  c->ncells = ncells;
  c->nx = nx;
  c->n_vis = (int64_t)nf * ntb;
  c->n = (int)n;
  c->nt = (int)((n + BEOR_TB - 1) / BEOR_TB);
  c->T.release();
  CKC(c, c->A.alloc(sizeof(double2) * (size_t)nf * ntb * ncells));
  CKC(c, c->W.alloc(sizeof(double2) * (size_t)nf * nx));
  CKC(c, to_device(c->A.p, A, sizeof(double2) * (size_t)nf * ntb * ncells, 0));
  CKC(c, to_device(c->W.p, W, sizeof(double2) * (size_t)nf * nx, 0));
  CKC(c, cudaDeviceSynchronize());
  c->have_data = false;
  c->have_pre = false;
  return BEOR_OK;
}

int beor_set_data(beor_ctx* c, const beor_c128* d, const double* noise_var) {
  int r = check_ready(c);
  if (r) return r;
  if (c->model_kind == 0) return BEOR_ESTATE;
  if (!d || !noise_var) return BEOR_EINVAL;
  cudaSetDevice(c->device);
  std::vector<double> nv(c->n_vis);
  if (is_device_ptr(noise_var)) {
    CKC(c, cudaMemcpy(nv.data(), noise_var, sizeof(double) * c->n_vis, cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(nv.data(), noise_var, sizeof(double) * c->n_vis);
  }
  for (double x : nv)
    if (!(x > 0.0) || !std::isfinite(x)) return BEOR_EINVAL;
  for (double& x : nv) x = 1.0 / x;
  CKC(c, c->w.alloc(sizeof(double) * c->n_vis));
  CKC(c, cudaMemcpy(c->w.p, nv.data(), sizeof(double) * c->n_vis, cudaMemcpyHostToDevice));
  CKC(c, c->d.alloc(sizeof(double2) * c->n_vis));
  CKC(c, to_device(c->d.p, d, sizeof(double2) * c->n_vis, 0));
  CKC(c, cudaDeviceSynchronize());
  c->have_data = true;
  c->have_pre = false;
  drop_plans_of(c);
  return BEOR_OK;
}

int beor_precompute(beor_ctx* c, void* stream) {
  int r = check_ready(c);
  if (r) return r;
  if (!c->have_data) return BEOR_ESTATE;
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  drop_plans_of(c);
  CKC(c, c->M.alloc(sizeof(double2) * (size_t)tri_count(c->nt) * BEOR_TILE_ELEMS));
  CKC(c, c->dbar.alloc(sizeof(double2) * (size_t)c->nt * BEOR_TB));
  if (c->model_kind == 1) {
    CKC(c, precompute_dense(c->T.as<double2>(), c->n_vis, c->n, c->ld, c->w.as<double>(), c->d.as<double2>(), c->nt,
                            c->M.as<double2>(), c->dbar.as<double2>(), s, c->precision == BEOR_PREC_MIXED));
  } else {
    DevBuf G, u;
    CKC(c, G.alloc(sizeof(double2) * (size_t)c->nf * c->ncells * c->ncells));
    CKC(c, u.alloc(sizeof(double2) * (size_t)c->nf * c->ncells));
    CKC(c, precompute_factored(c->A.as<double2>(), c->W.as<double2>(), c->nf, c->ntb, c->ncells, c->nx,
                               c->w.as<double>(), c->d.as<double2>(), c->n, c->nt, G.as<double2>(), u.as<double2>(),
                               c->M.as<double2>(), c->dbar.as<double2>(), s));
    CKC(c, cudaStreamSynchronize(s));
  }
  if (c->precision == BEOR_PREC_MIXED) {
    const int64_t ne = tri_count(c->nt) * BEOR_TILE_ELEMS;
    CKC(c, c->Mdf.alloc(sizeof(float4) * (size_t)ne));
    CKC(c, split_double_float(c->M.as<double2>(), ne, c->Mdf.as<float4>(), s));
    const int64_t nf = (int64_t)c->nt * c->nt * BEOR_TILE_ELEMS;
    CKC(c, c->Mf.alloc(sizeof(float4) * (size_t)nf));
    CKC(c, c->Mft.alloc(sizeof(float2) * (size_t)nf));
    CKC(c, split_full_triple(c->M.as<double2>(), c->n, c->nt, c->Mf.as<float4>(), c->Mft.as<float2>(), s));
  }
  CKC(c, cudaStreamSynchronize(s));
  c->have_pre = true;
  return BEOR_OK;
}

static int lnl_multi_impl(beor_ctx* const* ctxs, int nsets, const double* const* phi, const int* B,
                          double* const* lnl_out, int32_t* const* status_out, void* stream, bool need_x,
                          int slot = 0, bool async = false) {
  if (!ctxs || nsets <= 0 || !phi || !B) return BEOR_EINVAL;
  if (async) {
    if (!lnl_out || !status_out) return BEOR_EINVAL;
    for (int s = 0; s < nsets; ++s)
      if (!phi[s] || !lnl_out[s] || !status_out[s] || !is_device_ptr(phi[s]) || !is_device_ptr(lnl_out[s]) ||
          !is_device_ptr(status_out[s]))
        return BEOR_EINVAL;
  }
  for (int s = 0; s < nsets; ++s) {
    int r = check_ready(ctxs[s]);
    if (r) return r;
    if (!ctxs[s]->have_pre) return BEOR_ESTATE;
    if (ctxs[s]->device != ctxs[0]->device || ctxs[s]->precision != ctxs[0]->precision) return BEOR_EINVAL;
    if (B[s] <= 0 || B[s] > 4096 || !phi[s]) return BEOR_EINVAL;
  }
  beor_ctx* c0 = ctxs[0];
  cudaSetDevice(c0->device);
  cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lk(g_mu);
  need_x = need_x && ctxs[0]->precision == BEOR_PREC_MIXED;
  Plan* pl = find_plan(ctxs, nsets, B, need_x, slot);
  if (!pl) {
    int r = build_plan(ctxs, nsets, B, need_x, slot, &pl);
    if (r) return r;
    g_plans.push_back(pl);
  }
  for (int s = 0; s < nsets; ++s) {
    // validate phi values (finite) on the host when possible
    size_t bytes = sizeof(double) * (size_t)B[s] * ctxs[s]->n_k;
    if (!is_device_ptr(phi[s])) {
      for (size_t i = 0; i < (size_t)B[s] * ctxs[s]->n_k; ++i)
        if (!std::isfinite(phi[s][i])) return BEOR_EINVAL;
    }
    CKC(c0, to_device(pl->phis.as<double>() + pl->phi_off[s], phi[s], bytes, st));
  }
  const bool first_use = !pl->exec;
  if (!pl->exec) {
    // first use: run once directly (sets kernel attributes), then capture
    int64_t nl = 0;
    pl->lookahead = pl->sch.lookahead != 0;
    pl->wait_ns = g_wait_ns;
    pl->skip_copy = g_skip_copy;
    pl->view.wait_ns = g_wait_ns;
    pl->view.test_skip_copy = g_skip_copy;
    CKC(c0, run_sequence(*pl, st, &nl, false));
    pl->launches = nl;
    CKC(c0, cudaStreamSynchronize(st));
    cudaStream_t cs;
    CKC(c0, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    pl->prof = g_profiling;
    if (e == cudaSuccess) e = run_sequence(*pl, cs, nullptr, pl->prof);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&pl->exec, g, 0);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return fail_cuda(c0, e);
    }
    pl->graph = g;
  } else {
    CKC(c0, cudaEventRecord(pl->ev0, st));
    CKC(c0, cudaGraphLaunch(pl->exec, st));
    CKC(c0, cudaEventRecord(pl->ev1, st));
  }
  for (int s = 0; s < nsets; ++s) {
    int f = pl->first[s];
    if (lnl_out && lnl_out[s]) CKC(c0, from_device(lnl_out[s], pl->view.lnl + f, sizeof(double) * B[s], st));
    if (status_out && status_out[s])
      CKC(c0, from_device(status_out[s], pl->view.status + f, sizeof(int32_t) * B[s], st));
  }
  // asynchronous call on a captured batch: done once the work is enqueued
  // (errors of bounded device waits are reported by beor_lnl_multi_wait)
  if (async && pl->launches > 0 && pl->exec && !first_use) return BEOR_OK;
  CKC(c0, cudaStreamSynchronize(st));
  CKC(c0, cudaGetLastError());
  int bounds = 0;
  {
    int fl[2] = {0, 0};   // error, bounds
    CKC(c0, cudaMemcpy(fl, pl->view.flags, sizeof(fl), cudaMemcpyDeviceToHost));
    const int err = fl[0];
    bounds = fl[1];
    if (err) {
      for (int s = 0; s < nsets; ++s) {
        ctxs[s]->poisoned = true;
        ctxs[s]->stats.device_error = err;
      }
      return BEOR_ETIMEOUT;
    }
  }
  float ms = 0.0f;
  if (cudaEventElapsedTime(&ms, pl->ev0, pl->ev1) != cudaSuccess) {
    cudaGetLastError();
    ms = -1.0f;
  }
  // per-class device time (profiled graphs only), and the evaluation's
  // timeline: each launch's interval between its bracketing events (which
  // includes any wait for SMs behind other streams' kernels); the time in
  // which no launch of any stream is in flight is the cost of the graph's
  // dependency edges and launch latencies
  double cls_ms[kClasses] = {0};
  int64_t cls_n[kClasses] = {0};
  double busy_any = -1.0, busy_main = -1.0;
  if (pl->prof && ms >= 0.0f) {
    std::vector<std::pair<double, double>> iv_all, iv_main;
    bool ok = true;
    for (size_t i = 0; i < pl->pcls.size() && 2 * i + 1 < pl->pev.size(); ++i) {
      float t = 0.0f, a = 0.0f, b = 0.0f;
      if (cudaEventElapsedTime(&t, pl->pev[2 * i], pl->pev[2 * i + 1]) == cudaSuccess) {
        cls_ms[pl->pcls[i]] += t;
        cls_n[pl->pcls[i]] += 1;
      } else {
        cudaGetLastError();
      }
      if (cudaEventElapsedTime(&a, pl->ev0, pl->pev[2 * i]) == cudaSuccess &&
          cudaEventElapsedTime(&b, pl->ev0, pl->pev[2 * i + 1]) == cudaSuccess) {
        iv_all.emplace_back(a, b);
        if (i < pl->pstr.size() && pl->pstr[i] == 0) iv_main.emplace_back(a, b);
      } else {
        cudaGetLastError();
        ok = false;
      }
    }
    auto union_len = [](std::vector<std::pair<double, double>>& iv) {
      std::sort(iv.begin(), iv.end());
      double tot = 0.0, cs = -1e300, ce = -1e300;
      for (const auto& x : iv) {
        if (x.first > ce) {
          if (ce > cs) tot += ce - cs;
          cs = x.first;
          ce = x.second;
        } else if (x.second > ce) {
          ce = x.second;
        }
      }
      if (ce > cs) tot += ce - cs;
      return tot;
    };
    if (ok) {
      busy_any = union_len(iv_all);
      busy_main = union_len(iv_main);
    }
  }
  // diagnostics
  std::vector<double> resid(pl->P);
  CKC(c0, cudaMemcpy(resid.data(), pl->view.resid, sizeof(double) * pl->P, cudaMemcpyDeviceToHost));
  for (int s = 0; s < nsets; ++s) {
    beor_ctx* c = ctxs[s];
    c->stats.ms_last = ms;
    c->stats.device_error = 0;
    c->stats.bounds_error = bounds;
    c->stats.kernel_launches = pl->launches;
    c->stats.refine_iters_max = pl->mixed && pl->refine_x ? kRefineIters : 0;
    double mx = 0.0;
    for (int b = 0; b < B[s]; ++b) mx = std::max(mx, resid[pl->first[s] + b]);
    c->stats.resid_rel_max = mx;
    for (int q = 0; q < kClasses; ++q) {
      c->stats.ms_class[q] = cls_ms[q];
      c->stats.n_class[q] = cls_n[q];
    }
    c->stats.ms_busy_any = busy_any;
    c->stats.ms_busy_main = busy_main;
    c->last_plan = pl;
    c->last_first = pl->first[s];
  }
  return BEOR_OK;
}

int beor_lnl_multi(beor_ctx* const* ctxs, int nsets, const double* const* phi, const int* B,
                   double* const* lnl_out, int32_t* const* status_out, void* stream) {
  return lnl_multi_impl(ctxs, nsets, phi, B, lnl_out, status_out, stream, false);
}

int beor_lnl_multi_async(beor_ctx* const* ctxs, int nsets, const double* const* phi, const int* B,
                         double* const* lnl_out, int32_t* const* status_out, int slot, void* stream) {
  if (slot < 0 || slot >= 4) return BEOR_EINVAL;
  return lnl_multi_impl(ctxs, nsets, phi, B, lnl_out, status_out, stream, false, slot, true);
}

int beor_lnl_multi_wait(beor_ctx* const* ctxs, int nsets, const int* B, int slot, void* stream) {
  if (!ctxs || nsets <= 0 || !B || slot < 0 || slot >= 4) return BEOR_EINVAL;
  Plan* pl = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    pl = find_plan(ctxs, nsets, B, false, slot);
  }
  if (!pl) return BEOR_ESTATE;
  beor_ctx* c0 = ctxs[0];
  cudaSetDevice(c0->device);
  CKC(c0, cudaStreamSynchronize((cudaStream_t)stream));
  int err = 0;
  CKC(c0, cudaMemcpy(&err, &pl->view.flags->error, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    for (int s = 0; s < nsets; ++s) {
      ctxs[s]->poisoned = true;
      ctxs[s]->stats.device_error = err;
    }
    return BEOR_ETIMEOUT;
  }
  return BEOR_OK;
}

int beor_lnl(beor_ctx* c, const double* phi, int B, double* lnl_out, int32_t* status_out, void* stream) {
  return beor_lnl_multi(&c, 1, &phi, &B, &lnl_out, &status_out, stream);
}

int beor_posterior_mean(beor_ctx* c, const double* phi, beor_c128* abar_out, int32_t* status_out, void* stream) {
  if (!abar_out) return BEOR_EINVAL;
  int32_t st = 0;
  double l = 0.0;
  int B = 1;
  double* lo = &l;
  int32_t* so = &st;
  int r = lnl_multi_impl(&c, 1, &phi, &B, &lo, &so, stream, true);
  if (r) return r;
  Plan* pl = c->last_plan;
  CKC(c, from_device(abar_out, pl->view.vec_x + pl->h_prob[c->last_first].row_off, sizeof(double2) * c->n,
                     (cudaStream_t)stream));
  CKC(c, cudaStreamSynchronize((cudaStream_t)stream));
  if (status_out) {
    if (is_device_ptr(status_out))
      CKC(c, cudaMemcpy(status_out, &st, sizeof(int32_t), cudaMemcpyHostToDevice));
    else
      *status_out = st;
  }
  return BEOR_OK;
}

int beor_get_model_dims(const beor_ctx* c, int64_t* n_vis, int64_t* n_model, int* n_k) {
  if (!c) return BEOR_EINVAL;
  if (n_vis) *n_vis = c->n_vis;
  if (n_model) *n_model = c->n;
  if (n_k) *n_k = c->n_k;
  return BEOR_OK;
}

int beor_get_M(beor_ctx* c, beor_c128* M_out) {
  int r = check_ready(c);
  if (r) return r;
  if (!c->have_pre || !M_out) return c->have_pre ? BEOR_EINVAL : BEOR_ESTATE;
  cudaSetDevice(c->device);
  std::vector<double2> t((size_t)tri_count(c->nt) * BEOR_TILE_ELEMS);
  CKC(c, cudaMemcpy(t.data(), c->M.p, sizeof(double2) * t.size(), cudaMemcpyDeviceToHost));
  const int64_t n = c->n;
  std::vector<double2> full((size_t)n * n);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j <= i; ++j) {
      int I = (int)(i / BEOR_TB), J = (int)(j / BEOR_TB);
      double2 v = t[(size_t)(tri_index(I, J) * BEOR_TILE_ELEMS + (j % BEOR_TB) * BEOR_TB + (i % BEOR_TB))];
      full[(size_t)(i * n + j)] = v;
      full[(size_t)(j * n + i)] = make_double2(v.x, -v.y);
    }
  if (is_device_ptr(M_out)) {
    CKC(c, cudaMemcpy(M_out, full.data(), sizeof(double2) * full.size(), cudaMemcpyHostToDevice));
  } else {
    std::memcpy(M_out, full.data(), sizeof(double2) * full.size());
  }
  return BEOR_OK;
}

int beor_get_dbar(beor_ctx* c, beor_c128* out) {
  int r = check_ready(c);
  if (r) return r;
  if (!c->have_pre) return BEOR_ESTATE;
  if (!out) return BEOR_EINVAL;
  cudaSetDevice(c->device);
  CKC(c, from_device(out, c->dbar.p, sizeof(double2) * c->n, 0));
  CKC(c, cudaDeviceSynchronize());
  return BEOR_OK;
}

// graphs captured with another setting are rebuilt on their next use
static void drop_stale_graphs() {
  for (Plan* p : g_plans) {
    if ((p->prof != g_profiling || p->wait_ns != g_wait_ns || p->skip_copy != g_skip_copy) && p->exec) {
      cudaGraphExecDestroy(p->exec);
      cudaGraphDestroy(p->graph);
      p->exec = nullptr;
      p->graph = nullptr;
    }
  }
}

int beor_set_profiling(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_profiling = on != 0;
  drop_stale_graphs();
  return BEOR_OK;
}

int beor_set_lookahead(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_lookahead = on != 0;
  drop_plans_with_stale_schedule();
  return BEOR_OK;
}

static int check_shape(beor_ctx* const* ctxs, int nsets, const int* B) {
  if (!ctxs || nsets <= 0 || !B) return BEOR_EINVAL;
  for (int s = 0; s < nsets; ++s) {
    if (!ctxs[s] || B[s] <= 0 || B[s] > 4096) return BEOR_EINVAL;
    if (ctxs[s]->n <= 0) return BEOR_ESTATE;
  }
  return BEOR_OK;
}

int beor_set_schedule(beor_ctx* const* ctxs, int nsets, const int* B, const beor_schedule* sch) {
  int r = check_shape(ctxs, nsets, B);
  if (r) return r;
  if (sch && (sch->rest_ctas < 0 || sch->col_ctas < 0 || sch->rest_ctas > 65535 || sch->col_ctas > 65535))
    return BEOR_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  const std::string key = shape_key(ctxs, nsets, B, false);
  if (sch) {
    beor_schedule c = *sch;
    c.lookahead = c.lookahead != 0;
    c.align_ends = c.align_ends != 0;
    c.reserve_diag = c.reserve_diag != 0;
    g_schedules[key] = c;
  } else {
    g_schedules.erase(key);
  }
  drop_plans_with_stale_schedule();
  return BEOR_OK;
}

int beor_get_schedule(beor_ctx* const* ctxs, int nsets, const int* B, beor_schedule* out) {
  int r = check_shape(ctxs, nsets, B);
  if (r) return r;
  if (!out) return BEOR_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  *out = schedule_of(shape_key(ctxs, nsets, B, false));
  return BEOR_OK;
}

int beor_set_wait_test(int skip_one_copy, double limit_ms) {
  if (!(limit_ms >= 0.0) || limit_ms > 60000.0) return BEOR_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  g_skip_copy = skip_one_copy != 0;
  g_wait_ns = (unsigned long long)(limit_ms * 1e6);
  drop_stale_graphs();
  return BEOR_OK;
}

int beor_get_stats(const beor_ctx* c, beor_stats* out) {
  if (!c || !out) return BEOR_EINVAL;
  *out = c->stats;
  return BEOR_OK;
}

int beor_get_terms(const beor_ctx* c, double* logdet_phi, double* logdet_sigma, double* q, int B) {
  if (!c || !c->last_plan) return BEOR_ESTATE;
  Plan* pl = c->last_plan;
  int f = c->last_first;
  if (B <= 0 || f + B > pl->P) return BEOR_EINVAL;
  cudaSetDevice(c->device);
  if (logdet_phi) CKC(nullptr, cudaMemcpy(logdet_phi, pl->view.logdet_phi + f, sizeof(double) * B, cudaMemcpyDeviceToHost));
  if (logdet_sigma)
    CKC(nullptr, cudaMemcpy(logdet_sigma, pl->view.logdet_sigma + f, sizeof(double) * B, cudaMemcpyDeviceToHost));
  if (q) CKC(nullptr, cudaMemcpy(q, pl->view.q + f, sizeof(double) * B, cudaMemcpyDeviceToHost));
  return BEOR_OK;
}

int beor_get_factor(const beor_ctx* c, int b, beor_c128* L_out) {
  if (!c || !c->last_plan || !L_out) return BEOR_EINVAL;
  Plan* pl = c->last_plan;
  const int p = c->last_first + b;
  if (b < 0 || p >= pl->P || pl->h_prob[p].set != pl->h_prob[c->last_first].set) return BEOR_EINVAL;
  cudaSetDevice(c->device);
  const Prob& pr = pl->h_prob[p];
  const size_t ntile = (size_t)tri_count(pr.nt) * BEOR_TILE_ELEMS;
  std::vector<double2> t(ntile);
  if (pl->mixed) {
    std::vector<float4> f(ntile);
    CKC(nullptr, cudaMemcpy(f.data(), reinterpret_cast<float4*>(pl->view.ws) + pr.ws_off, sizeof(float4) * ntile,
                            cudaMemcpyDeviceToHost));
    for (size_t e = 0; e < ntile; ++e)
      t[e] = make_double2((double)f[e].x + (double)f[e].y, (double)f[e].z + (double)f[e].w);
  } else {
    CKC(nullptr, cudaMemcpy(t.data(), reinterpret_cast<double2*>(pl->view.ws) + pr.ws_off, sizeof(double2) * ntile,
                            cudaMemcpyDeviceToHost));
  }
  const int64_t n = pr.n;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) {
      double2 v = make_double2(0.0, 0.0);
      if (j <= i) {
        int I = (int)(i / BEOR_TB), J = (int)(j / BEOR_TB);
        v = t[(size_t)(tri_index(I, J) * BEOR_TILE_ELEMS + (j % BEOR_TB) * BEOR_TB + (i % BEOR_TB))];
      }
      L_out[i * n + j].re = v.x;
      L_out[i * n + j].im = v.y;
    }
  return BEOR_OK;
}

}  // extern "C"
