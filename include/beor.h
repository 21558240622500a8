/*
 * beor.h -- C ABI of the GB300 BayesEoR likelihood library.
 *
 * The library evaluates, for batches of prior points phi, the marginal
 * likelihood of the joint EoR + foreground linear model that the paper's
 * sampler explores (Sec. "Statement of need": the amplitudes are marginalised
 * so that the power spectrum is sampled directly from its marginal posterior;
 * Eq. for P(k_i): one power amplitude per spherical k shell):
 *
 *     Sigma(phi) = T^H N^-1 T + Phi(phi)^-1,     dbar = T^H N^-1 d
 *     abar       = Sigma^-1 dbar
 *     lnL(phi)   = -1/2 log|Phi| - 1/2 log|Sigma| + 1/2 dbar^H Sigma^-1 dbar
 *
 * T is the instrument forward model (Sec. "Running BayesEoR": primary beam
 * and uv sampling of each baseline), N the diagonal noise covariance and
 * Phi the diagonal prior.  EoR model amplitude j in k bin kbin[j] has prior
 * variance 10^phi[kbin[j]]; foreground (LSSM) amplitudes, kbin[j] == -1, have
 * the fixed variance lssm_prior_var.
 *
 * Conventions for every call:
 *  - Return value: BEOR_OK or a negative BEOR_E* code.  After BEOR_ECUDA or
 *    BEOR_ETIMEOUT the context is poisoned and later calls return
 *    BEOR_ESTATE.  beor_strerror() names a code.
 *  - Ownership: the caller owns every buffer it passes.  Inputs are copied
 *    (host or device memory, detected per pointer) before the call returns
 *    or, for stream-ordered calls, before the work enqueued on the stream
 *    reads them; no caller pointer is retained.  Output buffers may be host
 *    or device memory.  Host outputs are written when the call returns
 *    (the call synchronises the stream); device outputs are valid once the
 *    given stream reaches the end of the enqueued work.
 *  - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).
 *  - Order: a model (beor_set_T or beor_set_instrument), then beor_set_data,
 *    then beor_precompute, then beor_lnl / beor_lnl_multi /
 *    beor_posterior_mean; otherwise BEOR_ESTATE.
 *  - Threads: one context must not be used by two threads at once.
 *  - Complex numbers are beor_c128 {re, im} pairs (same layout as
 *    std::complex<double> / numpy complex128); matrices are row-major.
 *  - Per-point status: 0 = ok; j > 0 = Sigma not positive definite at
 *    1-based column j (lnL = -inf); -1 = the mixed-precision result may be
 *    outside its tolerance (lnL still returned): for beor_lnl /
 *    beor_lnl_multi, the estimated error of the residual-corrected
 *    quadratic form is above 1e-2; for beor_posterior_mean, the last
 *    iterative-refinement correction is above 1e-4 of the solution;
 *    -2 = the point's phi (passed in device memory) is not finite: the
 *    point is skipped and its lnL is NaN (phi in host memory is checked
 *    before launch instead, BEOR_EINVAL).
 */
#ifndef BEOR_H
#define BEOR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct beor_ctx beor_ctx;
typedef struct { double re, im; } beor_c128;

enum {
  BEOR_OK = 0,
  BEOR_EINVAL = -1,    /* bad argument (size, pointer, value) */
  BEOR_ENOMEM = -2,    /* device or host allocation failed */
  BEOR_ECUDA = -3,     /* a CUDA call or kernel failed */
  BEOR_ETIMEOUT = -4,  /* a bounded device-side wait gave up */
  BEOR_ESTATE = -5,    /* call out of order, or context poisoned */
  BEOR_ENOTSUP = -6    /* feature not available on this device */
};

enum { BEOR_PREC_FP64 = 0, BEOR_PREC_MIXED = 1 };

/* Create a context on CUDA device `device`.
 * precision = BEOR_PREC_FP64: every step in IEEE float64 (the comparator).
 * precision = BEOR_PREC_MIXED: trailing and panel updates of the blocked
 *   Cholesky run as exact bf16 slice products on the tensor cores with fp32
 *   accumulation, the working matrix is kept as a pair of fp32 words per
 *   real number, the diagonal-block Cholesky factorisations and the
 *   log-determinants are float64 (the blocks' inverses are formed on the
 *   fp32 pipe to ~2^-48), and a float64-accurate residual against the
 *   float64 precompute corrects the quadratic form (lnL) or refines the
 *   solution (posterior mean). */
int beor_create(beor_ctx **out, int device, int precision);
int beor_destroy(beor_ctx *ctx);

/* Dense instrument model (Sec. "Running BayesEoR"; T maps model amplitudes
 * to visibilities).  T: n_vis x n_model complex, row-major with leading
 * dimension ld >= n_model, host or device.  kbin: n_model int32 in
 * [-1, n_k); -1 marks a foreground amplitude.  n_k >= 1.
 * lssm_prior_var > 0.  Errors: BEOR_EINVAL for sizes <= 0, a kbin value
 * out of range or an empty k bin. */
int beor_set_T(beor_ctx *ctx, const beor_c128 *T, int64_t n_vis, int64_t n_model,
               int64_t ld, const int32_t *kbin, int n_k, double lssm_prior_var);

/* Factored instrument model: T[(f,tb),(c,x)] = A[f][tb][c] * W[f][x], the
 * per-frequency response of each baseline/time to each uv cell times the
 * spectral basis (eta modes and foreground spectra) of each model column.
 * A: nf x ntb x ncells complex (row-major), W: nf x nx complex; the model
 * index is j = c*nx + x and the visibility index (f*ntb + tb).  The
 * precompute then never forms T.  Same kbin / n_k / lssm_prior_var rules as
 * beor_set_T with n_model = ncells*nx. */
int beor_set_instrument(beor_ctx *ctx, const beor_c128 *A, const beor_c128 *W, int nf,
                        int64_t ntb, int ncells, int nx, const int32_t *kbin, int n_k,
                        double lssm_prior_var);

/* Instrument geometry (all host memory, copied).  Sec. "Running BayesEoR":
 * the instrument model is the primary beam and the uv sampling. */
typedef struct {
  int nu;                        /* uv grid side, odd, 3..255: cells |i_u|, |i_v| <= (nu-1)/2, (0,0) removed */
  int nf;                        /* frequency channels (= eta modes) */
  int nf_grid;                   /* channels of the band that sets the uv cell (0 = nf): sub-bands of
                                    one band pass the band's count so that they share its grid */
  int n_lssm;                    /* foreground spectra (0..8) */
  int n_pix;                     /* sky pixels per side (2..256) */
  int n_bl, n_t, n_k;            /* baselines, time samples, k shells */
  double f0_hz, df_hz;           /* channel f at f0 + f df */
  double beam_fwhm_rad;          /* achromatic Gaussian primary beam */
  double latitude_rad;           /* array latitude; drift scan pointed at the zenith */
  double lssm_prior_var;         /* prior variance of every foreground amplitude */
  const double *bl_enu_m;        /* n_bl x 3: east, north, up (metres) */
  const double *hour_angle_rad;  /* n_t hour angles of the pointing */
  const double *lssm_beta;       /* n_lssm spectral indices (may be NULL when n_lssm = 0) */
} beor_instrument_desc;

/* Builds the factored instrument from its geometry on the device and sets
 * it as beor_set_instrument would: per channel f, A_f = NUDFT_f . diag(beam)
 * . F_uv (the uv cells to an n_pix x n_pix sky grid by the unitary inverse
 * 2-D DFT, the Gaussian beam, and each baseline / time sample's response
 * exp(-2 pi i (u l + v m)) at its uv point in wavelengths at f), rows
 * (t * n_bl + b); W = [E | S], E the unitary inverse eta-DFT over the
 * channels (eta = -nf/2 .. nf/2 - 1), S the power laws (f/f0)^-beta, each
 * column of unit 2-norm; model index j = c * (nf + n_lssm) + x, cells c
 * with i_u fastest.  The uv cell du = (longest baseline at the top channel
 * of nf_grid) / ((nu-1)/2), the sky grid spans 1 / du.  k bins: |k| =
 * sqrt(i_u^2 + i_v^2 + eta^2) of the EoR modes, n_k log-spaced shells from
 * the smallest to the largest |k| (k_i <= |k| < k_(i+1), the largest in the
 * last shell); foreground modes -1.  Visibility index (f * n_t + t) * n_bl
 * + b, so beor_set_data takes d and the noise in that order.  Errors:
 * BEOR_EINVAL for sizes or values out of range, a zero-length baseline set,
 * or an empty k shell; BEOR_ENOMEM. */
int beor_set_instrument_desc(beor_ctx *ctx, const beor_instrument_desc *desc);

/* Data vector d (n_vis complex) and noise variances (n_vis, all > 0): the
 * diagonal of N.  Host or device. */
int beor_set_data(beor_ctx *ctx, const beor_c128 *d, const double *noise_var);

/* One-off precompute of M = T^H N^-1 T (float64, Hermitian, lower triangle
 * authoritative) and dbar = T^H N^-1 d, enqueued on `stream` and completed
 * before return. */
int beor_precompute(beor_ctx *ctx, void *stream);

/* lnL for B prior points.  phi: B x n_k float64, row-major, log10 power
 * amplitudes (host or device).  lnl_out: B float64, status_out: B int32
 * (host or device).  The whole batch is factorised together; the call
 * returns after the results are written.  1 <= B <= 4096 (BEOR_EINVAL
 * otherwise, including an empty batch); non-finite phi in host memory is
 * BEOR_EINVAL.
 * Workspaces: the first call for a batch shape (its contexts and their B;
 * lnL, posterior mean and each asynchronous slot count separately)
 * allocates that batch's device workspaces -- per point the packed lower
 * triangle of Sigma at 16 bytes per complex element (about 92 MB at
 * n_model = 3280, 1.07 GB at 11,424) plus bf16 slices and vectors -- and
 * captures its CUDA graph (BEOR_ENOMEM if they do not fit).  Both are kept
 * for later calls of the same shape and released when one of its contexts
 * is re-set (beor_set_T, beor_set_instrument, beor_set_data,
 * beor_precompute) or destroyed, so callers with varying B should use a
 * few sizes (e.g. pad to powers of two).
 * Mixed precision: the quadratic form q = dbar^H Sigma^-1 dbar is evaluated
 * from the first solution x~ of the approximate factor L~ and one float64
 * residual r = dbar - Sigma x~ as q = dbar^H x~ + x~^H r + |L~^-1 r|^2
 * (exact up to the factor error of the last, second-order term). */
int beor_lnl(beor_ctx *ctx, const double *phi, int B, double *lnl_out, int32_t *status_out,
             void *stream);

/* Batched evaluation across several contexts (e.g. sub-band problems of
 * uneven model dimension), all on one device with one precision: set s
 * evaluates B[s] points phi[s] (B[s] x n_k[s]) into lnl_out[s], status_out[s].
 * One batched factorisation covers every problem of every set. */
int beor_lnl_multi(beor_ctx *const *ctxs, int n_sets, const double *const *phi, const int *B,
                   double *const *lnl_out, int32_t *const *status_out, void *stream);

/* Asynchronous form of beor_lnl_multi, for callers with several independent
 * batches (e.g. a sampler's training set): `slot` (0..3) selects one of up
 * to four independent copies of the batch's workspaces, so that batches
 * enqueued on different streams with different slots run concurrently and
 * the latency-bound last block steps of one overlap the heavy steps of the
 * next.  phi, lnl_out and status_out must be device memory (BEOR_EINVAL
 * otherwise).  The first call for a batch shape and slot runs synchronously
 * (it captures the batch's graph); later calls return once the work is
 * enqueued on `stream`, and the outputs are valid when the stream reaches
 * that point.  Calls on one slot must be ordered (same stream, or ordered
 * by the caller); calls on different slots share only read-only data.
 * beor_lnl_multi_wait synchronises `stream` and reports a bounded
 * device-side wait that gave up (BEOR_ETIMEOUT); beor_get_stats reflects
 * synchronous calls only. */
int beor_lnl_multi_async(beor_ctx *const *ctxs, int n_sets, const double *const *phi, const int *B,
                         double *const *lnl_out, int32_t *const *status_out, int slot, void *stream);
int beor_lnl_multi_wait(beor_ctx *const *ctxs, int n_sets, const int *B, int slot, void *stream);

/* Posterior mean (maximum-a-posteriori amplitudes) abar = Sigma^-1 dbar for
 * one prior point phi (n_k).  abar_out: n_model complex (host or device). */
int beor_posterior_mean(beor_ctx *ctx, const double *phi, beor_c128 *abar_out,
                        int32_t *status_out, void *stream);

int beor_get_model_dims(const beor_ctx *ctx, int64_t *n_vis, int64_t *n_model, int *n_k);

/* Copies of the precompute for inspection: M (n_model x n_model, full
 * Hermitian, row-major) and dbar (n_model).  Host or device output. */
int beor_get_M(beor_ctx *ctx, beor_c128 *M_out);
int beor_get_dbar(beor_ctx *ctx, beor_c128 *dbar_out);

/* Diagnostics of the last lnL / posterior-mean call on this context.
 * ms_class / n_class: device time and launch count per kernel class
 * (0 prior+init, 1 diagonal block, 2 slicing, 3 panel, 4 trailing update,
 * 5 triangular solves, 6 float64-accurate residual (and refinement update), 7 lnL), filled only
 * when profiling is on (beor_set_profiling); ms_last is -1 on the call that
 * captures a batch's graph. */
typedef struct {
  int refine_iters_max;     /* refinement steps taken (posterior mean; 0 for lnL calls) */
  double resid_rel_max;     /* posterior mean: largest last refinement correction ||d|| / ||x||;
                               mixed lnL: largest sqrt(|L~^-1 r|^2 / q), the relative error of
                               x~ in the Sigma norm */
  double ms_last;           /* device time of the last batched evaluation */
  int64_t kernel_launches;  /* kernels launched by the last batched evaluation */
  double ms_class[8];
  int64_t n_class[8];
  int32_t device_error;     /* after BEOR_ETIMEOUT: the bounded wait that gave up first (11 copy
                               producer, 12 tensor-core issuer waiting for operands, 13 issuer
                               waiting for the accumulators, 14 epilogue); 0 otherwise */
  double ms_busy_any;       /* profiling on: time of the last evaluation during which a kernel of
                               any stream was launched and not finished (the union of the
                               launches' intervals between their bracketing events); ms_last minus
                               this is the time lost to the graph's dependencies and launch
                               latencies.  -1 when not measured */
  double ms_busy_main;      /* the same for the launches of the main stream alone */
  int32_t bounds_error;     /* bounds-checked builds (beor_build_info() & 1): code of the first index
                               check of the last evaluation that failed (the access was skipped);
                               0 = none.  Always 0 in the regular build */
} beor_stats;
int beor_get_stats(const beor_ctx *ctx, beor_stats *out);

/* Process-wide switch: when on, batched evaluations record a CUDA event
 * before and after every kernel (inside the captured graph, on the kernel's
 * own stream) and report per-class device times in beor_stats; under the
 * look-ahead schedule launches of different classes overlap, so the class
 * times add up to more than ms_last.  Costs a few microseconds per kernel. */
int beor_set_profiling(int on);

/* Process-wide switch of the mixed-precision factorisation schedule (default
 * on).  On: look-ahead -- block step k's trailing update is split into the
 * next block column and the rest; the rest runs on a second, low-priority
 * stream while the diagonal block, slicing and panel of step k + 1 run at high
 * priority (the same blocked right-looking Cholesky, reordered as a task
 * graph: every tile sees the same operations, so the results are identical).
 * Off: one stream, steps in order.
 * Float64 contexts always use the in-order schedule. */
int beor_set_lookahead(int on);

/* Schedule of the batched mixed-precision factorisation (the blocked
 * right-looking Cholesky of every problem of a batch, run as a sequence of
 * batched launches per block step, captured in one CUDA graph).  None of
 * these settings changes an operation on any tile: factors and
 * log-determinants are identical under every schedule (the float64
 * residual of the quadratic form sums with atomics, so lnL may differ in
 * its last bits).
 *   lookahead:  1 = block step k's trailing update is split into the next
 *               block column (high priority, main stream) and the rest
 *               (low priority, second stream), so that the diagonal block,
 *               slicing and panel of step k + 1 overlap the rest of step k;
 *               0 = one stream, steps in order.
 *   rest_ctas:  CTAs of each launch that updates block columns j >= k + 2
 *               (persistent, tiles from a counter); 0 = one per SM.  Fewer
 *               leave SMs to the main stream's kernels.
 *   col_ctas:   the same for the next-column update and the panel product.
 *   align_ends: 1 = in a batch of uneven sizes, smaller problems start late
 *               so that all end on the last block step (their light final
 *               steps overlap); 0 = all start on step 0.
 *   reserve_diag: 1 = each launch for columns j >= k + 2 also leaves free as
 *               many SMs as step k + 1 has diagonal blocks (one CTA per
 *               problem, running beside it at high priority), so that they
 *               start at once; 0 = no such reserve. */
typedef struct {
  int lookahead;
  int rest_ctas;
  int col_ctas;
  int align_ends;
  int reserve_diag;
} beor_schedule;

/* Set (sch != NULL) or reset to the default (NULL) the schedule of lnL
 * evaluations of one batch shape: the model dimensions of ctxs (in order),
 * their B and their precision.  Batches of that shape built under another
 * schedule are released and rebuilt on their next use.  Default: lookahead
 * as beor_set_lookahead, rest_ctas = col_ctas = 0, align_ends = 1.
 * BEOR_EINVAL for B out of 1..4096 or negative CTA counts; BEOR_ESTATE for
 * a context without a model. */
int beor_set_schedule(beor_ctx *const *ctxs, int n_sets, const int *B, const beor_schedule *sch);
int beor_get_schedule(beor_ctx *const *ctxs, int n_sets, const int *B, beor_schedule *out);

/* Autotuner of the schedule for one batch shape (precomputed contexts,
 * phi[s]: B[s] x n_k points in host or device memory, as for
 * beor_lnl_multi).  If cache_path names a file holding an entry for this
 * device and shape, that schedule is applied and returned without timing.
 * Otherwise every candidate -- look-ahead on with rest_ctas in {one per SM,
 * 8, 16, 24 fewer}, align_ends in {1, 0} and reserve_diag in {0, 1}, and
 * look-ahead off with align_ends in {1, 0} -- is applied and timed: one
 * untimed evaluation (building the batch and its graph), then `reps`
 * evaluations (1..100), the fastest device time counting; the two fastest
 * and the default are then timed again, in turn, twice.  The fastest
 * candidate is applied
 * (beor_set_schedule) and, with cache_path, appended to the cache (one JSON
 * object per line).  chosen, ms_chosen (its time per evaluation) and
 * ms_default (the default schedule's time, -1 when read from the cache
 * without it) may be NULL.  Float64 contexts have only the in-order
 * schedule; the call then times it alone.  Allocates each candidate's
 * workspaces in turn; BEOR_ENOMEM if one does not fit. */
int beor_autotune(beor_ctx *const *ctxs, int n_sets, const double *const *phi, const int *B, int reps,
                  const char *cache_path, beor_schedule *chosen, double *ms_chosen, double *ms_default);

/* Test hook of the failure detection of the tensor-core kernels (process
 * wide, off by default: beor_set_wait_test(0, 0)).  Each role of those
 * kernels (copy producer, tensor-core issuer, epilogue) waits on the others
 * with a bounded wait; when one gives up, the kernel records which wait it
 * was, drains the copies and tensor-core work it issued, releases its
 * tensor memory and returns, and the call reports BEOR_ETIMEOUT (the
 * context is then poisoned).  limit_ms > 0 sets the role-wait limit
 * (0 = the default 2000 ms; the drain keeps its own 2 s limit);
 * skip_one_copy != 0 makes the first trailing-update CTA of the next
 * evaluations withhold one operand copy, so that the issuer's wait for it
 * can only end by the limit.  Graphs captured with other settings are
 * rebuilt on their next use.  BEOR_EINVAL for limit_ms < 0 or > 60000. */
int beor_set_wait_test(int skip_one_copy, double limit_ms);

/* Per-point log-determinant pieces of the last beor_lnl call on ctx (B
 * values each, host memory): log|Phi|, log|Sigma| and q = dbar^H abar. */
int beor_get_terms(const beor_ctx *ctx, double *logdet_phi, double *logdet_sigma, double *q,
                   int B);

/* Cholesky factor L (n_model x n_model, lower, row-major, host memory) of
 * prior point b of the last beor_lnl call on ctx, as left in the working
 * matrix by the factorisation (diagnostics and tests).
 * Both read the last batch's workspaces: once any context of that batch is
 * re-set or destroyed, beor_get_terms returns BEOR_ESTATE and
 * beor_get_factor BEOR_EINVAL until the next evaluation. */
int beor_get_factor(const beor_ctx *ctx, int b, beor_c128 *L_out);

/* dbar = T^H N^-1 d of a factored instrument (same arguments and result as
 * the dbar of beor_set_instrument + beor_set_data + beor_precompute), for
 * callers that cannot allocate device memory -- e.g. code running where
 * another framework already owns all device memory in its own pool, or a
 * loop that must never stall on cudaMalloc / cudaFree.  This call allocates
 * nothing: the per-frequency partial sums live in a fixed 1 MiB device
 * array built into the library, so it needs nf * ncells <= 65536 and
 * returns BEOR_EINVAL beyond that.  All pointers must be memory of the
 * current device, or managed memory (BEOR_EINVAL otherwise, host memory and
 * other GPUs' memory included): A nf x ntb x ncells, W nf x nx, noise_var and d
 * nf*ntb, dbar_out ncells*nx.  The work is enqueued on `stream`; dbar_out
 * is valid when the stream reaches it.  The first call on a device looks up
 * the array's device address (make that first call before any stream
 * capture).  Every call reuses the same array, so calls that may overlap on
 * the GPU (different streams, or other host threads) race and must be
 * serialised by the caller.  The paper has no counterpart of this call. */
int beor_dbar_factored_noalloc(const beor_c128 *A, const beor_c128 *W, int nf, int64_t ntb,
                               int ncells, int nx, const double *noise_var, const beor_c128 *d,
                               beor_c128 *dbar_out, void *stream);

/* ---------------------------------------------------------------------
 * Learned emulator of lnL(phi) (pre-screening for the nested sampler).
 * The paper samples phi with nested sampling (Sec. "Summary": MultiNest,
 * with the evidence used for model selection); this emulator is an
 * addition of this library that the paper does not have: it only screens
 * candidate points, while every accepted point and the evidence use the
 * exact likelihood above.
 * A multilayer perceptron n_in -> depth x width GELU -> 1 with bf16 weights
 * and activations, fp32 accumulation and fp32 master weights / Adam state,
 * trained and evaluated by the library's own kernels.  Inputs and targets
 * are float32 (the network's own precision; callers convert the float64
 * phi and lnL), and training is one Adam step per call
 * (beor_mlp_train_step) so that the caller owns the epoch loop, the
 * minibatch order and the learning-rate schedule.
 * ------------------------------------------------------------------- */
typedef struct beor_mlp beor_mlp;

/* Create on `device`; weights drawn from a counter-based generator seeded
 * by `seed` (He-uniform).  width must be a multiple of 16, 16 <= width <=
 * 256, 1 <= depth <= 8, 1 <= n_in <= 16. */
int beor_mlp_create(beor_mlp **out, int device, int n_in, int width, int depth, uint64_t seed);
int beor_mlp_destroy(beor_mlp *mlp);

/* Input / target normalisation applied inside the network:
 * x_used = (x - x_shift) * x_scale per input, y = y_net * y_scale + y_shift. */
int beor_mlp_set_norm(beor_mlp *mlp, const float *x_shift, const float *x_scale, float y_shift,
                      float y_scale);

/* One Adam step (beta1, beta2, eps given) on a minibatch: x n x n_in float32,
 * y n float32 (host or device).  loss_out (host, may be NULL): mean squared
 * error of the minibatch before the step, in normalised units. */
int beor_mlp_train_step(beor_mlp *mlp, const float *x, const float *y, int n, float lr,
                        float beta1, float beta2, float eps, float *loss_out, void *stream);

/* Predictions for n points (x: n x n_in float32, y_out: n float32; host or
 * device). */
int beor_mlp_infer(beor_mlp *mlp, const float *x, int n, float *y_out, void *stream);

/* Parameter access (fp32 master copy) for checking against the oracle:
 * layer l (0..depth) weights W_l (out x in, row-major) and biases b_l.
 * Sizes: layer 0 is width x n_in, hidden layers width x width, the last
 * 1 x width. */
int beor_mlp_get_params(beor_mlp *mlp, int layer, float *W, float *b);
int beor_mlp_set_params(beor_mlp *mlp, int layer, const float *W, const float *b);

/* Gradients (fp32) of the mean squared loss of one batch with respect to
 * every parameter, written into the caller's buffers in the same layout as
 * beor_mlp_get_params, without updating the weights. */
int beor_mlp_grad(beor_mlp *mlp, const float *x, const float *y, int n, int layer, float *dW,
                  float *db, float *loss_out);

const char *beor_strerror(int code);

/* Name of the CUDA error behind the calling thread's last BEOR_ECUDA or
 * BEOR_ENOMEM ("cudaSuccess" if none). */
const char *beor_last_cuda_error(void);

/* Build variant: bit 0 set = the bounds-checked build (compiled with
 * BEOR_BOUNDS_CHECK), in which the factorisation, solve and residual kernels
 * check their packed-tile, slice-plane, vector and tensor-map indices,
 * record the first failure in beor_stats.bounds_error and skip the access
 * (nothing traps).  The stand-in for a device memory checker. */
int beor_build_info(void);

#ifdef __cplusplus
}
#endif

#endif /* BEOR_H */
