/*
 * anova.h -- C ABI of the GB300 ANOVA-NFFT kernel library.
 *
 * The library computes matrix-vector products with the extended Gaussian ANOVA kernel of
 * arXiv 2312.00538 (Wagner, Pearson, Stoll), Sec. 3:
 *
 *     kappa(x_i, x_j) = sum_{l=1}^{P} eta_l exp(-||x_j^{W_l} - x_i^{W_l}||^2 / ell_l^2),
 *     K v = K_1 v + ... + K_P v,
 *
 * each window W_l holding one to three features, and every K_l v evaluated by NFFT-based fast
 * summation (Sec. 3: trigonometric-polynomial kernel of bandwidth N, adjoint NFFT, diagonal
 * scaling by the Fourier coefficients, NFFT). On top of the matvec it provides the low-rank
 * preconditioners of Sec. 4-5 and the interior point method of Sec. 2 (Algorithm 1).
 *
 * Conventions for every entry point:
 *  - Every call returns an anova_status; no C++ exception crosses this boundary. On an error
 *    anova_last_error() returns a message for the calling thread; outputs are then unspecified.
 *  - The caller owns every buffer it passes. Plans and preconditioners own the device memory
 *    they allocate and release it in *_destroy.
 *  - "device" pointers are CUDA global-memory addresses on the device that was current when the
 *    plan was created; "host" pointers are ordinary CPU memory.
 *  - Work is issued on the CUDA stream given at plan creation (NULL = the legacy default
 *    stream). Calls returning device results are asynchronous with respect to the host unless
 *    stated otherwise; synchronise that stream before reading them.
 *  - Points must lie in [-0.2, 0.2] in every feature used by a window (the plan's fit interval
 *    for kernel differences is |t| <= 0.4); otherwise ANOVA_ERR_OUT_OF_RANGE.
 *
 * A plan may be used from one host thread at a time.
 */
#ifndef ANOVA_H
#define ANOVA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct anova_plan *anova_plan_t;
typedef struct lowrank *lowrank_t;

typedef enum {
    ANOVA_OK = 0,
    ANOVA_ERR_INVALID_ARG = 1,   /* a size, flag, pointer or parameter is not allowed */
    ANOVA_ERR_OUT_OF_RANGE = 2,  /* a point coordinate lies outside [-0.2, 0.2] */
    ANOVA_ERR_NONFINITE = 3,     /* an input holds NaN or Inf */
    ANOVA_ERR_OOM = 4,           /* a device or host allocation failed */
    ANOVA_ERR_CUDA = 5,          /* a CUDA runtime call or kernel launch failed */
    ANOVA_ERR_NOT_CONVERGED = 6, /* an iteration hit its limit before its tolerance */
    ANOVA_ERR_BREAKDOWN = 7,     /* a Krylov or factorisation step divided by zero */
    ANOVA_ERR_TIMEOUT = 8        /* a bounded device-side wait gave up */
} anova_status;

/* Plan flags (anova_nfft_plan `flags`): one precision, optionally one interpolation choice.
 * v and Kv use the plan's element type. The interpolation choice only matters for FP32 plans with
 * 3-feature windows and m = 4, which have two kernels computing the same sums: one on the FP32
 * pipe, one forming the inner sums along the last axis on the tensor cores (tf32 operands split
 * into high and low parts, FP32 accumulation). By default the plan picks per window group: the
 * tensor-core kernel when work items hold at least 512 points on average. */
enum {
    ANOVA_FP32 = 0,          /* float spread / FFT / interpolation with float accumulation */
    ANOVA_FP64 = 1,          /* double everywhere (the "precise" plan) */
    ANOVA_INTERP_TENSOR = 2, /* always the tensor-core interpolation where the plan has it */
    ANOVA_INTERP_SIMT = 4    /* never the tensor-core interpolation */
};

/* Low-rank preconditioner kinds (lowrank_precond_build `kind`). */
enum {
    PCHOL_GREEDY = 0, /* Algorithm 2: greedy pivoted Cholesky (Sec. 4) */
    NYSTROM = 1,      /* Nystrom K ~ (KQ)(Q^T K Q)^{-1}(KQ)^T with Q = pivoted columns (Sec. 4) */
    PCHOL_RANDOM = 2, /* randomly pivoted Cholesky: pivots drawn by the residual diagonal (Sec. 4) */
    PCHOL_PER_WINDOW = 3, /* greedy factors of each K_l, stacked: [L_1 ... L_P] (Sec. 4) */
    NYSTROM_RANDOM = 4    /* Nystrom with Q = orth(K G), G Gaussian, by matvecs (Sec. 4) */
};

/*
 * anova_nfft_plan -- build the fast-summation plan for K = sum_l K_l (Sec. 3).
 *
 * points  host, n x d, row-major FP64: point i is points[i*d .. i*d+d-1].
 * windows host, P x 3 int32, 0-based feature indices; a window of one or two features is padded
 *         with -1 after its valid entries (Sec. 3: W_l holds at most three features).
 * sigma   the kernel length scale ell of exp(-r^2/ell^2), shared by all windows; eta_l = 1.
 * N       even bandwidth of the trigonometric polynomial (Sec. 3, N in 2N); 4 <= N <= 256.
 * m       window cut-off of the NFFT (Sec. 3, O(m^d n)); the Kaiser-Bessel window covers 2m
 *         grid points per dimension on an oversampled grid of n_os = 2N points.
 *         FP32 plans accept 2 <= m <= 6, FP64 plans 3 <= m <= 8.
 * flags   ANOVA_FP32 or ANOVA_FP64, optionally | ANOVA_INTERP_TENSOR or | ANOVA_INTERP_SIMT
 *         (not both).
 * cuda_stream  a cudaStream_t (or NULL) on which every later call of this plan is issued.
 * out     receives the plan. The plan copies what it needs; `points` may be freed on return.
 *
 * Errors: INVALID_ARG (n < 1, d < 1, P < 1, bad window entries, N odd or out of range, m out of
 * range, sigma not positive), NONFINITE, OUT_OF_RANGE, OOM, CUDA. Synchronises the stream.
 */
anova_status anova_nfft_plan(const double *points, int64_t n, int d, const int32_t *windows, int P,
                             double sigma, int N, int m, int flags, void *cuda_stream,
                             anova_plan_t *out);

/*
 * anova_nfft_plan_ex -- as anova_nfft_plan, with an individual length scale ell_l and weight
 * eta_l per window (Sec. 3: "each kernel kappa_l is assigned an individual kernel parameter").
 * ell: host, P positive values. eta: host, P finite values, or NULL for all ones.
 */
anova_status anova_nfft_plan_ex(const double *points, int64_t n, int d, const int32_t *windows,
                                int P, const double *ell, const double *eta, int N, int m,
                                int flags, void *cuda_stream, anova_plan_t *out);

/*
 * anova_matvec -- Kv = K v for nrhs right-hand sides (Sec. 3, K v = K_1 v + ... + K_P v).
 *
 * v   device, n x nrhs column-major (column r at v + r*n), element type of the plan.
 * Kv  device, n x nrhs column-major, overwritten. Must not overlap v.
 * nrhs >= 1. Asynchronous on the plan's stream. The first call with a larger nrhs than any
 * earlier call enlarges the plan's workspace (a device allocation). Errors: INVALID_ARG, OOM,
 * CUDA.
 */
anova_status anova_matvec(anova_plan_t plan, const void *v, void *Kv, int nrhs);

/*
 * anova_matvec_host -- as anova_matvec with HOST buffers: copies v to the device, runs the
 * matvec and copies Kv back, then synchronises the plan's stream. Uses plan-owned staging
 * buffers (pinned host memory is faster but not required). After a call the copy in, the
 * matvec and the copy out are kept as one captured CUDA graph for the same (v_host, Kv_host,
 * nrhs); a following call with those buffers launches the graph (same kernels, same results),
 * any other call takes the stream path and captures again. The caller keeps the host buffers
 * valid while the plan may still use them, as with any asynchronous copy. Not thread-safe with
 * other calls on the same plan (as every plan call).
 */
anova_status anova_matvec_host(anova_plan_t plan, const void *v_host, void *Kv_host, int nrhs);

/*
 * anova_window_matvec -- K_l v for the single window l (0 <= l < P) of the plan, nrhs = 1,
 * device buffers of the plan's type (a stage of the same fast summation, for testing and for
 * per-window low-rank factors, Sec. 4 "applied to each individual matrix").
 */
anova_status anova_window_matvec(anova_plan_t plan, int l, const void *v, void *Kv);

/*
 * Stage entry points of one window l (nrhs = 1, device buffers of the plan's type). The grid has
 * n_os^{d_l} entries (n_os = 2N), row-major over the window's features in window order; grid
 * index u in [0, n_os) sits at position u/n_os - 1/2.
 *   anova_spread_grid : grid[u] = sum_i v_i prod_k psi(s_ik - u_k), s = (x + 1/2) n_os.
 *   anova_conv_grid   : out = IDFT(D .* DFT(in)), unnormalised inverse, with
 *                       D_J = eta_l prod_k b_{J_k} / Psi(J_k)^2 on J in I_N^{d_l}, 0 elsewhere.
 *   anova_interp_grid : f_i = sum_u grid[u] prod_k psi(s_ik - u_k), f in original point order.
 * psi is the Kaiser-Bessel window of cut-off m (normalised to psi(0) = 1) and Psi its Fourier
 * transform; b the 1-D Fourier coefficients of the Gaussian (see anova_kernel_coeffs).
 * anova_conv_grid reads every grid entry; the others touch only the footprint of the points.
 */
anova_status anova_spread_grid(anova_plan_t plan, int l, const void *v, void *grid);
anova_status anova_conv_grid(anova_plan_t plan, int l, const void *grid_in, void *grid_out);
anova_status anova_interp_grid(anova_plan_t plan, int l, const void *grid, void *f);

/*
 * Split matvec for a product whose points are split over several plans (row sharding, e.g. one
 * plan per GPU). The inner sum of the fast summation (Sec. 3: the adjoint NFFT, a sum over the
 * points) is additive over any partition of the points, so with the points split over plans
 * built from the same windows, N, m, precision and per-window ell_l, eta_l:
 *   (K v)[rows of plan k] = from_grids(plan k, sum over plans j of grids(plan j, v_j)).
 * anova_plan_grid_size -- grid_total: values of one right-hand side's grids, every window's
 *   n_os^{d_l} grid back to back (the same for all plans with the same windows and N).
 * anova_matvec_grids -- the spread of v (device, n x nrhs column-major, the plan's points) into
 *   every window's oversampled grid: grids (device, nrhs x grid_total, overwritten).
 * anova_matvec_from_grids -- the rest of the product for the plan's points from summed grids
 *   (device, nrhs x grid_total): every window's grid is convolved over the whole grid (FFT,
 *   scaling, inverse FFT; a sum over several plans is not confined to this plan's box), then
 *   interpolated at the plan's points and summed over windows into Kv (device, n x nrhs,
 *   overwritten). With one plan, grids then from_grids equals anova_matvec up to the order of sums.
 * Both run asynchronously on the plan's stream and use the plan's workspace (calls on one plan
 * are ordered by the caller, as for anova_matvec). Errors: INVALID_ARG (NULL, nrhs < 1,
 * overlapping buffers), OOM, CUDA.
 */
anova_status anova_plan_grid_size(anova_plan_t plan, int64_t *grid_total);
anova_status anova_matvec_grids(anova_plan_t plan, const void *v, void *grids, int nrhs);
anova_status anova_matvec_from_grids(anova_plan_t plan, const void *grids, void *Kv, int nrhs);

/*
 * anova_spread_grid_noalloc -- anova_spread_grid (same kernels, same grid) without any device
 * allocation in the call. The paper has no counterpart; this exists for callers that cannot
 * allocate device memory when they call: processes whose device memory is entirely reserved
 * up front by their own pool, and loops with a fixed time budget per call, where cudaMalloc
 * (which may wait for the whole device to become idle) is not acceptable.
 *
 * Scratch: the spread kernel's partial tiles go to one static device array of 16 MiB that the
 * library declares at file scope; every GPU that loads the library holds it until the process
 * exits. The window's tiles must fit: a window needs (its own spread work items)
 * x (B + 2m - 1)^{d_l} elements (B = 4, the bin edge in cells); a larger requirement returns
 * ANOVA_ERR_INVALID_ARG with the sizes in the message (use anova_spread_grid then). The call
 * makes no cudaMalloc, cudaFree or other allocating call; it clears the caller's grid itself.
 *
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture. The address is kept per
 * device ordinal for the life of the process: it does not survive cudaDeviceReset (or any other
 * destruction of the device's primary context), after which this entry point must not be called
 * again in that process. All calls share the one
 * array, which keeps the last call's tiles: calls that can overlap on the GPU (different
 * streams, plans or threads without ordering between them) race on it.
 * Arguments and errors as anova_spread_grid.
 */
anova_status anova_spread_grid_noalloc(anova_plan_t plan, int l, const void *v, void *grid);

/*
 * anova_cross_matvec -- the product with targets distinct from the sources, as in evaluating the
 * trained decision function f(x) = sum_i alpha_i y_i K(x_i, x) + b at new points (Sec. 6):
 *   f_j = sum_l eta_l sum_i w_i exp(-||t_j^{W_l} - s_i^{W_l}||^2 / ell_l^2),   j < n_target,
 * by NFFT fast summation: the sources are spread with `source`'s plan, each window's grid is
 * convolved in full (FFT, scaling, inverse FFT), and the result is interpolated at the targets
 * with `target`'s plan. Both plans must be built from the same windows, N, m, precision and
 * per-window ell_l, eta_l (otherwise ANOVA_ERR_INVALID_ARG); their points (and counts) differ.
 * w: device, n_source values of the plans' precision; f: device, n_target values (overwritten).
 * Allocates two grids of scratch for the call and synchronises both plans' streams; the plans'
 * own matvec state is not touched.
 */
anova_status anova_cross_matvec(anova_plan_t source, anova_plan_t target, const void *w, void *f);

/*
 * Prediction with the source half kept (Sec. 6: the decision function is evaluated at many new
 * points for one trained alpha). anova_cross_matvec redoes the spread and the full convolution of
 * the sources on every call; a model does them once.
 * anova_model_create -- spreads w (device, n_source values of the plan's precision) with
 *   `source`'s plan and convolves every window's grid in full (FFT, scaling, inverse FFT); the
 *   model keeps the convolved grids (n_os^{d_l} values per window, on the plan's device) and
 *   copies of the plan's window parameters, so the plan and w may be released afterwards.
 *   Synchronises the plan's stream. Errors: INVALID_ARG (NULL), OOM, CUDA.
 * anova_model_eval -- f_j = sum_l eta_l sum_i w_i exp(-||t_j^{W_l} - s_i^{W_l}||^2 / ell_l^2) at
 *   the target plan's points (device, n_target values, overwritten): the target plan's
 *   interpolation from the kept grids, then the window sum. The target plan must match the model
 *   as anova_cross_matvec's plans must match (else INVALID_ARG). Asynchronous on the target plan's
 *   stream, like anova_matvec; results equal anova_cross_matvec's up to the order of sums.
 * anova_model_destroy -- frees the grids (NULL is ignored).
 */
typedef struct anova_model *anova_model_t;
anova_status anova_model_create(anova_plan_t source, const void *w, anova_model_t *out);
anova_status anova_model_eval(anova_model_t model, anova_plan_t target, void *f);
void anova_model_destroy(anova_model_t model);

/*
 * anova_nfft_plan_tuned -- anova_nfft_plan_ex (same arguments and errors) followed by a search
 * over launch settings that leave the arithmetic of each point-window product unchanged; the
 * fastest plan is returned. Settings: the points-per-work-item cap of the spread/interpolation
 * work items (1024, 2048, 4096) and then, at the best cap, the grid lines per CTA of the FFT passes
 * (8, 16, 32) (each needs its own plan tables); for FP32 plans with m = 4 and a
 * 3-D window, the tensor-core or the FP32-pipe interpolation (unless `flags` fixes one); right-hand
 * sides per pass (16, 8, 4, below nrhs); for FP64 plans with P >= 2, windows on concurrent streams
 * or not. Each setting is timed over `reps` matvecs with `nrhs` columns (after one warm-up call)
 * with CUDA events on the plan's stream, inputs resident, caches warm (as in Krylov iterations).
 * Results of the returned plan equal the default plan's up to the order of floating-point sums.
 * nrhs in [1, 1024], reps in [1, 1000]; report (may be NULL) receives the choice:
 *   wi_max, interp (ANOVA_INTERP_TENSOR / ANOVA_INTERP_SIMT, 0 if not searched), rhs_chunk,
 *   fork_windows (0/1, 0 if not searched), candidates (settings timed), ms (mean ms per matvec at
 *   the choice), ms_default (the same with anova_nfft_plan_ex's settings), conv_lines.
 * Allocates n * nrhs elements twice for the timing inputs and frees them before returning.
 * Errors: those of anova_nfft_plan_ex; INVALID_ARG (nrhs, reps); TIMEOUT (a kernel wait ran out).
 */
typedef struct {
    int wi_max;
    int interp;
    int rhs_chunk;
    int fork_windows;
    int candidates;
    double ms;
    double ms_default;
    int conv_lines;
} anova_tune_report;

anova_status anova_nfft_plan_tuned(const double *points, int64_t n, int d, const int32_t *windows,
                                   int P, const double *ell, const double *eta, int N, int m,
                                   int flags, void *cuda_stream, int nrhs, int reps,
                                   anova_tune_report *report, anova_plan_t *out);

/*
 * Batched matvecs of independent problems: the matvecs of `count` plans (different points,
 * sizes, windows or precision; each plan at most once) captured as one CUDA graph, each plan's
 * stage chain on its own branch, so one launch runs them all concurrently.
 * anova_matvec_batch_create -- plans[k], v[k], Kv[k] (device, n_k x nrhs[k] of plan k's type,
 *   column-major; nrhs may be NULL for 1 each) are fixed into the graph: a run reads v[k] and
 *   overwrites Kv[k] as anova_matvec(plans[k], v[k], Kv[k], nrhs[k]) does, with identical
 *   results. Runs each matvec once before capturing (Kv is written), on each plan's stream, and
 *   synchronises. cuda_stream: the stream the graph is launched on (NULL = default stream).
 *   The plans must outlive the batch and not have stage timing on. Errors: INVALID_ARG (NULL,
 *   count outside [1, 4096], a plan twice, plans on several devices), OOM, CUDA.
 *   The graph uses each plan's own workspace buffers (grids, tiles, per-window results) as they
 *   were when it was captured. A plan's own calls and the batch's runs therefore share those
 *   buffers: the caller orders them (same stream, or events). A later call on a plan with more
 *   right-hand sides than the plan's workspace holds reallocates it; the batch then refuses to
 *   run (INVALID_ARG) and must be created again.
 * anova_matvec_batch_run -- one launch of the graph (asynchronous on the batch's stream).
 *   Errors: INVALID_ARG (NULL batch, or a plan's workspace reallocated since the capture), CUDA.
 * anova_matvec_batch_destroy -- frees the graph (NULL is ignored).
 */
typedef struct anova_batch *anova_batch_t;
anova_status anova_matvec_batch_create(int count, anova_plan_t const *plans, const void *const *v,
                                       void *const *Kv, const int *nrhs, void *cuda_stream,
                                       anova_batch_t *out);
anova_status anova_matvec_batch_run(anova_batch_t batch);
void anova_matvec_batch_destroy(anova_batch_t batch);

/* Plan facts. Any output pointer may be NULL. device_bytes = device memory the plan holds. */
anova_status anova_plan_info(anova_plan_t plan, int64_t *n, int *P, int *n_os, int *flags,
                             int64_t *device_bytes);

/*
 * Per-stage timing of anova_matvec (CUDA events recorded on the plan's stream between the
 * stages). Stages: ANOVA_STAGE_SPREAD (adjoint-NFFT spreading), ANOVA_STAGE_REDUCE (partial-tile
 * reduction onto the grid), ANOVA_STAGE_FFT (FFT / scaling / inverse FFT passes),
 * ANOVA_STAGE_INTERP (NFFT interpolation), ANOVA_STAGE_SUM (sum over windows).
 * anova_plan_set_timing: turns recording on (enable != 0) or off and clears what was recorded.
 * anova_plan_stage_times: synchronises the stream and returns in ms[ANOVA_NUM_STAGES] the total
 *   milliseconds per stage since the last reset, and in *launches the number of kernels the plan
 *   launched since then (counted whether or not timing is on). Either output may be NULL.
 */
enum {
    ANOVA_STAGE_SPREAD = 0,
    ANOVA_STAGE_REDUCE = 1,
    ANOVA_STAGE_FFT = 2,
    ANOVA_STAGE_INTERP = 3,
    ANOVA_STAGE_SUM = 4,
    ANOVA_NUM_STAGES = 5
};
anova_status anova_plan_set_timing(anova_plan_t plan, int enable);
anova_status anova_plan_stage_times(anova_plan_t plan, double *ms, int64_t *launches);

/*
 * Synchronises the plan's stream and reports kernel-side failures of the calls made so far:
 * ANOVA_ERR_TIMEOUT if a bounded wait inside a kernel ran out (the affected outputs are not
 * valid; the flag stays set), ANOVA_ERR_CUDA for the stream's CUDA error; ANOVA_OK otherwise. Kernels never trap or
 * spin without bound: a tensor-core completion that does not arrive within about a second makes
 * the kernel skip the dependent work, set the flag and return.
 */
anova_status anova_plan_check(anova_plan_t plan);

/*
 * anova_plan_set_wait_limit -- failure-detection hook: the number of polls each chunk's
 * tensor-core completion wait in the FP32 3-D interpolation makes before it gives up (default
 * 2^22, about a second; polls < 0 restores it, larger values are clamped to it). 0 makes every
 * such wait give up without polling, so the kernel takes its timeout path at its first chunk:
 * it sets the plan's flag (anova_plan_check then returns ANOVA_ERR_TIMEOUT), still waits with
 * the full limit for the products it started before it frees its tensor memory, and returns.
 * The results of calls made under a lowered limit are not valid. Synchronises the stream.
 * The paper has no counterpart (it concerns the kernels' own failure handling).
 */
anova_status anova_plan_set_wait_limit(anova_plan_t plan, int64_t polls);

/*
 * anova_measure_fp32_peak -- measures the FP32 multiply-add rate of the current GPU in TFLOP/s
 * (independent paired FMA chains on every SM, best of five CUDA-event-timed launches; a few
 * milliseconds). It is the measured roofline denominator of the spread and interpolation kernels,
 * which are bound by the FP32 pipe rather than by memory. The paper has no counterpart.
 * Errors: INVALID_ARG (NULL), CUDA.
 */
anova_status anova_measure_fp32_peak(double *tflops);

/* Release a plan and its device memory (NULL is ignored). Synchronises its stream. */
void anova_plan_destroy(anova_plan_t plan);

/*
 * Host-only plan mathematics, exported so that they can be checked without a GPU.
 *
 * anova_kernel_coeffs: the 1-D Fourier coefficients b_0..b_{N/2-1} of the trigonometric
 *   polynomial b_0 + 2 sum_{k>=1} b_k cos(2 pi k t) fitted (least squares, FP64) to
 *   exp(-t^2/ell^2) on |t| <= 0.4; b_{-N/2} = 0 (Sec. 3, kappa~ with bandwidth N).
 *   b: host, N/2 doubles.
 * anova_window_hat: Psi(k) = int psi(t) cos(2 pi k t / n_os) dt for k = 0..count-1, the
 *   transform of the normalised Kaiser-Bessel window of cut-off m on a grid of n_os points.
 */
anova_status anova_kernel_coeffs(double ell, int N, double *b);
anova_status anova_window_hat(int m, int n_os, int count, double *Psi);

/* Thread-local message of the last error of this thread ("" if none). Never NULL. */
const char *anova_last_error(void);

/* Library version string. */
const char *anova_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ANOVA_H */
