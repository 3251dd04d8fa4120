/*
 * anova_svm.h -- low-rank preconditioners and the SVM interior point method of arXiv 2312.00538
 * (Wagner, Pearson, Stoll) on top of the ANOVA-NFFT matvec of anova.h.
 *
 * The dual soft-margin SVM (Sec. 1, eq. (kernelsvm)): max_alpha e^T alpha - 1/2 alpha^T Y K Y alpha
 * subject to 0 <= alpha_i <= C, y^T alpha = 0, with the ANOVA kernel K of anova.h. The interior
 * point method is Algorithm 1 (Sec. 2); every Newton system (Sec. 2, eq. (Newton))
 *     [[Y K Y + Theta, -y], [-y^T, 0]] [d_alpha; d_lambda] = rhs
 * is solved by preconditioned MINRES (Secs. 3, 5) whose operator uses the FP32 plan, inside
 * iterative refinement against residuals computed with the FP64 plan. The preconditioner is
 * blockdiag(A^, y^T A^{-1} y) with A^ = Theta + Y L L^T Y from a low-rank factor K ~ L L^T
 * (Sec. 4: pivoted Cholesky, Algorithm 2, or Nystrom) applied by the Woodbury identity (Sec. 5).
 *
 * Conventions as in anova.h: status returns, thread-local anova_last_error(), caller-owned
 * buffers, work on the plan's stream.
 */
#ifndef ANOVA_SVM_H
#define ANOVA_SVM_H

#include "anova.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * lowrank_precond_build -- low-rank factor K ~ L L^T (L: n x rank, rank <= r) of the plan's
 * kernel K = sum_l K_l, with the kernel entries evaluated exactly (FP64) from the plan's
 * coordinates.
 *   kind = PCHOL_GREEDY: Algorithm 2 (greedy pivoted Cholesky), pivot = arg-max of the residual
 *          diagonal, ties to the lowest index; stops at rank r or when the largest residual
 *          diagonal is <= err_tol * max(diag K) (Table 1: err_tol = 1e-5).
 *   kind = NYSTROM: K(:,S) K(S,S)^{-1} K(S,:) on the pivot set S of the greedy pass, with the
 *          core K(S,S) factored as L D L^T and entries of D below 1e-10 max D set to that value
 *          (Sec. 4).
 *   kind = PCHOL_RANDOM: randomly pivoted Cholesky (Sec. 4, after Algorithm 2): pivot j is drawn
 *          with probability proportional to the residual diagonal d, as the first index s (in
 *          point order) with cumsum(max(d, 0))[s] > u_j sum(max(d, 0)), where u_j is output j of
 *          SplitMix64 started at `seed` (state seed + (j + 1) 0x9E3779B97F4A7C15 through its
 *          finaliser), top 53 bits scaled to [0, 1). Columns and stop rule as PCHOL_GREEDY.
 *   kind = PCHOL_PER_WINDOW: per-window stacked factors (Sec. 4): K_l ~ L_l L_l^T by Algorithm 2
 *          on window l's kernel alone, at rank r / P (at least 1) each, stop rule relative to
 *          eta_l; L = [L_1 ... L_P] in the plan's internal window order (windows sorted by
 *          decreasing dimension, stable), rank = the sum of the ranks reached; pivots are listed
 *          window after window, each window's from index 0.
 *   kind = NYSTROM_RANDOM: Nystrom with Q = orth(K G) (Sec. 4), G (n x r, column-major) of
 *          standard normals, entry t = j n + i the Box-Muller transform sqrt(-2 ln(1 - u))
 *          cos(2 pi u') of SplitMix64 outputs 2t and 2t + 1 (as above) started at `seed`. K G and
 *          K Q are multi-RHS matvecs of the plan, which must be FP64 (else INVALID_ARG). Q by
 *          Gram-Schmidt with re-orthogonalisation; columns whose norm falls below 1e-10 of their
 *          norm before are dropped, so rank <= r. Core as NYSTROM. err_tol is not used; the
 *          pivots reported by lowrank_info are -1.
 * seed is used by PCHOL_RANDOM and NYSTROM_RANDOM only.
 * The plan must outlive the preconditioner. Requires eta_l >= 0 (K positive semidefinite).
 * Errors: INVALID_ARG (r outside [1, 1024], bad kind, negative eta), OOM, CUDA.
 */
anova_status lowrank_precond_build(anova_plan_t plan, int kind, int r, double err_tol,
                                   uint64_t seed, lowrank_t *out);

/* Rank reached and (optionally, host, rank entries) the pivots in the order they were chosen. */
anova_status lowrank_info(lowrank_t lr, int *rank, int64_t *pivots);

/* Copy the FP64 factor L (n x rank, column-major) to the device buffer L. Synchronous. */
anova_status lowrank_factor(lowrank_t lr, double *L);

/*
 * lowrank_precond_set_theta -- prepare the Woodbury core for one interior point step:
 * M = I + L^T Theta^{-1} L (from an FP32 copy of L, FP64-accurate; see lowrank_set_core_path),
 * its Cholesky factor, and the Schur value s = y^T A^{-1} y. theta, y: device, n doubles;
 * theta > 0, y in {-1, +1}. Errors: BREAKDOWN if M or s is not positive, TIMEOUT if a bounded
 * tensor-core wait ran out. Synchronises the stream.
 */
anova_status lowrank_precond_set_theta(lowrank_t lr, const double *theta, const double *y);

/*
 * Computing path of the Woodbury core M = I + L^T Theta^{-1} L in lowrank_precond_set_theta.
 *   LOWRANK_CORE_TENSOR: on the tensor cores with FP64 accuracy (rank <= 256). A = Theta^{-1/2} L
 *     is split column by column into nine exact bf16 integer slices of 6 bits (error-free
 *     splitting: Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 59, 2012); slice products are summed
 *     exactly in the FP32 accumulator over 4096-row chunks and the chunk sums exactly in FP64, so M
 *     agrees with an FP64 evaluation to about 1e-15 of its norm; deterministic.
 *   LOWRANK_CORE_SIMT: FP64 tiles on the FP64 pipe (any rank).
 *   LOWRANK_CORE_AUTO (default): the tensor cores when rank <= 256, else the FP64 pipe.
 * lowrank_set_core_path -- selects the path for later set_theta calls. Errors: INVALID_ARG (bad
 *   path, or LOWRANK_CORE_TENSOR with rank > 256).
 * lowrank_core -- copies the core M of the last set_theta (before its factorisation; device,
 *   rank x rank row-major doubles; M may be NULL) and reports the path it took. Synchronous.
 *   Errors: INVALID_ARG (NULL lr, or no set_theta yet).
 */
enum { LOWRANK_CORE_AUTO = 0, LOWRANK_CORE_SIMT = 1, LOWRANK_CORE_TENSOR = 2 };
anova_status lowrank_set_core_path(lowrank_t lr, int path);
anova_status lowrank_core(lowrank_t lr, double *M, int *path_used);

/*
 * lowrank_precond_apply -- x = blockdiag(A^, s)^{-1} g for the saddle system of size n + 1:
 * x[0:n] = A^{-1} g[0:n] by the Woodbury identity (Sec. 5), x[n] = g[n] / s. theta and y must be
 * the arrays given to the last lowrank_precond_set_theta. g, x: device, n + 1 doubles, distinct.
 */
anova_status lowrank_precond_apply(lowrank_t lr, const double *theta, const double *y,
                                   const double *g, double *x);

void lowrank_destroy(lowrank_t lr);

/* Stopping rules of the interior point loop. */
enum {
    SVM_STOP_GAP = 0,  /* relative duality gap and |y^T alpha| below tol (default) */
    SVM_STOP_ALG1 = 1  /* Algorithm 1's test: mu and both relative infeasibilities below tol */
};

/* Krylov method of the Newton solves (Sec. 5). Both run on the FP32 operator with FP64
 * refinement; the FP64 fallback solve is MINRES either way.
 *   SVM_KRYLOV_MINRES: MINRES with the SPD block preconditioner blockdiag(A^, y^T A^{-1} y).
 *   SVM_KRYLOV_GMRES: right-preconditioned GMRES with the paper's P = [[A^, 0], [-y^T, -1]],
 *     krylov_max Arnoldi steps without restart (basis of (krylov_max + 1) (n + 1) doubles). */
enum {
    SVM_KRYLOV_MINRES = 0,
    SVM_KRYLOV_GMRES = 1
};

/* Barrier schedules (Sec. 2: mu is reduced by a constant sigma or by a sigma_it per iteration). */
enum {
    SVM_SIGMA_CONSTANT = 0,  /* mu <- sigma mu */
    SVM_SIGMA_ADAPTIVE = 1   /* mu <- (1 - (1 - sigma) s_prev) mu, s_prev = last step (default) */
};

typedef struct {
    int max_iter;            /* interior point iterations (Table 1: 50) */
    double sigma_barrier;    /* barrier reduction mu <- sigma mu (Table 1: 0.6) */
    double gamma;            /* step factor to the boundary (Table 1: 0.99995) */
    int sigma_rule;          /* SVM_SIGMA_ADAPTIVE (default) or SVM_SIGMA_CONSTANT */
    double alpha0;           /* initial alpha_i; <= 0 selects min(C/2, 1/2) */
    int stop;                /* SVM_STOP_GAP or SVM_STOP_ALG1 */
    int krylov_max;          /* MINRES iterations per solve (Table 1: 100) */
    double krylov_tol;       /* relative residual of each Newton solve (default 1e-8) */
    int refine_max;          /* FP64 refinement passes per Newton solve (default 4); when the
                                FP32-operator passes stop reducing the FP64 residual, the solve
                                finishes with MINRES on the FP64 operator */
    int precond;             /* PCHOL_GREEDY, NYSTROM, PCHOL_RANDOM, PCHOL_PER_WINDOW, NYSTROM_RANDOM */
    int rank;                /* preconditioner rank (default 200, at most n) */
    double err_tol;          /* pivoted-Cholesky tolerance (Table 1: 1e-5) */
    uint64_t seed;
    double ell;              /* kernel length scale (default 1) */
    const int32_t *windows;  /* P x 3 windows (-1 padded); NULL: consecutive 3-feature windows */
    int P;
    int N, m;                /* FP32 plan (default 32, 4) */
    int N_precise, m_precise;/* FP64 plan for the objectives, K (y .* alpha) and the
                                preconditioner (default 64, 6) */
    int scale_features;      /* 1: min-max scale every feature into [-0.2, 0.2] first */
    void *cuda_stream;
    int krylov;              /* SVM_KRYLOV_MINRES (default) or SVM_KRYLOV_GMRES */
    int autotune;            /* 1: every plan by anova_nfft_plan_tuned (nrhs 1, 3 reps); default 0 */
    int m_refine;            /* window cut-off of a second FP64 plan (bandwidth N_precise) that
                                gives the refinement residuals of the Newton solves and the
                                FP64-operator MINRES (default 4; 0 or m_precise: the FP64 plan
                                above serves both). Its error (~1e-8 relative at m = 4) is far below
                                the Newton solves' residual tolerance; the objectives and the
                                stopping test keep the FP64 plan above, and K (y .* alpha) is
                                recomputed with it every 8 steps and before convergence is
                                accepted */
} svm_opts;

typedef struct {
    int iterations;          /* interior point iterations done */
    int krylov_iterations;   /* MINRES iterations over all Newton solves */
    int refinements;         /* refinement passes over all Newton solves */
    int fp64_krylov_iterations; /* MINRES iterations run on the FP64 operator (fallback) */
    int rank;                /* preconditioner rank */
    int converged;           /* 1 if the stopping rule was met */
    double mu;               /* final barrier parameter */
    double dual;             /* e^T alpha - 1/2 alpha^T Y K Y alpha (FP64 plan) */
    double primal;           /* 1/2 alpha^T Y K Y alpha + C sum hinge(1 - y_i (f_i + b)) */
    double rel_gap;          /* (primal - dual) / max(1, |primal|) */
    double xi_alpha;         /* |y^T alpha| / max(1, |y^T alpha^0|) */
    double time_ms;          /* wall time of the solve */
} svm_stats;

/* Table 1 defaults and the readings documented with the library. */
void svm_opts_default(svm_opts *opts);

/*
 * svm_ipm_solve -- train the soft-margin kernel SVM by Algorithm 1.
 * X: host, n x d row-major FP64 points (in [-0.2, 0.2] unless opts->scale_features);
 * y: host, n labels in {-1, +1}; C > 0; tol > 0 (stopping tolerance of opts->stop).
 * alpha: host, n doubles (output); b: host, the bias b = -lambda (output); stats nullable.
 * Returns NOT_CONVERGED (with the last iterate in alpha, b) if max_iter is reached first.
 */
anova_status svm_ipm_solve(const double *X, int64_t n, int d, const double *y, double C,
                           double tol, const svm_opts *opts, double *alpha, double *b,
                           svm_stats *stats);

/* One problem of a batch (inputs as svm_ipm_solve; outputs filled by svm_ipm_solve_batch). */
typedef struct {
    const double *X;         /* host, n x d row-major */
    int64_t n;
    int d;
    const double *y;         /* host, n labels in {-1, +1} */
    double C;
    double ell;              /* kernel length scale; <= 0 takes opts->ell */
    const int32_t *windows;  /* P x 3 (-1 padded); NULL takes opts->windows / consecutive windows */
    int P;
    double *alpha;           /* host, n doubles (output) */
    double b;                /* output: bias b = -lambda */
    svm_stats stats;         /* output */
    anova_status status;     /* output: status of this problem's solve */
} svm_problem;

/*
 * svm_ipm_solve_batch -- solve `count` independent problems, `concurrency` at a time: each of
 * `concurrency` host workers owns a CUDA stream of the current device and solves its share of
 * the problems one after another on it, so the small kernels and host round trips of several
 * solves overlap on the GPU. Every problem is solved exactly as svm_ipm_solve would solve it
 * alone with the same opts (opts->cuda_stream is replaced by the worker's stream), so each result
 * is bitwise the same alone and in the batch. Returns ANOVA_OK if every problem succeeded,
 * otherwise the first failing problem's status (each problem carries its own status).
 */
anova_status svm_ipm_solve_batch(svm_problem *problems, int count, double tol,
                                 const svm_opts *opts, int concurrency);

/*
 * Serving: a request loop over svm_ipm_solve. The paper has no serving layer; this follows the
 * traffic its Sec. 6 parameter search generates (many solves of different sizes and (C, ell)).
 *
 * svm_server_create starts `slots` workers on the current device, each with its own CUDA stream.
 * Requests (svm_problem, whose input and output buffers must stay valid until the request
 * completes) are queued by svm_server_submit and started in arrival order as soon as a worker is
 * free AND the device-memory estimate of the request fits in `hbm_budget_bytes` together with the
 * requests already running (a request larger than the whole budget runs alone). While the oldest
 * queued request does not fit, the oldest younger request that fits starts instead (backfill); the
 * same oldest request is passed at most 4 times, after which nothing younger starts until it has
 * started (a bound on its wait for memory). While a solve
 * runs, its plans, grids, preconditioner and iterates stay on the device; solves on different
 * workers overlap on the GPU. Each result is bitwise the one svm_ipm_solve gives alone with the
 * same opts. Latency of a request = completion time - submission time.
 */
typedef struct svm_server *svm_server_t;

typedef struct {
    int64_t submitted, completed, running, queued;
    int64_t reserved_bytes;       /* device-memory estimate of the running requests */
    int64_t peak_reserved_bytes;  /* the largest reserved_bytes seen */
    double p50_latency_ms, p99_latency_ms, mean_latency_ms;  /* over completed requests */
    int64_t backfilled;           /* requests started ahead of an older one that did not fit */
} svm_server_stats;

anova_status svm_server_create(const svm_opts *opts, double tol, int slots, int64_t hbm_budget_bytes,
                               svm_server_t *out);
/* Queue one request; returns at once. *ticket identifies it for svm_server_wait. */
anova_status svm_server_submit(svm_server_t server, svm_problem *problem, int64_t *ticket);
/* Block until the request completes; returns its status (also stored in problem->status). */
anova_status svm_server_wait(svm_server_t server, int64_t ticket);
/* Block until every submitted request has completed. */
anova_status svm_server_drain(svm_server_t server);
anova_status svm_server_get_stats(svm_server_t server, svm_server_stats *stats);
/* Device-memory estimate (bytes) the server reserves for a request of n points and P windows
 * solved with `opts` (NULL: defaults): both plans, the low-rank factor and the solver vectors.
 * Returns 0 for n < 1 or P < 1. */
int64_t svm_request_footprint(int64_t n, int P, const svm_opts *opts);
/* The workers' admission rule as a pure host function (no device work), for tests and for
 * replaying a schedule. footprints[k] (bytes) and passed[k] (how many younger requests started
 * ahead of it) describe the queued requests in arrival order; reserved_bytes is the estimate of
 * the running requests and running their number. Stores in *pick the index of the request to
 * start next, or -1 for none: the oldest when reserved_bytes + its footprint <= budget_bytes or
 * running == 0; otherwise, if the oldest has been passed fewer than 4 times, the oldest younger
 * request that fits; otherwise none. ANOVA_ERR_INVALID_ARG (and *pick = -1 where pick is not
 * NULL) for a NULL pick, count < 0, or NULL arrays with count > 0. */
anova_status svm_server_admission(const int64_t *footprints, const int32_t *passed, int count,
                                  int64_t reserved_bytes, int64_t budget_bytes, int running, int *pick);
/* Drains, stops the workers and frees the server. */
void svm_server_destroy(svm_server_t server);

/* sizeof of this ABI's structs by name: "anova_tune_report", "svm_opts", "svm_stats",
 * "svm_problem", "svm_server_stats". A binding that mirrors their layouts can check its copies
 * against these. Returns 0 for NULL or an unknown name. Host only. */
int64_t anova_abi_struct_size(const char *name);

#ifdef __cplusplus
}
#endif

#endif /* ANOVA_SVM_H */
