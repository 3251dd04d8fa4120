// Interior point method for the kernel SVM dual (arXiv 2312.00538, Sec. 2, Algorithm 1) with
// Newton systems (eq. (Newton)) solved by preconditioned MINRES (Secs. 3, 5) on the FP32
// ANOVA-NFFT operator, refined against FP64-plan residuals. Vectors live on the device in FP64.
// The Krylov recurrences run on the device too: one-thread kernels keep the scalars (Lanczos
// beta, the Givens rotations, the residual estimate; for GMRES the Hessenberg column) in device
// memory, dot products are per-block partial sums added in a fixed order (reproducible), and an
// FP32 Krylov solve is one CUDA graph whose conditional while node runs the iterations until the
// device-side convergence test clears its condition. The host only drives the Newton steps and
// the FP64 refinement around each solve. Also exports the low-rank preconditioner calls of
// anova_svm.h.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <thread>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "../../include/anova_svm.h"
#include "anova_internal.h"
#include "lowrank_internal.h"

namespace anova {
anova_status create_plan(const double *points, int64_t n, int d, const int32_t *windows, int P,
                         const double *ell, const double *eta, int N, int m, int flags,
                         void *stream, anova_plan_t *out);
void destroy_plan(anova_plan *p);
anova_status tune_plan(const double *points, int64_t n, int d, const int32_t *windows, int P, const double *ell,
                       const double *eta, int N, int m, int flags, void *stream, int nrhs, int reps,
                       anova_tune_report *report, anova_plan_t *out);

namespace {

constexpr int kRedBlocks = 256;

__global__ void k_dot(const double *__restrict__ a, const double *__restrict__ b, long long n,
                      double *__restrict__ part) {
    __shared__ double ws[32];
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s += a[i] * b[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) part[blockIdx.x] = s;
    }
}

// out = scale * sum(part[0..np)) written on the device (no host round trip)
__global__ void k_sum_to(const double *__restrict__ part, int np, double scale, double *__restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < np; ++i) s += part[i];
        *out = scale * s;
    }
}

__global__ void k_yx_f32(const double *__restrict__ x, const double *__restrict__ y, long long n, float *__restrict__ t) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        t[i] = (float)(y[i] * x[i]);
}

__global__ void k_yx_f64(const double *__restrict__ x, const double *__restrict__ y, long long n, double *__restrict__ t) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        t[i] = y[i] * x[i];
}

// out[i] = y_i (K t)_i + theta_i x_i - y_i x_n   (the (1,1) and (1,2) blocks of eq. (Newton))
template <typename K>
__global__ void k_saddle_post(const K *__restrict__ Kt, const double *__restrict__ x, const double *__restrict__ y,
                              const double *__restrict__ theta, long long n, double *__restrict__ out) {
    const double xn = x[n];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = y[i] * (double)Kt[i] + theta[i] * x[i] - y[i] * xn;
}

__global__ void k_axpy(double a, const double *__restrict__ x, long long n, double *__restrict__ y) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] += a * x[i];
}

__global__ void k_sub(const double *__restrict__ a, const double *__restrict__ b, long long n, double *__restrict__ out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = a[i] - b[i];
}

__global__ void k_fill_d(double *x, long long n, double v) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] = v;
}

// Theta = mu (1/alpha^2 + 1/(C - alpha)^2) (Sec. 2)
__global__ void k_theta(const double *__restrict__ al, double mu, double C, long long n, double *__restrict__ th) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double a = al[i], c = C - a;
        th[i] = mu * (1.0 / (a * a) + 1.0 / (c * c));
    }
}

// rhs_i = 1 - y_i f_i + lambda y_i + mu/alpha_i - mu/(C - alpha_i), f = K (y .* alpha) (eq. (Newton))
__global__ void k_newton_rhs(const double *__restrict__ al, const double *__restrict__ y, const double *__restrict__ f,
                             double lam, double mu, double C, long long n, double *__restrict__ rhs) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double a = al[i];
        rhs[i] = 1.0 - y[i] * f[i] + lam * y[i] + mu / a - mu / (C - a);
    }
}

// per-block minimum of the step that keeps 0 <= alpha + s d <= C
__global__ void k_step_partial(const double *__restrict__ al, const double *__restrict__ d, double C, long long n,
                               double *__restrict__ part) {
    __shared__ double ws[32];
    double s = INFINITY;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double di = d[i];
        if (di < 0.0) s = fmin(s, -al[i] / di);
        else if (di > 0.0) s = fmin(s, (C - al[i]) / di);
    }
    for (int o = 16; o > 0; o >>= 1) s = fmin(s, __shfl_down_sync(0xffffffffu, s, o));
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : INFINITY;
        for (int o = 16; o > 0; o >>= 1) s = fmin(s, __shfl_down_sync(0xffffffffu, s, o));
        if (threadIdx.x == 0) part[blockIdx.x] = s;
    }
}

// sums for the objectives: [0] sum alpha, [1] (y.*alpha)^T f, [2] sum hinge(1 - y (f + b)),
// [3] y^T alpha, [4] ||xi_lambda||^2 with the current mu
__global__ void k_objective_partial(const double *__restrict__ al, const double *__restrict__ y,
                                    const double *__restrict__ f, double b, double lam, double mu, double C,
                                    long long n, double *__restrict__ part) {
    __shared__ double ws[5][32];
    double s[5] = {0, 0, 0, 0, 0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double a = al[i], yi = y[i], fi = f[i];
        s[0] += a;
        s[1] += yi * a * fi;
        s[2] += fmax(0.0, 1.0 - yi * (fi + b));
        s[3] += yi * a;
        const double xl = 1.0 - yi * fi + lam * yi + mu / a - mu / (C - a);
        s[4] += xl * xl;
    }
    for (int k = 0; k < 5; ++k) {
        double v = s[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) ws[k][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        for (int k = 0; k < 5; ++k) {
            double v = threadIdx.x < (blockDim.x >> 5) ? ws[k][threadIdx.x] : 0.0;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (threadIdx.x == 0) part[k * gridDim.x + blockIdx.x] = v;
        }
    }
}

int blocks_for(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, kRedBlocks)); }

// ------------------------------------------------------------------ device-resident MINRES
// The scalar recurrence of MINRES (Paige-Saunders) runs in one-thread kernels on the solver's
// stream and the vector kernels read their coefficients from device memory, so an iteration needs
// no host round trip; the host only watches a copy of the `active` flag, a few iterations behind.
struct MinresState {
    double beta1, beta, beta_prev, phibar;
    double c_prev2, s_prev2, c_prev, s_prev;
    double alpha, beta_next_sq;  // written by the dot products of the iteration
    double inv_beta, eps, delta, inv_gamma, phi, rtol;
    int active, do_w, iters, status;  // status: 1 indefinite preconditioner, 2 singular tridiagonal
    int maxit;
};

// beta1^2 (the first preconditioned norm) is in beta_next_sq
__global__ void k_mr_init(MinresState *s, double rtol, int maxit) {
    const double b2 = s->beta_next_sq;
    s->rtol = rtol;
    s->maxit = maxit;
    s->iters = 0;
    s->do_w = 0;
    s->status = 0;
    s->active = 0;
    if (b2 < 0.0) {
        s->status = 1;
        return;
    }
    const double b1 = sqrt(b2);
    s->beta1 = b1;
    s->beta = b1;
    s->beta_prev = 0.0;
    s->phibar = b1;
    s->c_prev2 = 1.0;
    s->s_prev2 = 0.0;
    s->c_prev = 1.0;
    s->s_prev = 0.0;
    s->inv_beta = b1 > 0.0 ? 1.0 / b1 : 0.0;
    s->active = b1 > 0.0 ? 1 : 0;
}

// v = y / beta
__global__ void k_mr_scale(const double *__restrict__ y, const MinresState *__restrict__ s, long long n,
                           double *__restrict__ v) {
    if (!s->active) return;
    const double f = s->inv_beta;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        v[i] = f * y[i];
}

// r_next = A v - (alpha / beta) r_cur - (beta / beta_prev) r_prev
__global__ void k_mr_lin3(const double *__restrict__ Av, const double *__restrict__ rc, const double *__restrict__ rp,
                          const MinresState *__restrict__ s, long long n, double *__restrict__ rn) {
    if (!s->active) return;
    const double sb = -s->alpha / s->beta, sc = s->beta_prev > 0.0 ? -s->beta / s->beta_prev : 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        rn[i] = Av[i] + sb * rc[i] + sc * rp[i];
}

__device__ void mr_step(MinresState *s) {
    const double bns = s->beta_next_sq;
    if (bns < 0.0) {
        s->status = 1;
        s->active = 0;
        return;
    }
    const double beta_next = sqrt(bns), beta = s->beta, alpha = s->alpha;
    const double eps = s->s_prev2 * beta;
    const double dbar = s->c_prev2 * beta;
    const double delta = s->c_prev * dbar + s->s_prev * alpha;
    const double gbar = -s->s_prev * dbar + s->c_prev * alpha;
    const double gamma = hypot(gbar, beta_next);
    if (gamma == 0.0) {
        s->status = 2;
        s->active = 0;
        return;
    }
    const double c = gbar / gamma, sn = beta_next / gamma;
    s->phi = c * s->phibar;
    s->phibar = -sn * s->phibar;
    s->eps = eps;
    s->delta = delta;
    s->inv_gamma = 1.0 / gamma;
    s->do_w = 1;
    s->c_prev2 = s->c_prev;
    s->s_prev2 = s->s_prev;
    s->c_prev = c;
    s->s_prev = sn;
    s->beta_prev = beta;
    s->beta = beta_next;
    s->inv_beta = beta_next > 0.0 ? 1.0 / beta_next : 0.0;
    s->iters += 1;
    if (fabs(s->phibar) <= s->rtol * s->beta1 || beta_next == 0.0 || s->iters >= s->maxit) s->active = 0;
}

// the Givens step of the iteration and the convergence test |phibar| <= rtol beta1; inside a
// graph, `loop` is the handle of the enclosing while node and receives the `active` flag
__global__ void k_mr_step(MinresState *s, cudaGraphConditionalHandle loop) {
    s->do_w = 0;
    if (s->active) mr_step(s);
    if (loop) cudaGraphSetConditional(loop, s->active ? 1u : 0u);
}


// w_new = (v - eps w2 - delta w1) / gamma; x += phi w_new; then w2 <- w1, w1 <- w_new (the two
// newest directions stay in fixed buffers)
__global__ void k_mr_w(const double *__restrict__ v, double *__restrict__ w1, double *__restrict__ w2,
                       const MinresState *__restrict__ s, long long n, double *__restrict__ x) {
    if (!s->do_w) return;
    const double eps = s->eps, delta = s->delta, ig = s->inv_gamma, phi = s->phi;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double a = w1[i];
        const double w = (v[i] - eps * w2[i] - delta * a) * ig;
        w2[i] = a;
        w1[i] = w;
        x[i] += phi * w;
    }
}

// the Lanczos vectors move down one place: r_prev <- r_cur <- r_next, y_cur <- y_next
__global__ void k_mr_rotate(double *__restrict__ r_prev, double *__restrict__ r_cur, const double *__restrict__ r_next,
                            double *__restrict__ y_cur, const double *__restrict__ y_next,
                            const MinresState *__restrict__ s, long long n) {
    if (!s->do_w) return;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        r_prev[i] = r_cur[i];
        r_cur[i] = r_next[i];
        y_cur[i] = y_next[i];
    }
}

// ------------------------------------------------------------------ device-resident GMRES
// Right-preconditioned GMRES (Saad and Schultz) with the paper's block-triangular P (Sec. 5),
// no restart inside a call. Arnoldi with classical Gram-Schmidt done twice (each pass: all dot
// products in one launch, then one update), Givens rotations in a one-thread kernel; the basis
// column j, the Hessenberg matrix and the rotations live in device memory and the kernels read j
// from there, so the iteration is a fixed launch sequence (captured as a graph while loop).
struct GmresState {
    double beta, rtol, resid, hnext;
    int j, m, active, status;
};
constexpr int kGsBlocks = 64;  // row blocks of the Gram-Schmidt dot products

__global__ void k_gm_init(GmresState *s, const double *__restrict__ bnorm2, double rtol, int m, double *g) {
    const double b = sqrt(fmax(*bnorm2, 0.0));
    s->beta = b;
    s->rtol = rtol;
    s->resid = b;
    s->m = m;
    s->j = 0;
    s->status = 0;
    s->active = b > 0.0 ? 1 : 0;
    g[0] = b;
}

// V(:, 0) = b / beta
__global__ void k_gm_first(const double *__restrict__ b, const GmresState *__restrict__ s, long long n,
                           double *__restrict__ V0) {
    if (!s->active) return;
    const double f = 1.0 / s->beta;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        V0[i] = f * b[i];
}

// vj = V(:, j)
__global__ void k_gm_col(const double *__restrict__ V, const GmresState *__restrict__ s, long long n,
                         double *__restrict__ vj) {
    if (!s->active) return;
    const double *c = V + (size_t)s->j * n;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        vj[i] = c[i];
}

// the last entry of P^{-1} g: x_n = -(g_n + y^T x[0:n]) with y^T x[0:n] in `part`
__global__ void k_tri_last(const double *__restrict__ part, int np, const double *__restrict__ g, long long n,
                           double *__restrict__ x) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < np; ++i) t += part[i];
        x[n] = -(g[n] + t);
    }
}

// partial dot products of the columns i <= j of V with w: block (x, i) sums its row range
__global__ void __launch_bounds__(256) k_gm_dots(const double *__restrict__ V, const double *__restrict__ w,
                                                 long long n, const GmresState *__restrict__ s,
                                                 double *__restrict__ gpart) {
    __shared__ double ws[8];
    const int i = blockIdx.y;
    if (!s->active || i > s->j) return;
    const long long chunk = (n + gridDim.x - 1) / gridDim.x;
    const long long lo = (long long)blockIdx.x * chunk, hi = min(n, lo + chunk);
    const double *c = V + (size_t)i * n;
    double t = 0.0;
    for (long long r = lo + threadIdx.x; r < hi; r += blockDim.x) t += c[r] * w[r];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double u = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) u += ws[k];
        gpart[(size_t)i * gridDim.x + blockIdx.x] = u;
    }
}

// h_i = sum of the partials (fixed order); H(i, j) (+)= h_i; hbuf = h
__global__ void k_gm_hsum(const double *__restrict__ gpart, int nparts, const GmresState *__restrict__ s,
                          double *__restrict__ H, double *__restrict__ hbuf, int accumulate) {
    if (!s->active) return;
    const int j = s->j, ld = s->m + 1;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        double h = 0.0;
        for (int k = 0; k < nparts; ++k) h += gpart[(size_t)i * nparts + k];
        hbuf[i] = h;
        H[i + (size_t)j * ld] = accumulate ? H[i + (size_t)j * ld] + h : h;
    }
}

// w -= V(:, 0..j) h
__global__ void k_gm_sub(const double *__restrict__ V, const double *__restrict__ hbuf,
                         const GmresState *__restrict__ s, long long n, double *__restrict__ w) {
    if (!s->active) return;
    const int j = s->j;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        double t = w[r];
        for (int i = 0; i <= j; ++i) t -= hbuf[i] * V[(size_t)i * n + r];
        w[r] = t;
    }
}

// H(j + 1, j) = ||w|| (squared norm in `part`)
__global__ void k_gm_norm(const double *__restrict__ part, int np, GmresState *s, double *__restrict__ H) {
    if (threadIdx.x != 0 || blockIdx.x != 0 || !s->active) return;
    double t = 0.0;
    for (int i = 0; i < np; ++i) t += part[i];
    const double h = sqrt(fmax(t, 0.0));
    s->hnext = h;
    H[(s->j + 1) + (size_t)s->j * (s->m + 1)] = h;
}

// V(:, j + 1) = w / H(j + 1, j) (zero after a lucky breakdown)
__global__ void k_gm_next(const double *__restrict__ w, const GmresState *__restrict__ s, long long n,
                          double *__restrict__ V) {
    if (!s->active) return;
    const double h = s->hnext, f = h > 0.0 ? 1.0 / h : 0.0;
    double *c = V + (size_t)(s->j + 1) * n;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
        c[r] = f * w[r];
}

// Givens rotations on column j, the residual norm |g_{j+1}|, the stop test
__global__ void k_gm_step(GmresState *s, double *H, double *cs, double *sn, double *g,
                          cudaGraphConditionalHandle loop) {
    if (s->active) {
        const int j = s->j, ld = s->m + 1;
        double *h = H + (size_t)j * ld;
        for (int i = 0; i < j; ++i) {
            const double t = cs[i] * h[i] + sn[i] * h[i + 1];
            h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
            h[i] = t;
        }
        const double rho = hypot(h[j], h[j + 1]);
        if (rho == 0.0) {
            s->status = 2;
            s->active = 0;
        } else {
            cs[j] = h[j] / rho;
            sn[j] = h[j + 1] / rho;
            h[j] = rho;
            h[j + 1] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            s->j = j + 1;
            s->resid = fabs(g[j + 1]);
            if (s->resid <= s->rtol * s->beta || s->j >= s->m) s->active = 0;
        }
    }
    if (loop) cudaGraphSetConditional(loop, s->active ? 1u : 0u);
}

// y = H(:j, :j)^{-1} g(:j) by back substitution
__global__ void k_gm_solve(const GmresState *__restrict__ s, const double *__restrict__ H,
                           const double *__restrict__ g, double *__restrict__ yv) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int j = s->j, ld = s->m + 1;
    for (int i = j - 1; i >= 0; --i) {
        double t = g[i];
        for (int k = i + 1; k < j; ++k) t -= H[i + (size_t)k * ld] * yv[k];
        yv[i] = t / H[i + (size_t)i * ld];
    }
}

// u = V(:, :j) y
__global__ void k_gm_combine(const double *__restrict__ V, const double *__restrict__ yv,
                             const GmresState *__restrict__ s, long long n, double *__restrict__ u) {
    const int j = s->j;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        double t = 0.0;
        for (int i = 0; i < j; ++i) t += yv[i] * V[(size_t)i * n + r];
        u[r] = t;
    }
}

// ------------------------------------------------------------------ solver state
struct Solver {
    anova_plan *p32 = nullptr, *p64 = nullptr;
    anova_plan *p64r = nullptr;  // FP64 plan of the refinement residuals (may be p64)
    lowrank *lr = nullptr;
    cudaStream_t st = nullptr;
    long long n = 0;
    const double *y = nullptr, *theta = nullptr;  // device
    double *part = nullptr;                      // kRedBlocks * 5 partials
    std::vector<double> hpart;
    float *t32 = nullptr, *k32 = nullptr;
    double *t64 = nullptr, *k64 = nullptr;
    int krylov_total = 0, refine_total = 0, fp64_krylov_total = 0;
    // device-resident MINRES: scalar state, host copy of its flags, and the FP32 iteration
    // captured as the body of a conditional while node (built on the first FP32 solve)
    MinresState *ms = nullptr;
    int *hflags = nullptr;            // pinned {active, do_w, iters, status}
    cudaEvent_t ev = nullptr;
    cudaStream_t cap = nullptr;       // private stream the iteration is captured on
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const double *graph_b = nullptr;  // buffers the graph was captured with
    double *graph_x = nullptr;
    // GMRES (svm_opts.krylov = SVM_KRYLOV_GMRES): basis, Hessenberg data and its graph
    int gm_m = 0;
    GmresState *gs = nullptr;
    double *V = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *yv = nullptr, *hbuf = nullptr,
           *gpart = nullptr, *bnorm2 = nullptr;
    double *vj = nullptr, *z = nullptr, *w = nullptr, *u = nullptr;
    cudaGraph_t gm_graph = nullptr;
    cudaGraphExec_t gm_exec = nullptr;

    anova_status dot(const double *a, const double *b, long long len, double *out) {
        const int nb = blocks_for(len);
        k_dot<<<nb, 256, 0, st>>>(a, b, len, part);
        ANOVA_CUDA_TRY(cudaGetLastError());
        hpart.resize(nb);
        ANOVA_CUDA_TRY(cudaMemcpyAsync(hpart.data(), part, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
        ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
        double s = 0.0;
        for (int i = 0; i < nb; ++i) s += hpart[i];
        *out = s;
        return ANOVA_OK;
    }

    // out = A x for the saddle matrix of eq. (Newton); precise selects the FP64 refinement plan
    anova_status apply(const double *x, double *out, bool precise) {
        const int nb = blocks_for(n);
        anova_status s;
        if (precise) {
            k_yx_f64<<<nb, 256, 0, st>>>(x, y, n, t64);
            if ((s = run_matvec_t<double>(p64r, t64, k64, 1, -1)) != ANOVA_OK) return s;
            k_saddle_post<double><<<nb, 256, 0, st>>>(k64, x, y, theta, n, out);
        } else {
            k_yx_f32<<<nb, 256, 0, st>>>(x, y, n, t32);
            if ((s = run_matvec_t<float>(p32, t32, k32, 1, -1)) != ANOVA_OK) return s;
            k_saddle_post<float><<<nb, 256, 0, st>>>(k32, x, y, theta, n, out);
        }
        // out[n] = -y^T x[0:n]
        k_dot<<<nb, 256, 0, st>>>(y, x, n, part);
        k_sum_to<<<1, 32, 0, st>>>(part, nb, -1.0, out + n);
        ANOVA_CUDA_TRY(cudaGetLastError());
        return ANOVA_OK;
    }

    // K (y .* a) with the FP64 plan into f
    anova_status kya(const double *a, double *f) {
        const int nb = blocks_for(n);
        k_yx_f64<<<nb, 256, 0, st>>>(a, y, n, t64);
        ANOVA_CUDA_TRY(cudaGetLastError());
        return run_matvec_t<double>(p64, t64, f, 1, -1);
    }
};

// One MINRES iteration on fixed buffers (work[0..8]) and stream st; `loop` is the handle of the
// enclosing graph while node (0 outside a graph).
anova_status minres_iteration(Solver &S, double *x, double *work[10], bool precise, cudaStream_t st,
                              cudaGraphConditionalHandle loop) {
    const long long N1 = S.n + 1;
    const int nb = blocks_for(N1);
    double *r_prev = work[0], *r_cur = work[1], *r_next = work[2], *y_cur = work[3], *y_next = work[4];
    double *v = work[5], *Av = work[6], *w1 = work[7], *w2 = work[8];
    anova_status s;
    k_mr_scale<<<nb, 256, 0, st>>>(y_cur, S.ms, N1, v);
    if ((s = S.apply(v, Av, precise)) != ANOVA_OK) return s;
    k_dot<<<nb, 256, 0, st>>>(v, Av, N1, S.part);
    k_sum_to<<<1, 32, 0, st>>>(S.part, nb, 1.0, &S.ms->alpha);
    k_mr_lin3<<<nb, 256, 0, st>>>(Av, r_cur, r_prev, S.ms, N1, r_next);
    if ((s = lowrank_apply_impl(S.lr, S.theta, S.y, r_next, y_next)) != ANOVA_OK) return s;
    k_dot<<<nb, 256, 0, st>>>(r_next, y_next, N1, S.part);
    k_sum_to<<<1, 32, 0, st>>>(S.part, nb, 1.0, &S.ms->beta_next_sq);
    k_mr_step<<<1, 1, 0, st>>>(S.ms, loop);
    k_mr_w<<<nb, 256, 0, st>>>(v, w1, w2, S.ms, N1, x);
    k_mr_rotate<<<nb, 256, 0, st>>>(r_prev, r_cur, r_next, y_cur, y_next, S.ms, N1);
    ANOVA_CUDA_TRY(cudaGetLastError());
    return ANOVA_OK;
}

// Capture the FP32 iteration as the body of a while node whose condition k_mr_step sets. The
// plans and the solver launch on their `stream` fields, which point at the capture stream while
// the body is recorded.
anova_status build_minres_graph(Solver &S, const double *b, double *x, double *work[10]) {
    if (S.exec) {
        cudaGraphExecDestroy(S.exec);
        S.exec = nullptr;
    }
    if (S.graph) {
        cudaGraphDestroy(S.graph);
        S.graph = nullptr;
    }
    if (!S.cap) ANOVA_CUDA_TRY(cudaStreamCreateWithFlags(&S.cap, cudaStreamNonBlocking));
    ANOVA_CUDA_TRY(cudaGraphCreate(&S.graph, 0));
    cudaGraphConditionalHandle loop = 0;
    ANOVA_CUDA_TRY(cudaGraphConditionalHandleCreate(&loop, S.graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = loop;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    ANOVA_CUDA_TRY(cudaGraphAddNode(&node, S.graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStream_t saved[3] = {S.st, S.p32->stream, S.lr->plan->stream};
    S.st = S.p32->stream = S.lr->plan->stream = S.cap;
    cudaError_t e = cudaStreamBeginCaptureToGraph(S.cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    anova_status s = ANOVA_OK;
    if (e == cudaSuccess) {
        s = minres_iteration(S, x, work, false, S.cap, loop);
        cudaGraph_t captured = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(S.cap, &captured);
        if (e2 != cudaSuccess && s == ANOVA_OK) s = cuda_fail(e2, "cudaStreamEndCapture");
    } else {
        s = cuda_fail(e, "cudaStreamBeginCaptureToGraph");
    }
    S.st = saved[0];
    S.p32->stream = saved[1];
    S.lr->plan->stream = saved[2];
    if (s != ANOVA_OK) return s;
    ANOVA_CUDA_TRY(cudaGraphInstantiate(&S.exec, S.graph, 0));
    S.graph_b = b;
    S.graph_x = x;
    return ANOVA_OK;
}

// Preconditioned MINRES (Paige-Saunders) for A x = b, x0 = 0, vectors of length n + 1, run on
// the device (see MinresState). FP32 solves launch one graph whose while node repeats the
// iteration until the device-side test stops it; FP64 solves (few iterations) run the same
// iteration from the host, reading the device flags after each one.
anova_status minres(Solver &S, const double *b, double *x, double rtol, int maxit, double *work[10], int *iters,
                    bool precise = false) {
    const long long N1 = S.n + 1;
    const int nb = blocks_for(N1);
    double *r_prev = work[0], *r_cur = work[1], *y_cur = work[3], *w1 = work[7], *w2 = work[8];
    cudaStream_t st = S.st;
    anova_status s;
    if (!precise && (!S.exec || S.graph_b != b || S.graph_x != x)) {
        // the body's first run inside a graph must not allocate: warm the FP32 operator first
        if ((s = S.apply(work[5], work[6], false)) != ANOVA_OK) return s;
        if ((s = build_minres_graph(S, b, x, work)) != ANOVA_OK) return s;
    }
    ANOVA_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * N1, st));
    ANOVA_CUDA_TRY(cudaMemsetAsync(r_prev, 0, sizeof(double) * N1, st));
    ANOVA_CUDA_TRY(cudaMemsetAsync(w1, 0, sizeof(double) * N1, st));
    ANOVA_CUDA_TRY(cudaMemsetAsync(w2, 0, sizeof(double) * N1, st));
    ANOVA_CUDA_TRY(cudaMemcpyAsync(r_cur, b, sizeof(double) * N1, cudaMemcpyDeviceToDevice, st));
    if ((s = lowrank_apply_impl(S.lr, S.theta, S.y, r_cur, y_cur)) != ANOVA_OK) return s;
    k_dot<<<nb, 256, 0, st>>>(r_cur, y_cur, N1, S.part);
    k_sum_to<<<1, 32, 0, st>>>(S.part, nb, 1.0, &S.ms->beta_next_sq);
    k_mr_init<<<1, 1, 0, st>>>(S.ms, rtol, maxit);
    ANOVA_CUDA_TRY(cudaGetLastError());
    if (!precise) {
        ANOVA_CUDA_TRY(cudaGraphLaunch(S.exec, st));
    } else {
        for (int it = 1; it <= maxit; ++it) {
            if ((s = minres_iteration(S, x, work, true, st, 0)) != ANOVA_OK) return s;
            ANOVA_CUDA_TRY(cudaMemcpyAsync(S.hflags, &S.ms->active, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
            ANOVA_CUDA_TRY(cudaEventRecord(S.ev, st));
            ANOVA_CUDA_TRY(cudaEventSynchronize(S.ev));
            if (!S.hflags[0]) break;
        }
    }
    int fin[4];
    ANOVA_CUDA_TRY(cudaMemcpyAsync(fin, &S.ms->active, sizeof(fin), cudaMemcpyDeviceToHost, st));
    ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
    *iters = fin[2];
    if (precise) S.fp64_krylov_total += *iters;
    else S.krylov_total += *iters;
    if (fin[3] == 1) return fail(ANOVA_ERR_BREAKDOWN, "MINRES: preconditioner is not positive definite");
    if (fin[3] == 2) return fail(ANOVA_ERR_BREAKDOWN, "MINRES: singular tridiagonal");
    return ANOVA_OK;
}

// x = P^{-1} g for the paper's P = [[A^, 0], [-y^T, -1]] (Sec. 5)
anova_status tri_apply(Solver &S, const double *g, double *x) {
    anova_status s;
    if ((s = woodbury_apply(S.lr, S.theta, S.y, g, x, false)) != ANOVA_OK) return s;
    const int nb = blocks_for(S.n);
    k_dot<<<nb, 256, 0, S.st>>>(S.y, x, S.n, S.part);
    k_tri_last<<<1, 32, 0, S.st>>>(S.part, nb, g, S.n, x);
    ANOVA_CUDA_TRY(cudaGetLastError());
    return ANOVA_OK;
}

// One GMRES iteration (column j of the Arnoldi process) on stream S.st.
anova_status gmres_iteration(Solver &S, cudaGraphConditionalHandle loop) {
    const long long N1 = S.n + 1;
    const int nb = blocks_for(N1);
    cudaStream_t st = S.st;
    anova_status s;
    k_gm_col<<<nb, 256, 0, st>>>(S.V, S.gs, N1, S.vj);
    if ((s = tri_apply(S, S.vj, S.z)) != ANOVA_OK) return s;
    if ((s = S.apply(S.z, S.w, false)) != ANOVA_OK) return s;
    for (int pass = 0; pass < 2; ++pass) {
        k_gm_dots<<<dim3(kGsBlocks, S.gm_m + 1), 256, 0, st>>>(S.V, S.w, N1, S.gs, S.gpart);
        k_gm_hsum<<<1, 128, 0, st>>>(S.gpart, kGsBlocks, S.gs, S.H, S.hbuf, pass);
        k_gm_sub<<<nb, 256, 0, st>>>(S.V, S.hbuf, S.gs, N1, S.w);
    }
    k_dot<<<nb, 256, 0, st>>>(S.w, S.w, N1, S.part);
    k_gm_norm<<<1, 32, 0, st>>>(S.part, nb, S.gs, S.H);
    k_gm_next<<<nb, 256, 0, st>>>(S.w, S.gs, N1, S.V);
    k_gm_step<<<1, 1, 0, st>>>(S.gs, S.H, S.cs, S.sn, S.g, loop);
    ANOVA_CUDA_TRY(cudaGetLastError());
    return ANOVA_OK;
}

anova_status build_gmres_graph(Solver &S) {
    if (!S.cap) ANOVA_CUDA_TRY(cudaStreamCreateWithFlags(&S.cap, cudaStreamNonBlocking));
    ANOVA_CUDA_TRY(cudaGraphCreate(&S.gm_graph, 0));
    cudaGraphConditionalHandle loop = 0;
    ANOVA_CUDA_TRY(cudaGraphConditionalHandleCreate(&loop, S.gm_graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = loop;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    ANOVA_CUDA_TRY(cudaGraphAddNode(&node, S.gm_graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStream_t saved[3] = {S.st, S.p32->stream, S.lr->plan->stream};
    S.st = S.p32->stream = S.lr->plan->stream = S.cap;
    cudaError_t e = cudaStreamBeginCaptureToGraph(S.cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    anova_status s = ANOVA_OK;
    if (e == cudaSuccess) {
        s = gmres_iteration(S, loop);
        cudaGraph_t captured = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(S.cap, &captured);
        if (e2 != cudaSuccess && s == ANOVA_OK) s = cuda_fail(e2, "cudaStreamEndCapture");
    } else {
        s = cuda_fail(e, "cudaStreamBeginCaptureToGraph");
    }
    S.st = saved[0];
    S.p32->stream = saved[1];
    S.lr->plan->stream = saved[2];
    if (s != ANOVA_OK) return s;
    ANOVA_CUDA_TRY(cudaGraphInstantiate(&S.gm_exec, S.gm_graph, 0));
    return ANOVA_OK;
}

// Right-preconditioned GMRES for A x = b on the FP32 operator, x0 = 0 (one graph launch for the
// Arnoldi loop, then the small triangular solve and x = P^{-1} V y).
anova_status gmres(Solver &S, const double *b, double *x, double rtol, int *iters) {
    const long long N1 = S.n + 1;
    const int nb = blocks_for(N1);
    cudaStream_t st = S.st;
    anova_status s;
    if (!S.gm_exec) {
        if ((s = S.apply(S.z, S.w, false)) != ANOVA_OK) return s;  // the operator must not allocate in the graph
        if ((s = build_gmres_graph(S)) != ANOVA_OK) return s;
    }
    k_dot<<<nb, 256, 0, st>>>(b, b, N1, S.part);
    k_sum_to<<<1, 32, 0, st>>>(S.part, nb, 1.0, S.bnorm2);
    k_gm_init<<<1, 1, 0, st>>>(S.gs, S.bnorm2, rtol, S.gm_m, S.g);
    k_gm_first<<<nb, 256, 0, st>>>(b, S.gs, N1, S.V);
    ANOVA_CUDA_TRY(cudaGetLastError());
    ANOVA_CUDA_TRY(cudaGraphLaunch(S.gm_exec, st));
    k_gm_solve<<<1, 1, 0, st>>>(S.gs, S.H, S.g, S.yv);
    k_gm_combine<<<nb, 256, 0, st>>>(S.V, S.yv, S.gs, N1, S.u);
    if ((s = tri_apply(S, S.u, x)) != ANOVA_OK) return s;
    int fin[4];
    ANOVA_CUDA_TRY(cudaMemcpyAsync(fin, &S.gs->j, sizeof(fin), cudaMemcpyDeviceToHost, st));
    ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
    *iters = fin[0];
    S.krylov_total += *iters;
    if (fin[3] == 2) return fail(ANOVA_ERR_BREAKDOWN, "GMRES: singular Hessenberg matrix");
    return ANOVA_OK;
}

}  // namespace
}  // namespace anova

using namespace anova;

extern "C" {

anova_status lowrank_precond_build(anova_plan_t plan, int kind, int r, double err_tol, uint64_t seed,
                                   lowrank_t *out) {
    try {
        return lowrank_build_impl(plan, kind, r, err_tol, seed, out);
    } catch (...) {
        return fail(ANOVA_ERR_OOM, "host allocation failed");
    }
}

anova_status lowrank_info(lowrank_t lr, int *rank, int64_t *pivots) {
    if (!lr) return fail(ANOVA_ERR_INVALID_ARG, "preconditioner is NULL");
    if (rank) *rank = lr->rank;
    if (pivots)
        for (int i = 0; i < lr->rank; ++i) pivots[i] = lr->piv[i];
    return ANOVA_OK;
}

anova_status lowrank_factor(lowrank_t lr, double *L) {
    if (!lr || !L) return fail(ANOVA_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t st = lr->plan->stream;
    ANOVA_CUDA_TRY(cudaMemcpyAsync(L, lr->L64, sizeof(double) * lr->n * lr->rank, cudaMemcpyDeviceToDevice, st));
    ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
    return ANOVA_OK;
}

anova_status lowrank_set_core_path(lowrank_t lr, int path) {
    if (!lr) return fail(ANOVA_ERR_INVALID_ARG, "NULL argument");
    if (path != LOWRANK_CORE_AUTO && path != LOWRANK_CORE_SIMT && path != LOWRANK_CORE_TENSOR)
        return fail(ANOVA_ERR_INVALID_ARG, "unknown core path");
    if (path == LOWRANK_CORE_TENSOR && !core_tc_supported(lr))
        return fail(ANOVA_ERR_INVALID_ARG, "tensor-core Woodbury core needs rank <= 256");
    lr->core_path = path;
    return ANOVA_OK;
}

anova_status lowrank_core(lowrank_t lr, double *M, int *path_used) {
    if (!lr) return fail(ANOVA_ERR_INVALID_ARG, "NULL argument");
    if (!lr->core_ready) return fail(ANOVA_ERR_INVALID_ARG, "call lowrank_precond_set_theta first");
    cudaStream_t st = lr->plan->stream;
    if (M)
        ANOVA_CUDA_TRY(cudaMemcpyAsync(M, lr->Mcore, sizeof(double) * lr->rank * lr->rank, cudaMemcpyDeviceToDevice, st));
    ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
    if (path_used) *path_used = lr->core_used;
    return ANOVA_OK;
}

anova_status lowrank_precond_set_theta(lowrank_t lr, const double *theta, const double *y) {
    if (!lr || !theta || !y) return fail(ANOVA_ERR_INVALID_ARG, "NULL argument");
    return lowrank_set_theta_impl(lr, theta, y);
}

anova_status lowrank_precond_apply(lowrank_t lr, const double *theta, const double *y, const double *g, double *x) {
    if (!lr || !theta || !y || !g || !x) return fail(ANOVA_ERR_INVALID_ARG, "NULL argument");
    if (g == x) return fail(ANOVA_ERR_INVALID_ARG, "g and x must be distinct");
    return lowrank_apply_impl(lr, theta, y, g, x);
}

void lowrank_destroy(lowrank_t lr) {
    if (!lr) return;
    cudaStreamSynchronize(lr->plan->stream);
    lowrank_release(lr);
}

void svm_opts_default(svm_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->max_iter = 50;
    o->sigma_barrier = 0.6;
    o->gamma = 0.99995;
    o->sigma_rule = SVM_SIGMA_ADAPTIVE;
    o->alpha0 = 0.0;
    o->stop = SVM_STOP_GAP;
    o->krylov_max = 100;
    o->krylov_tol = 1e-8;
    o->refine_max = 4;
    o->precond = PCHOL_GREEDY;
    o->krylov = SVM_KRYLOV_MINRES;
    o->autotune = 0;
    o->rank = 200;
    o->err_tol = 1e-5;
    o->seed = 0;
    o->ell = 1.0;
    o->windows = nullptr;
    o->P = 0;
    o->N = 32;
    o->m = 4;
    o->N_precise = 64;
    o->m_precise = 6;
    o->m_refine = 4;
    o->scale_features = 0;
    o->cuda_stream = nullptr;
}

anova_status svm_ipm_solve(const double *X, int64_t n, int d, const double *yh, double C, double tol,
                           const svm_opts *opts_in, double *alpha_out, double *b_out, svm_stats *stats) {
    try {
        const auto t_start = std::chrono::steady_clock::now();
        svm_opts o;
        svm_opts_default(&o);
        if (opts_in) o = *opts_in;
        if (!X || !yh || !alpha_out || !b_out) return fail(ANOVA_ERR_INVALID_ARG, "NULL argument");
        if (n < 2 || d < 1) return fail(ANOVA_ERR_INVALID_ARG, "need n >= 2 and d >= 1");
        if (!(C > 0.0) || !std::isfinite(C)) return fail(ANOVA_ERR_INVALID_ARG, "C must be positive");
        if (!(tol > 0.0)) return fail(ANOVA_ERR_INVALID_ARG, "tol must be positive");
        if (o.max_iter < 1 || o.krylov_max < 1 || o.refine_max < 1 || !(o.sigma_barrier > 0 && o.sigma_barrier < 1) ||
            (o.krylov != SVM_KRYLOV_MINRES && o.krylov != SVM_KRYLOV_GMRES) ||
            (o.krylov == SVM_KRYLOV_GMRES && o.krylov_max > 1000) || (o.autotune != 0 && o.autotune != 1) ||
            !(o.gamma > 0 && o.gamma < 1) || !(o.krylov_tol > 0) || !(o.ell > 0) ||
            (o.m_refine != 0 && (o.m_refine < 3 || o.m_refine > 6)))
            return fail(ANOVA_ERR_INVALID_ARG, "invalid svm_opts");
        bool has_pos = false, has_neg = false;
        for (int64_t i = 0; i < n; ++i) {
            if (yh[i] == 1.0) has_pos = true;
            else if (yh[i] == -1.0) has_neg = true;
            else return fail(ANOVA_ERR_INVALID_ARG, "labels must be -1 or +1");
        }
        if (!has_pos || !has_neg) return fail(ANOVA_ERR_INVALID_ARG, "both classes must occur");
        // points (optionally min-max scaled) and windows
        std::vector<double> Xs;
        const double *Xp = X;
        if (o.scale_features) {
            Xs.assign(X, X + n * d);
            for (int k = 0; k < d; ++k) {
                double mn = INFINITY, mx = -INFINITY;
                for (int64_t i = 0; i < n; ++i) {
                    const double v = X[i * d + k];
                    if (!std::isfinite(v)) return fail(ANOVA_ERR_NONFINITE, "points hold NaN or Inf");
                    mn = std::min(mn, v);
                    mx = std::max(mx, v);
                }
                for (int64_t i = 0; i < n; ++i)
                    Xs[i * d + k] = mx > mn ? -kBoxHalf + 2 * kBoxHalf * (X[i * d + k] - mn) / (mx - mn) : 0.0;
            }
            Xp = Xs.data();
        }
        std::vector<int32_t> W;
        int P = o.P;
        if (o.windows) {
            W.assign(o.windows, o.windows + 3 * P);
        } else {
            P = (d + 2) / 3;
            W.assign(3 * P, -1);
            for (int l = 0; l < P; ++l)
                for (int k = 0; k < 3 && 3 * l + k < d; ++k) W[3 * l + k] = 3 * l + k;
        }
        std::vector<double> ell(std::max(P, 1), o.ell);
        // the FP32 plan, the FP64 plan and the refinement residuals' FP64 plan (same points and
        // bandwidth, a shorter window); without tuning, the first and the last are built on helper
        // threads while this thread builds the FP64 plan (their host work overlaps)
        const bool sep_refine = o.m_refine != 0 && o.m_refine != o.m_precise;
        auto build = [&](int N_, int m_, int prec, anova_plan **out) -> anova_status {
            return o.autotune ? tune_plan(Xp, n, d, W.data(), P, ell.data(), nullptr, N_, m_, prec, o.cuda_stream, 1, 3,
                                          nullptr, out)
                              : create_plan(Xp, n, d, W.data(), P, ell.data(), nullptr, N_, m_, prec, o.cuda_stream, out);
        };
        struct Helper {
            anova_plan *plan = nullptr;
            anova_status status = ANOVA_OK;
            std::string error;
            std::thread th;
            ~Helper() {
                if (th.joinable()) th.join();
                if (plan) destroy_plan(plan);
            }
        } h32, h64r;
        int dev = 0;
        ANOVA_CUDA_TRY(cudaGetDevice(&dev));
        auto start = [&](Helper &h, int N_, int m_, int prec) {
            h.th = std::thread([&h, &build, dev, N_, m_, prec]() {
                cudaSetDevice(dev);
                h.status = build(N_, m_, prec, &h.plan);
                if (h.status != ANOVA_OK) h.error = anova_last_error();
            });
        };
        anova_status s;
        anova_plan *p64 = nullptr;
        if (o.autotune) {
            // tuned plans are timed one at a time
            if ((s = build(o.N, o.m, ANOVA_FP32, &h32.plan)) != ANOVA_OK) return s;
            if ((s = build(o.N_precise, o.m_precise, ANOVA_FP64, &p64)) != ANOVA_OK) return s;
            if (sep_refine && (s = build(o.N_precise, o.m_refine, ANOVA_FP64, &h64r.plan)) != ANOVA_OK) {
                destroy_plan(p64);
                return s;
            }
        } else {
            start(h32, o.N, o.m, ANOVA_FP32);
            if (sep_refine) start(h64r, o.N_precise, o.m_refine, ANOVA_FP64);
            s = build(o.N_precise, o.m_precise, ANOVA_FP64, &p64);
            if (h32.th.joinable()) h32.th.join();
            if (h64r.th.joinable()) h64r.th.join();
            if (s != ANOVA_OK) return s;
            for (Helper *h : {&h32, &h64r})
                if (h->status != ANOVA_OK) {
                    destroy_plan(p64);
                    set_error(h->error);
                    return h->status;
                }
        }
        anova_plan *p32 = h32.plan;
        h32.plan = nullptr;
        std::unique_ptr<anova_plan, void (*)(anova_plan *)> g32(p32, destroy_plan);
        std::unique_ptr<anova_plan, void (*)(anova_plan *)> g64(p64, destroy_plan);
        anova_plan *p64r = sep_refine ? h64r.plan : p64;
        h64r.plan = nullptr;
        std::unique_ptr<anova_plan, void (*)(anova_plan *)> g64r(p64r != p64 ? p64r : nullptr, destroy_plan);
        lowrank *lr = nullptr;
        if ((s = lowrank_build_impl(p64, o.precond, (int)std::min<int64_t>(o.rank, n), o.err_tol, o.seed, &lr)) != ANOVA_OK)
            return s;
        std::unique_ptr<lowrank, void (*)(lowrank *)> glr(lr, lowrank_release);

        Solver S;
        S.p32 = p32;
        S.p64 = p64;
        S.p64r = p64r;
        S.lr = lr;
        S.st = p64->stream;
        S.n = n;
        cudaStream_t st = S.st;
        const long long N1 = n + 1;
        // device vectors
        std::vector<void *> bufs;
        auto dalloc = [&](size_t bytes, void **ptr) -> bool {
            if (cudaMalloc(ptr, bytes) != cudaSuccess) return false;
            bufs.push_back(*ptr);
            return true;
        };
        struct Freer {
            std::vector<void *> &b;
            ~Freer() {
                for (void *x : b) cudaFree(x);
            }
        } freer{bufs};
        double *dy, *dal, *dth, *df, *drhs, *ddelta, *dr, *dtmp, *dcorr, *dpart2;
        double *work[10];
        bool ok = dalloc(sizeof(double) * n, (void **)&dy) && dalloc(sizeof(double) * n, (void **)&dal) &&
                  dalloc(sizeof(double) * n, (void **)&dth) && dalloc(sizeof(double) * n, (void **)&df) &&
                  dalloc(sizeof(double) * N1, (void **)&drhs) && dalloc(sizeof(double) * N1, (void **)&ddelta) &&
                  dalloc(sizeof(double) * N1, (void **)&dr) && dalloc(sizeof(double) * N1, (void **)&dtmp) &&
                  dalloc(sizeof(double) * N1, (void **)&dcorr) && dalloc(sizeof(double) * kRedBlocks * 5, (void **)&S.part) &&
                  dalloc(sizeof(double) * kRedBlocks * 5, (void **)&dpart2) &&
                  dalloc(sizeof(float) * n, (void **)&S.t32) && dalloc(sizeof(float) * n, (void **)&S.k32) &&
                  dalloc(sizeof(double) * n, (void **)&S.t64) && dalloc(sizeof(double) * n, (void **)&S.k64);
        for (int k = 0; k < 10 && ok; ++k) ok = dalloc(sizeof(double) * N1, (void **)&work[k]);
        ok = ok && dalloc(sizeof(MinresState), (void **)&S.ms);
        if (o.krylov == SVM_KRYLOV_GMRES) {
            const int m = o.krylov_max;
            S.gm_m = m;
            ok = ok && dalloc(sizeof(GmresState), (void **)&S.gs) &&
                 dalloc(sizeof(double) * N1 * (m + 1), (void **)&S.V) &&
                 dalloc(sizeof(double) * (size_t)(m + 1) * m, (void **)&S.H) && dalloc(sizeof(double) * m, (void **)&S.cs) &&
                 dalloc(sizeof(double) * m, (void **)&S.sn) && dalloc(sizeof(double) * (m + 1), (void **)&S.g) &&
                 dalloc(sizeof(double) * m, (void **)&S.yv) && dalloc(sizeof(double) * (m + 1), (void **)&S.hbuf) &&
                 dalloc(sizeof(double) * kGsBlocks * (m + 1), (void **)&S.gpart) &&
                 dalloc(sizeof(double), (void **)&S.bnorm2) && dalloc(sizeof(double) * N1, (void **)&S.vj) &&
                 dalloc(sizeof(double) * N1, (void **)&S.z) && dalloc(sizeof(double) * N1, (void **)&S.w) &&
                 dalloc(sizeof(double) * N1, (void **)&S.u);
        }
        if (!ok) return fail(ANOVA_ERR_OOM, "solver allocation failed");
        struct HostRes {
            Solver &s;
            ~HostRes() {
                if (s.exec) cudaGraphExecDestroy(s.exec);
                if (s.graph) cudaGraphDestroy(s.graph);
                if (s.gm_exec) cudaGraphExecDestroy(s.gm_exec);
                if (s.gm_graph) cudaGraphDestroy(s.gm_graph);
                if (s.cap) {
                    cudaStreamSynchronize(s.cap);
                    cudaStreamDestroy(s.cap);
                }
                if (s.hflags) cudaFreeHost(s.hflags);
                if (s.ev) cudaEventDestroy(s.ev);
            }
        } host_res{S};
        ANOVA_CUDA_TRY(cudaHostAlloc((void **)&S.hflags, sizeof(int) * 4, cudaHostAllocDefault));
        ANOVA_CUDA_TRY(cudaEventCreateWithFlags(&S.ev, cudaEventDisableTiming));
        S.y = dy;
        S.theta = dth;
        ANOVA_CUDA_TRY(cudaMemcpyAsync(dy, yh, sizeof(double) * n, cudaMemcpyHostToDevice, st));
        const int nb = blocks_for(n);
        // Algorithm 1: alpha^0 (default min(C/2, 1/2)), lambda^0 = 0, mu_0 = 1
        const double a0 = o.alpha0 > 0.0 ? o.alpha0 : std::min(C / 2.0, 0.5);
        if (!(a0 < C)) return fail(ANOVA_ERR_INVALID_ARG, "alpha0 must lie in (0, C)");
        k_fill_d<<<nb, 256, 0, st>>>(dal, n, a0);
        double lam = 0.0, mu = 1.0, s_prev = 1.0;
        if ((s = S.kya(dal, df)) != ANOVA_OK) return s;
        std::vector<double> hp(kRedBlocks * 5);
        auto objectives = [&](double *sums) -> anova_status {
            k_objective_partial<<<nb, 256, 0, st>>>(dal, dy, df, -lam, lam, mu, C, n, dpart2);
            ANOVA_CUDA_TRY(cudaGetLastError());
            ANOVA_CUDA_TRY(cudaMemcpyAsync(hp.data(), dpart2, sizeof(double) * 5 * nb, cudaMemcpyDeviceToHost, st));
            ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
            for (int k = 0; k < 5; ++k) {
                double acc = 0.0;
                for (int i = 0; i < nb; ++i) acc += hp[k * nb + i];
                sums[k] = acc;
            }
            return ANOVA_OK;
        };
        double sums[5];
        if ((s = objectives(sums)) != ANOVA_OK) return s;
        const double nxa0 = std::max(1.0, std::fabs(sums[3]));
        const double nxl0 = std::max(1.0, std::sqrt(sums[4]));
        double dual = sums[0] - 0.5 * sums[1], primal = 0.5 * sums[1] + C * sums[2];
        double xa = std::fabs(sums[3]) / nxa0, xl = std::sqrt(sums[4]) / nxl0;
        int it = 0;
        bool converged = false;
        auto done = [&]() {
            if (o.stop == SVM_STOP_ALG1) return !(mu > tol || xa > tol || xl > tol);
            if (it == 0) return false;
            return (primal - dual) / std::max(1.0, std::fabs(primal)) <= tol && xa <= tol;
        };
        std::vector<double> hstep(kRedBlocks);
        // f = K (y .* alpha) is updated as f += step K (y .* d_alpha) when the last FP64 residual
        // of the Newton solve was taken at the final direction (that product is then at hand),
        // and recomputed in full every kFullKya steps and before convergence is accepted
        constexpr int kFullKya = 8;
        bool f_incremental = false;
        auto refresh = [&]() -> anova_status {
            anova_status r;
            if ((r = S.kya(dal, df)) != ANOVA_OK) return r;
            if ((r = objectives(sums)) != ANOVA_OK) return r;
            dual = sums[0] - 0.5 * sums[1];
            primal = 0.5 * sums[1] + C * sums[2];
            xa = std::fabs(sums[3]) / nxa0;
            xl = std::sqrt(sums[4]) / nxl0;
            f_incremental = false;
            return ANOVA_OK;
        };
        while (it < o.max_iter) {
            if (done() && f_incremental && (s = refresh()) != ANOVA_OK) return s;
            if (done()) {
                converged = true;
                break;
            }
            mu *= o.sigma_rule == SVM_SIGMA_CONSTANT ? o.sigma_barrier : 1.0 - (1.0 - o.sigma_barrier) * s_prev;
            k_theta<<<nb, 256, 0, st>>>(dal, mu, C, n, dth);
            k_newton_rhs<<<nb, 256, 0, st>>>(dal, dy, df, lam, mu, C, n, drhs);
            k_dot<<<nb, 256, 0, st>>>(dy, dal, n, S.part);
            k_sum_to<<<1, 32, 0, st>>>(S.part, nb, 1.0, drhs + n);  // y^T alpha
            ANOVA_CUDA_TRY(cudaGetLastError());
            if ((s = lowrank_set_theta_impl(lr, dth, dy)) != ANOVA_OK) return s;
            // Newton direction: MINRES on the FP32 operator, refined with FP64 residuals
            double gnorm2;
            if ((s = S.dot(drhs, drhs, N1, &gnorm2)) != ANOVA_OK) return s;
            const double gnorm = std::sqrt(gnorm2);
            ANOVA_CUDA_TRY(cudaMemsetAsync(ddelta, 0, sizeof(double) * N1, st));
            ANOVA_CUDA_TRY(cudaMemcpyAsync(dr, drhs, sizeof(double) * N1, cudaMemcpyDeviceToDevice, st));
            const double inner_tol = std::max(o.krylov_tol, 1e-6);
            double rel_prev = 1.0;
            bool solved = false;
            bool kdelta_ready = false;  // S.k64 = K (y .* d_alpha) for the final direction
            for (int k = 0; k < o.refine_max; ++k) {
                int iters = 0;
                if (o.krylov == SVM_KRYLOV_GMRES) {
                    if ((s = gmres(S, dr, dcorr, inner_tol, &iters)) != ANOVA_OK) return s;
                } else if ((s = minres(S, dr, dcorr, inner_tol, o.krylov_max, work, &iters)) != ANOVA_OK) {
                    return s;
                }
                k_axpy<<<blocks_for(N1), 256, 0, st>>>(1.0, dcorr, N1, ddelta);
                if ((s = S.apply(ddelta, dtmp, true)) != ANOVA_OK) return s;
                k_sub<<<blocks_for(N1), 256, 0, st>>>(drhs, dtmp, N1, dr);
                S.refine_total += 1;
                double rn2;
                if ((s = S.dot(dr, dr, N1, &rn2)) != ANOVA_OK) return s;
                const double rel = std::sqrt(rn2) / gnorm;
                if (rel <= o.krylov_tol) {
                    solved = true;
                    kdelta_ready = true;
                    break;
                }
                if (rel > 0.5 * rel_prev) break;  // the FP32 operator no longer reduces the residual
                rel_prev = rel;
            }
            if (!solved) {
                // finish on the FP64 operator (same preconditioner) from the current direction
                double rn2;
                if ((s = S.dot(dr, dr, N1, &rn2)) != ANOVA_OK) return s;
                const double rel = std::sqrt(rn2) / gnorm;
                if (rel > o.krylov_tol) {
                    int iters = 0;
                    if ((s = minres(S, dr, dcorr, o.krylov_tol / rel, o.krylov_max, work, &iters, true)) != ANOVA_OK)
                        return s;
                    k_axpy<<<blocks_for(N1), 256, 0, st>>>(1.0, dcorr, N1, ddelta);
                }
            }
            // step to the boundary (Algorithm 1: s_alpha = s_lambda, times gamma_0)
            k_step_partial<<<nb, 256, 0, st>>>(dal, ddelta, C, n, S.part);
            ANOVA_CUDA_TRY(cudaGetLastError());
            ANOVA_CUDA_TRY(cudaMemcpyAsync(hstep.data(), S.part, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
            double dlam = 0.0;
            ANOVA_CUDA_TRY(cudaMemcpyAsync(&dlam, ddelta + n, sizeof(double), cudaMemcpyDeviceToHost, st));
            ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
            double smax = 1.0;
            for (int i = 0; i < nb; ++i) smax = std::min(smax, hstep[i]);
            const double step = o.gamma * smax;
            s_prev = step;
            k_axpy<<<nb, 256, 0, st>>>(step, ddelta, n, dal);
            lam += step * dlam;
            if (kdelta_ready && (it + 1) % kFullKya != 0) {
                k_axpy<<<nb, 256, 0, st>>>(step, S.k64, n, df);
                ANOVA_CUDA_TRY(cudaGetLastError());
                f_incremental = true;
            } else {
                if ((s = S.kya(dal, df)) != ANOVA_OK) return s;
                f_incremental = false;
            }
            ++it;
            if ((s = objectives(sums)) != ANOVA_OK) return s;
            dual = sums[0] - 0.5 * sums[1];
            primal = 0.5 * sums[1] + C * sums[2];
            xa = std::fabs(sums[3]) / nxa0;
            xl = std::sqrt(sums[4]) / nxl0;
            if (!std::isfinite(dual) || !std::isfinite(primal))
                return fail(ANOVA_ERR_NONFINITE, "interior point iterate is not finite");
        }
        if (!converged && f_incremental && (s = refresh()) != ANOVA_OK) return s;
        if (!converged && done()) converged = true;
        ANOVA_CUDA_TRY(cudaMemcpyAsync(alpha_out, dal, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
        ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
        *b_out = -lam;
        if (stats) {
            stats->iterations = it;
            stats->krylov_iterations = S.krylov_total;
            stats->refinements = S.refine_total;
            stats->fp64_krylov_iterations = S.fp64_krylov_total;
            stats->rank = lr->rank;
            stats->converged = converged ? 1 : 0;
            stats->mu = mu;
            stats->dual = dual;
            stats->primal = primal;
            stats->rel_gap = (primal - dual) / std::max(1.0, std::fabs(primal));
            stats->xi_alpha = xa;
            stats->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
        }
        if (!converged) return fail(ANOVA_ERR_NOT_CONVERGED, "interior point method reached max_iter");
        return ANOVA_OK;
    } catch (const std::bad_alloc &) {
        return fail(ANOVA_ERR_OOM, "host allocation failed");
    } catch (...) {
        return fail(ANOVA_ERR_INVALID_ARG, "unexpected exception");
    }
}

anova_status svm_ipm_solve_batch(svm_problem *problems, int count, double tol, const svm_opts *opts_in,
                                 int concurrency) {
    if (count < 0 || (count > 0 && !problems)) return fail(ANOVA_ERR_INVALID_ARG, "bad problem array");
    if (count == 0) return ANOVA_OK;
    svm_opts base;
    svm_opts_default(&base);
    if (opts_in) base = *opts_in;
    int dev = 0;
    ANOVA_CUDA_TRY(cudaGetDevice(&dev));
    const int workers = std::max(1, std::min(concurrency, count));
    std::atomic<int> next{0};
    auto worker = [&]() {
        cudaSetDevice(dev);
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (int i = next.fetch_add(1); i < count; i = next.fetch_add(1)) {
                problems[i].status = ANOVA_ERR_CUDA;
            }
            return;
        }
        for (int i = next.fetch_add(1); i < count; i = next.fetch_add(1)) {
            svm_problem &pr = problems[i];
            svm_opts o = base;
            o.cuda_stream = st;
            if (pr.ell > 0) o.ell = pr.ell;
            if (pr.windows) {
                o.windows = pr.windows;
                o.P = pr.P;
            }
            std::memset(&pr.stats, 0, sizeof(pr.stats));
            pr.b = 0.0;
            pr.status = svm_ipm_solve(pr.X, pr.n, pr.d, pr.y, pr.C, tol, &o, pr.alpha, &pr.b, &pr.stats);
        }
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    };
    if (workers == 1) {
        worker();
    } else {
        std::vector<std::thread> pool;
        pool.reserve(workers);
        for (int t = 0; t < workers; ++t) pool.emplace_back(worker);
        for (auto &t : pool) t.join();
    }
    for (int i = 0; i < count; ++i)
        if (problems[i].status != ANOVA_OK)
            return fail(problems[i].status, "problem " + std::to_string(i) + " of the batch failed");
    return ANOVA_OK;
}

}  // extern "C"
