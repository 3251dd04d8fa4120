// Low-rank kernel approximations and the Woodbury preconditioner (arXiv 2312.00538, Secs. 4-5).
//
//  * Algorithm 2 (greedy pivoted Cholesky) of K = sum_l K_l, column by column on the device in
//    FP64: each column of K is evaluated from the plan's FP64 window coordinates (the kernel's
//    definition, Sec. 3), the projection on the previous columns is removed, the residual
//    diagonal is updated, and the next pivot is its arg-max (ties to the lowest index). The
//    pivot never travels to the host during the build.
//  * Nystrom (Sec. 4) on the pivoted columns S: K ~ K(:,S) K(S,S)^{-1} K(S,:), with the core
//    factored as L D L^T and small D entries replaced by a threshold.
//  * Woodbury (Sec. 5): A^ = Theta + Y L L^T Y, A^{-1} = Theta^{-1} - Theta^{-1} Y L M^{-1} L^T Y
//    Theta^{-1}, M = I + L^T Theta^{-1} L (Y Theta^{-1} Y = Theta^{-1} since y_i^2 = 1). M is
//    accumulated in FP64 from an FP32 copy of the n x r panel and factored by Cholesky on the
//    device; the apply reads the FP32 panel twice, its products accumulated in FP32 pairs.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "anova_internal.h"
#include "../../include/anova_svm.h"
#include "lowrank_internal.h"


namespace anova {
namespace {

struct KernParams {
    int P;
    int dw[kMaxWindows];
    double inv_ell2[kMaxWindows];
    double eta[kMaxWindows];
};

struct ValIdx {
    double v;
    long long i;
};

__device__ __forceinline__ ValIdx better(ValIdx a, ValIdx b) {
    // larger value wins; equal values -> lower index
    if (b.v > a.v || (b.v == a.v && b.i < a.i)) return b;
    return a;
}

__device__ __forceinline__ ValIdx warp_argmax(ValIdx x) {
    for (int o = 16; o > 0; o >>= 1) {
        ValIdx y;
        y.v = __shfl_down_sync(0xffffffffu, x.v, o);
        y.i = __shfl_down_sync(0xffffffffu, x.i, o);
        x = better(x, y);
    }
    return x;
}

// kernel entry K(i, p) from the FP64 window coordinates
__device__ __forceinline__ double kernel_entry(const double *__restrict__ xw, long long n, long long i,
                                               long long p, const KernParams &kp) {
    double s = 0.0;
    for (int w = 0; w < kp.P; ++w) {
        double d2 = 0.0;
        for (int k = 0; k < kp.dw[w]; ++k) {
            const double *x = xw + ((long long)w * 3 + k) * n;
            const double t = x[i] - x[p];
            d2 += t * t;
        }
        s += kp.eta[w] * exp(-d2 * kp.inv_ell2[w]);
    }
    return s;
}

__global__ void k_fill(double *x, long long n, double v) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] = v;
}

// Column j of Algorithm 2: L(:, j) = (K(:, p) - L(:, :j) L(p, :j)^T) / sqrt(d_p), d -= L(:, j)^2,
// and a per-block arg-max of the updated residual diagonal.
__global__ void __launch_bounds__(256) k_pchol_column(int j, const double *__restrict__ xw, long long n,
                                                      KernParams kp, double *__restrict__ L,
                                                      double *__restrict__ d, const long long *__restrict__ piv,
                                                      const double *__restrict__ dpiv, const int *__restrict__ stop,
                                                      ValIdx *__restrict__ partial) {
    extern __shared__ double lp[];
    __shared__ ValIdx wbest[8];
    if (*stop >= 0) return;  // the build already stopped at a smaller rank
    const long long p = piv[j];
    const double inv_sd = 1.0 / sqrt(dpiv[j]);
    for (int q = threadIdx.x; q < j; q += blockDim.x) lp[q] = L[(long long)q * n + p];
    __syncthreads();
    ValIdx best{-INFINITY, (long long)1 << 62};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double col = kernel_entry(xw, n, i, p, kp);
        for (int q = 0; q < j; ++q) col -= L[(long long)q * n + i] * lp[q];
        const double lij = col * inv_sd;
        L[(long long)j * n + i] = lij;
        const double di = d[i] - lij * lij;
        d[i] = di;
        best = better(best, ValIdx{di, i});
    }
    best = warp_argmax(best);
    if ((threadIdx.x & 31) == 0) wbest[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x < 32) {
        ValIdx b = threadIdx.x < (blockDim.x >> 5) ? wbest[threadIdx.x] : ValIdx{-INFINITY, (long long)1 << 62};
        b = warp_argmax(b);
        if (threadIdx.x == 0) partial[blockIdx.x] = b;
    }
}

// Next pivot = arg-max over the blocks' partials; stop when rank r is reached or the residual
// diagonal is small (Algorithm 2: K_ll > 0 and r < k; tolerance err_tol * max diag).
__global__ void k_pchol_pick(int j, int nparts, const ValIdx *__restrict__ partial, long long *piv,
                             double *dpiv, int *stop, int rmax, double thresh) {
    if (*stop >= 0) return;
    ValIdx b{-INFINITY, (long long)1 << 62};
    for (int t = threadIdx.x; t < nparts; t += 32) b = better(b, partial[t]);
    b = warp_argmax(b);
    if (threadIdx.x == 0) {
        if (j + 1 >= rmax) {
            *stop = j + 1;
        } else if (!(b.v > thresh)) {
            *stop = j + 1;
        } else {
            piv[j + 1] = b.i;
            dpiv[j + 1] = b.v;
        }
    }
}

// ------------------------------------------------------------------ randomly pivoted Cholesky
// Output j of SplitMix64 started at `seed` (Steele, Lea and Flood, 2014): the state
// seed + (j + 1) * 0x9E3779B97F4A7C15 through the generator's finaliser; top 53 bits in [0, 1).
__device__ __forceinline__ double splitmix_uniform(unsigned long long seed, long long j) {
    unsigned long long z = seed + (unsigned long long)(j + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * 0x1.0p-53;
}

// sums of max(d, 0) over contiguous chunks [b chunk, (b + 1) chunk), in a fixed order
__global__ void __launch_bounds__(256) k_rp_chunk_sums(const double *__restrict__ d, long long n, long long chunk,
                                                       const int *__restrict__ stop, double *__restrict__ part) {
    __shared__ double ws[8];
    if (*stop >= 0) return;
    const long long lo = (long long)blockIdx.x * chunk, hi = min(n, lo + chunk);
    double s = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) s += fmax(d[i], 0.0);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        part[blockIdx.x] = t;
    }
}

// Pivot j + 1 (j = -1: the first) drawn in proportion to the residual diagonal: the first index s
// with cumsum(max(d, 0))[s] > u_{j+1} * sum. Stop rule as the greedy pick (rank, or the largest
// residual diagonal <= thresh); `argmax` holds the column kernel's per-block maxima (nargmax of
// them; none before the first column, when the largest entry is dmax0).
__global__ void k_rp_pick(int j, unsigned long long seed, const double *__restrict__ d, long long n,
                          long long chunk, int nchunks, const double *__restrict__ part,
                          const ValIdx *__restrict__ argmax, int nargmax, double dmax0, long long *piv,
                          double *dpiv, int *stop, int rmax, double thresh) {
    if (threadIdx.x != 0 || *stop >= 0) return;
    double dmax = dmax0;
    if (nargmax > 0) {
        dmax = -INFINITY;
        for (int t = 0; t < nargmax; ++t) dmax = fmax(dmax, argmax[t].v);
    }
    if (j + 1 >= rmax || !(dmax > thresh) || !(dmax > 0.0)) {
        *stop = j + 1;
        return;
    }
    double total = 0.0;
    for (int b = 0; b < nchunks; ++b) total += part[b];
    const double target = splitmix_uniform(seed, j + 1) * total;
    double run = 0.0;
    int b = 0;
    while (b < nchunks - 1 && run + part[b] <= target) run += part[b++];
    const long long lo = (long long)b * chunk, hi = min(n, lo + chunk);
    long long s = hi - 1;
    for (long long i = lo; i < hi; ++i) {
        run += fmax(d[i], 0.0);
        if (run > target) {
            s = i;
            break;
        }
    }
    // a draw that lands on a zero residual (rounding at a chunk edge) moves to the last positive one
    while (s > 0 && !(d[s] > 0.0)) --s;
    piv[j + 1] = s;
    dpiv[j + 1] = d[s];
}

__global__ void k_to_float(const double *__restrict__ a, float *__restrict__ b, long long cnt) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (long long)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

// ---------------------------------------------------------------- Woodbury core
// Partial Gram matrices of the scaled panel over row chunks: part[c](a, b) = sum_{i in chunk c}
// L(i, a) L(i, b) / theta_i, for 32 x 32 tiles of the lower triangle, FP64 accumulation.
constexpr int kCoreRows = 2048;

__global__ void __launch_bounds__(256) k_core_partial(const float *__restrict__ L, const double *__restrict__ itheta,
                                                      long long n, int r, int chunk_rows, const int2 *__restrict__ tiles,
                                                      double *__restrict__ part) {
    __shared__ double A[32][33];
    __shared__ double Bm[32][33];
    const int2 t = tiles[blockIdx.x];
    const int a0 = t.x * 32, b0 = t.y * 32;
    const long long i0 = (long long)blockIdx.y * chunk_rows;
    const long long i1 = min(n, i0 + chunk_rows);
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 x 32
    double acc[4] = {0, 0, 0, 0};
    for (long long ib = i0; ib < i1; ib += 32) {
        // stage 32 rows of the a-columns (scaled by 1/theta) and the b-columns
        for (int e = threadIdx.x; e < 32 * 32; e += 256) {
            const int rr = e & 31, cc = e >> 5;
            const long long i = ib + rr;
            double va = 0.0, vb = 0.0;
            if (i < i1) {
                const double it = itheta[i];
                if (a0 + cc < r) va = (double)L[(long long)(a0 + cc) * n + i] * it;
                if (b0 + cc < r) vb = (double)L[(long long)(b0 + cc) * n + i];
            }
            A[cc][rr] = va;
            Bm[cc][rr] = vb;
        }
        __syncthreads();
#pragma unroll 4
        for (int rr = 0; rr < 32; ++rr) {
            const double vb = Bm[tx][rr];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fma(A[ty + 8 * q][rr], vb, acc[q]);
        }
        __syncthreads();
    }
    const int ntiles = gridDim.x;
    for (int q = 0; q < 4; ++q) {
        const int aa = ty + 8 * q;
        part[(((long long)blockIdx.y * ntiles + blockIdx.x) * 32 + aa) * 32 + tx] = acc[q];
    }
}

// M = I + sum over chunks (fixed order), written as a full symmetric r x r matrix.
__global__ void k_core_sum(const double *__restrict__ part, int nchunks, int ntiles,
                           const int2 *__restrict__ tiles, int r, double *__restrict__ M) {
    const int tile = blockIdx.x;
    const int2 t = tiles[tile];
    for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
        const int aa = e >> 5, bb = e & 31;
        const int a = t.x * 32 + aa, b = t.y * 32 + bb;
        if (a >= r || b >= r) continue;
        // one thread writes both mirrored entries (in a diagonal tile only the lower half works),
        // so M does not depend on which of two slightly different sums lands last
        if (t.x == t.y && bb > aa) continue;
        double s = 0.0;
        for (int c = 0; c < nchunks; ++c) s += part[(((long long)c * ntiles + tile) * 32 + aa) * 32 + bb];
        if (a == b) s += 1.0;
        M[(long long)a * r + b] = s;
        M[(long long)b * r + a] = s;
    }
}

// In-place Cholesky M = R R^T of the SPD r x r matrix M (row-major, lower factor R kept; the
// strict upper triangle is left as it was), one CTA, right-looking: pivot, scale the column by the
// pivot's reciprocal, then a warp per trailing row updates it. Sets *info = 0 on success, k + 1 if
// the k-th pivot is not positive. idx maps (i, j <= i) to the storage of A.
template <typename Idx>
__device__ __forceinline__ void cholesky_cta(double *A, int r, int *bad_out, double *dinv, Idx idx) {
    __shared__ double inv_piv;
    __shared__ int bad;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int k = 0; k < r; ++k) {
        if (threadIdx.x == 0) {
            const double dk = A[idx(k, k)];
            if (!(dk > 0.0)) bad = k + 1;
            const double pv = sqrt(dk > 0.0 ? dk : 1.0);
            A[idx(k, k)] = pv;
            inv_piv = 1.0 / pv;
            dinv[k] = inv_piv;
        }
        __syncthreads();
        if (bad) break;
        for (int i = k + 1 + threadIdx.x; i < r; i += blockDim.x) A[idx(i, k)] *= inv_piv;
        __syncthreads();
        for (int i = k + 1 + warp; i < r; i += nwarps) {
            const double lik = A[idx(i, k)];
            for (int jj = k + 1 + lane; jj <= i; jj += 32) A[idx(i, jj)] -= lik * A[idx(jj, k)];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *bad_out = bad;
}

struct RowMajorIdx {
    int r;
    __device__ __forceinline__ long long operator()(int i, int j) const { return (long long)i * r + j; }
};
struct PackedIdx {
    __device__ __forceinline__ int operator()(int i, int j) const { return i * (i + 1) / 2 + j; }
};

__global__ void __launch_bounds__(1024) k_cholesky(double *M, int r, int *info, double *dinv) {
    cholesky_cta(M, r, info, dinv, RowMajorIdx{r});
}

// The same with the lower triangle packed in shared memory (r(r + 1)/2 doubles, r <= kSmemCholMax).
constexpr int kSmemCholMax = 240;

__global__ void __launch_bounds__(1024) k_cholesky_smem(double *M, int r, int *info, double *dinv) {
    extern __shared__ double A[];
    for (int i = threadIdx.x >> 5; i < r; i += blockDim.x >> 5)
        for (int j = threadIdx.x & 31; j <= i; j += 32) A[i * (i + 1) / 2 + j] = M[(long long)i * r + j];
    __syncthreads();
    cholesky_cta(A, r, info, dinv, PackedIdx{});
    __syncthreads();
    for (int i = threadIdx.x >> 5; i < r; i += blockDim.x >> 5)
        for (int j = threadIdx.x & 31; j <= i; j += 32) M[(long long)i * r + j] = A[i * (i + 1) / 2 + j];
}

// W = R^{-1} for the lower Cholesky factor R (row-major; dinv = reciprocals of its diagonal):
// one warp per column j runs the forward substitution R w = e_j (w_i = 0 for i < j); W is written
// row-major (Wl, lower) and column-major (Wc), zeros above the diagonal. Then M^{-1} v = W^T (W v):
// two parallel triangular products per application instead of two sequential substitutions. One
// warp per CTA, so that the columns' FP64 work spreads over the SMs.
__global__ void __launch_bounds__(32) k_tri_inv(const double *__restrict__ R, const double *__restrict__ dinv, int r,
                                                double *__restrict__ Wl, double *__restrict__ Wc) {
    extern __shared__ double w[];
    const int lane = threadIdx.x;
    const int j = blockIdx.x;
    for (int i = j; i < r; ++i) {
        double s = 0.0;
        for (int k = j + lane; k < i; k += 32) s = fma(R[(long long)i * r + k], w[k], s);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const double wi = ((i == j ? 1.0 : 0.0) - s) * dinv[i];
        if (lane == 0) w[i] = wi;
        __syncwarp();
    }
    for (int i = lane; i < r; i += 32) {
        const double v = i >= j ? w[i] : 0.0;
        Wl[(long long)i * r + j] = v;
        Wc[(long long)j * r + i] = v;
    }
}

// out[q] = sum over k of A[q r + k] x[k], k <= q (lower = 1) or k >= q (lower = 0); a warp per q.
__global__ void __launch_bounds__(256) k_trmv(const double *__restrict__ A, int r, int lower,
                                              const double *__restrict__ x, double *__restrict__ out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = blockIdx.x * 8 + warp;
    if (q >= r) return;
    const int k0 = lower ? 0 : q, k1 = lower ? q + 1 : r;
    double s = 0.0;
    for (int k = k0 + lane; k < k1; k += 32) s = fma(A[(long long)q * r + k], x[k], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) out[q] = s;
}

__global__ void k_recip(const double *__restrict__ a, long long n, double *__restrict__ out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = 1.0 / a[i];
}

// rows per chunk of the apply's first panel product
constexpr int kApplyRows = 1024;

// The two n x r panel products of the apply in FP32 pairs instead of FP64 (GB300's FP64 pipe runs
// at 1/64 of FP32): a product l * a with an FP32 factor a is split exactly into p + e
// (e = fma(l, a, -p)), sums are carried as S + C with the rounding error of every addition to S
// recovered exactly (two-sum) into C, and the FP64 operand is split into two FP32 parts
// (a = fl32(h), b = fl32(h - a)). The result matches FP64 accumulation to ~2^-44 of the sum of
// the terms' magnitudes.
// (explicitly rounded operations: no contraction into fused multiply-adds may change them)
__device__ __forceinline__ void two_sum_acc(float &S, float &C, float p) {
    const float t = __fadd_rn(S, p);
    const float bp = __fsub_rn(t, S);
    C = __fadd_rn(C, __fadd_rn(__fsub_rn(S, __fsub_rn(t, bp)), __fsub_rn(p, bp)));
    S = t;
}
__device__ __forceinline__ void pair_fma_acc(float &S, float &C, float l, float a, float b) {
    const float p = __fmul_rn(l, a);
    const float e = __fmaf_rn(l, a, -p);
    two_sum_acc(S, C, p);
    C = __fadd_rn(C, __fmaf_rn(l, b, e));
}

// h = y .* g ./ theta split into FP32 parts: ha = fl32(h), hb = fl32(h - ha)
__global__ void k_scaled_rhs_split(const double *__restrict__ y, const double *__restrict__ g,
                                   const double *__restrict__ itheta, long long n, float *__restrict__ ha,
                                   float *__restrict__ hb) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double h = y[i] * g[i] * itheta[i];
        const float a = __double2float_rn(h);
        ha[i] = a;
        hb[i] = __double2float_rn(h - (double)a);
    }
}

// u_part[c](q) = sum_{i in chunk c} L(i, q) h_i in FP32 pairs. Grid: (row chunks, groups of 8
// columns); one warp per column, lanes over the chunk's rows.
__global__ void __launch_bounds__(256) k_panel_t_pair(const float *__restrict__ L, const float *__restrict__ ha,
                                                      const float *__restrict__ hb, long long n, int r,
                                                      double *__restrict__ upart) {
    const long long i0 = (long long)blockIdx.x * kApplyRows;
    const long long i1 = min(n, i0 + kApplyRows);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = blockIdx.y * 8 + warp;
    if (q >= r) return;
    const float *col = L + (long long)q * n;
    float S = 0.0f, C = 0.0f;
    for (long long i = i0 + lane; i < i1; i += 32) pair_fma_acc(S, C, col[i], ha[i], hb[i]);
    for (int o = 16; o > 0; o >>= 1) {
        const float So = __shfl_down_sync(0xffffffffu, S, o), Co = __shfl_down_sync(0xffffffffu, C, o);
        two_sum_acc(S, C, So);
        C = __fadd_rn(C, Co);
    }
    if (lane == 0) upart[(long long)blockIdx.x * r + q] = (double)S + (double)C;
}

// u = sum of the chunks' partials: one warp per column, lanes over chunks, a fixed order
__global__ void __launch_bounds__(256) k_panel_t_sum_warp(const double *__restrict__ upart, int nchunks, int r,
                                                          double *__restrict__ u) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = blockIdx.x * 8 + warp;
    if (q >= r) return;
    double s = 0.0;
    for (int c = lane; c < nchunks; c += 32) s += upart[(long long)c * r + q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) u[q] = s;
}

// x_i = g_i / theta_i - (y_i / theta_i) sum_q L(i, q) z_q for i < n; x_n = g_n / s_schur, the sum
// over q in FP32 pairs (z split into FP32 parts in shared memory). 32 rows per CTA (one per lane);
// the 8 warps split the columns q and their partial sums are added in a fixed order.
__global__ void __launch_bounds__(256) k_panel_n_pair(const float *__restrict__ L, const double *__restrict__ itheta,
                                                      const double *__restrict__ y, const double *__restrict__ g,
                                                      const double *__restrict__ z, long long n, int r,
                                                      double *__restrict__ x, const double *__restrict__ schur) {
    extern __shared__ float smf[];
    float *za = smf, *zb = smf + r;
    float *ps = smf + 2 * r;  // [8][32] pairs
    for (int q = threadIdx.x; q < r; q += blockDim.x) {
        const double zq = z[q];
        const float a = __double2float_rn(zq);
        za[q] = a;
        zb[q] = __double2float_rn(zq - (double)a);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long i = (long long)blockIdx.x * 32 + lane;
    float S = 0.0f, C = 0.0f;
    if (i < n)
        for (int q = warp; q < r; q += 8) pair_fma_acc(S, C, L[(long long)q * n + i], za[q], zb[q]);
    ps[2 * (warp * 32 + lane)] = S;
    ps[2 * (warp * 32 + lane) + 1] = C;
    __syncthreads();
    if (warp == 0 && i < n) {
        float S0 = ps[2 * lane], C0 = ps[2 * lane + 1];
#pragma unroll
        for (int w = 1; w < 8; ++w) {
            two_sum_acc(S0, C0, ps[2 * (w * 32 + lane)]);
            C0 = __fadd_rn(C0, ps[2 * (w * 32 + lane) + 1]);
        }
        const double t = (double)S0 + (double)C0;
        const double it = itheta[i];
        x[i] = g[i] * it - y[i] * it * t;
    }
    if (schur && blockIdx.x == 0 && threadIdx.x == 0) x[n] = g[n] / *schur;
}

// s = y^T A^{-1} y from the Woodbury apply of y (partial dots, then one block)
__global__ void k_dot_partial(const double *__restrict__ a, const double *__restrict__ b, long long n,
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

__global__ void k_sum_parts(const double *__restrict__ part, int np, double *__restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < np; ++i) s += part[i];
        *out = s;
    }
}

// Nystrom core on the pivot set: C = K(S, S) (r x r), then L <- L_S-based factor. With the
// pivoted-Cholesky columns, K(:, S) = L R^T where R = L(S, :) (lower triangular in pivot order),
// so C = R R^T and K(:,S) C^{-1} K(S,:) = L L^T: the Nystrom approximation on S equals the
// pivoted-Cholesky one. The L D L^T route of Sec. 4 is therefore applied to C directly and the
// factor Z = K(:, S) L_C^{-T} D^{-1/2} replaces L.
__global__ void k_gather_core(const double *__restrict__ xw, long long n, KernParams kp,
                              const long long *__restrict__ piv, int r, double *__restrict__ C) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < r * r; e += gridDim.x * blockDim.x) {
        const int a = e / r, b = e % r;
        C[e] = kernel_entry(xw, n, piv[a], piv[b], kp);
    }
}

// L D L^T without pivoting, one CTA, in place (unit lower factor below the diagonal, D on it);
// D entries below thresh are replaced by thresh.
__global__ void __launch_bounds__(1024) k_ldl(double *C, int r, double rel_thresh) {
    __shared__ double dk_s, thr;
    if (threadIdx.x == 0) {
        double mx = 0.0;
        for (int k = 0; k < r; ++k) mx = fmax(mx, fabs(C[(long long)k * r + k]));
        thr = rel_thresh * mx;
    }
    __syncthreads();
    for (int k = 0; k < r; ++k) {
        if (threadIdx.x == 0) {
            double dk = C[(long long)k * r + k];
            if (dk < thr) dk = thr;
            C[(long long)k * r + k] = dk;
            dk_s = dk;
        }
        __syncthreads();
        for (int i = k + 1 + threadIdx.x; i < r; i += blockDim.x) C[(long long)i * r + k] /= dk_s;
        __syncthreads();
        const int m = r - k - 1;
        for (long long e = threadIdx.x; e < (long long)m * m; e += blockDim.x) {
            const int i = k + 1 + (int)(e / m), jj = k + 1 + (int)(e % m);
            if (jj <= i) C[(long long)i * r + jj] -= C[(long long)i * r + k] * C[(long long)jj * r + k] * dk_s;
        }
        __syncthreads();
    }
}

// Z(:, q) for the Nystrom factor: row i solves L_C z^T = (K Q)(i, :) forward, then scales by
// D^{-1/2}. (K Q)(i, a) is K(i, S_a) for a pivot set S (Wq == nullptr), else Wq[a n + i].
__global__ void __launch_bounds__(128) k_nystrom_rows(const double *__restrict__ xw, long long n, KernParams kp,
                                                      const long long *__restrict__ piv, const double *__restrict__ C,
                                                      int r, double *__restrict__ Z, const double *__restrict__ Wq) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        for (int a = 0; a < r; ++a) {
            double s = Wq ? Wq[(long long)a * n + i] : kernel_entry(xw, n, i, piv[a], kp);
            for (int b = 0; b < a; ++b) s -= C[(long long)a * r + b] * Z[(long long)b * n + i];
            Z[(long long)a * n + i] = s;
        }
        for (int a = 0; a < r; ++a) Z[(long long)a * n + i] /= sqrt(C[(long long)a * r + a]);
    }
}

// ---------------------------------------------------------------- randomised Nystrom (Sec. 4)
// Entry t = j n + i of the Gaussian G in K G: the Box-Muller transform (Box and Muller, 1958)
// sqrt(-2 ln(1 - u)) cos(2 pi u') of the SplitMix64 uniforms u = number 2t, u' = number 2t + 1.
__global__ void k_gauss(double *__restrict__ G, long long cnt, unsigned long long seed) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += (long long)gridDim.x * blockDim.x) {
        const double u = splitmix_uniform(seed, 2 * t), u2 = splitmix_uniform(seed, 2 * t + 1);
        G[t] = sqrt(-2.0 * log(1.0 - u)) * cos(2.0 * 3.141592653589793 * u2);
    }
}

constexpr int kOrthRows = 2048;

// part[c * t + q] = sum over row chunk c of Q(i, q) v(i), q < t (one warp per column).
__global__ void __launch_bounds__(256) k_qt_partial(const double *__restrict__ Q, long long n, int t,
                                                    const double *__restrict__ v, double *__restrict__ part) {
    const long long i0 = (long long)blockIdx.x * kOrthRows;
    const long long i1 = min(n, i0 + kOrthRows);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int q = blockIdx.y * 8 + warp; q < t; q += gridDim.y * 8) {
        double s = 0.0;
        for (long long i = i0 + lane; i < i1; i += 32) s = fma(Q[(long long)q * n + i], v[i], s);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) part[(long long)blockIdx.x * t + q] = s;
    }
}

// h[q] = sum over chunks (fixed order) of part[c * t + q]
__global__ void k_sum_chunks(const double *__restrict__ part, int nch, int t, double *__restrict__ h) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < t; q += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < nch; ++c) s += part[(long long)c * t + q];
        h[q] = s;
    }
}

// v -= Q(:, :t) h
__global__ void __launch_bounds__(256) k_sub_qh(const double *__restrict__ Q, long long n, int t,
                                                const double *__restrict__ h, double *__restrict__ v) {
    extern __shared__ double hs[];
    for (int q = threadIdx.x; q < t; q += blockDim.x) hs[q] = h[q];
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < t; ++q) s = fma(Q[(long long)q * n + i], hs[q], s);
        v[i] -= s;
    }
}

__global__ void k_scale_to(const double *__restrict__ src, long long n, const double *__restrict__ nrm2,
                           double *__restrict__ dst) {
    const double inv = 1.0 / sqrt(*nrm2);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = src[i] * inv;
}

// Partial products S = A^T B of two n x k column-major FP64 panels over row chunks, 32 x 32 tiles
// (tile index a_tile * nt + b_tile), FP64 accumulation.
__global__ void __launch_bounds__(256) k_atb_partial(const double *__restrict__ A, const double *__restrict__ B,
                                                     long long n, int k, int nt, double *__restrict__ part) {
    __shared__ double As[32][33];
    __shared__ double Bs[32][33];
    const int a0 = (blockIdx.x / nt) * 32, b0 = (blockIdx.x % nt) * 32;
    const long long i0 = (long long)blockIdx.y * kCoreRows;
    const long long i1 = min(n, i0 + kCoreRows);
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    double acc[4] = {0, 0, 0, 0};
    for (long long ib = i0; ib < i1; ib += 32) {
        for (int e = threadIdx.x; e < 32 * 32; e += 256) {
            const int rr = e & 31, cc = e >> 5;
            const long long i = ib + rr;
            As[cc][rr] = (i < i1 && a0 + cc < k) ? A[(long long)(a0 + cc) * n + i] : 0.0;
            Bs[cc][rr] = (i < i1 && b0 + cc < k) ? B[(long long)(b0 + cc) * n + i] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int rr = 0; rr < 32; ++rr) {
            const double vb = Bs[tx][rr];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fma(As[ty + 8 * q][rr], vb, acc[q]);
        }
        __syncthreads();
    }
    for (int q = 0; q < 4; ++q)
        part[(((long long)blockIdx.y * gridDim.x + blockIdx.x) * 32 + ty + 8 * q) * 32 + tx] = acc[q];
}

// C = (S + S^T) / 2, S = sum over chunks (fixed order) of the partial tiles; C row-major k x k.
__global__ void k_atb_sym(const double *__restrict__ part, int nchunks, int nt, int k, double *__restrict__ C) {
    const int ntiles = nt * nt;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)k * k;
         e += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(e / k), b = (int)(e % k);
        if (b > a) continue;
        double sab = 0.0, sba = 0.0;
        const int tab = (a / 32) * nt + b / 32, tba = (b / 32) * nt + a / 32;
        for (int c = 0; c < nchunks; ++c) {
            sab += part[(((long long)c * ntiles + tab) * 32 + a % 32) * 32 + b % 32];
            sba += part[(((long long)c * ntiles + tba) * 32 + b % 32) * 32 + a % 32];
        }
        const double v = 0.5 * (sab + sba);
        C[(long long)a * k + b] = v;
        C[(long long)b * k + a] = v;
    }
}

KernParams kern_params(const anova_plan *p) {
    KernParams kp;
    std::memset(&kp, 0, sizeof(kp));
    kp.P = p->P;
    for (int w = 0; w < p->P; ++w) {
        kp.dw[w] = p->win[w].dw;
        kp.inv_ell2[w] = 1.0 / (p->win[w].ell * p->win[w].ell);
        kp.eta[w] = p->win[w].eta;
    }
    return kp;
}

int grid_for(long long n, int threads, int cap = 152 * 8) {
    return (int)std::max<long long>(1, std::min<long long>((n + threads - 1) / threads, cap));
}

}  // namespace

void lowrank_release(lowrank *lr) {
    if (!lr) return;
    void *bufs[] = {lr->L64, lr->L32, lr->d, lr->piv_dev, lr->dpiv, lr->stop, lr->partial, lr->M,
                    lr->u, lr->z, lr->upart, lr->tiles, lr->cpart, lr->info, lr->tmp,
                    lr->dpart, lr->schur, lr->Wl, lr->Wc, lr->tmp2, lr->dinv, lr->itheta, lr->hbuf,
                    lr->Mcore, lr->tc_Q, lr->tc_I, lr->tc_srow, lr->tc_srow32, lr->tc_cmax, lr->tc_work, lr->tc_status};
    for (void *b : bufs)
        if (b) cudaFree(b);
    delete lr;
}

static anova_status lowrank_finish(lowrank *lr);
static anova_status per_window_build(anova_plan *p, lowrank *lr, int r, double err_tol, int nb);
static anova_status nystrom_random_build(anova_plan *p, lowrank *lr, int k, uint64_t seed);

anova_status lowrank_build_impl(anova_plan *p, int kind, int r, double err_tol, uint64_t seed, lowrank **out) {
    if (!out) return fail(ANOVA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!p) return fail(ANOVA_ERR_INVALID_ARG, "plan is NULL");
    if (kind != PCHOL_GREEDY && kind != NYSTROM && kind != PCHOL_RANDOM && kind != PCHOL_PER_WINDOW &&
        kind != NYSTROM_RANDOM)
        return fail(ANOVA_ERR_INVALID_ARG, "unknown preconditioner kind");
    if (kind == NYSTROM_RANDOM && p && p->prec != ANOVA_FP64)
        return fail(ANOVA_ERR_INVALID_ARG, "the randomised Nystrom factor needs an FP64 plan");
    if (r < 1 || r > 1024) return fail(ANOVA_ERR_INVALID_ARG, "rank must be in [1, 1024]");
    if (!(err_tol >= 0.0) || !std::isfinite(err_tol)) return fail(ANOVA_ERR_INVALID_ARG, "err_tol must be >= 0");
    for (int w = 0; w < p->P; ++w)
        if (p->win[w].eta < 0) return fail(ANOVA_ERR_INVALID_ARG, "low-rank factors need eta_l >= 0 (K must be PSD)");
    const long long n = p->n;
    r = (int)std::min<long long>(r, n);
    lowrank *lr = new (std::nothrow) lowrank();
    if (!lr) return fail(ANOVA_ERR_OOM, "host allocation failed");
    lr->plan = p;
    lr->kind = kind;
    lr->rmax = r;
    lr->n = n;
    cudaStream_t st = p->stream;
    const int nb = grid_for(n, 256, 152 * 4);
    cudaError_t e;
    auto bail = [&](anova_status s) {
        lowrank_release(lr);
        return s;
    };
    if ((e = cudaMalloc(&lr->L64, sizeof(double) * n * r)) != cudaSuccess ||
        (e = cudaMalloc(&lr->d, sizeof(double) * n)) != cudaSuccess ||
        (e = cudaMalloc(&lr->piv_dev, sizeof(long long) * (r + 1))) != cudaSuccess ||
        (e = cudaMalloc(&lr->dpiv, sizeof(double) * (r + 1))) != cudaSuccess ||
        (e = cudaMalloc(&lr->stop, sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&lr->partial, 16 * (size_t)nb)) != cudaSuccess)
        return bail(fail(ANOVA_ERR_OOM, "low-rank allocation failed"));
    if (kind == NYSTROM_RANDOM) {
        anova_status s = nystrom_random_build(p, lr, r, seed);
        if (s != ANOVA_OK) return bail(s);
        *out = lr;
        return ANOVA_OK;
    }
    if (kind == PCHOL_PER_WINDOW) {
        anova_status s = per_window_build(p, lr, r, err_tol, nb);
        if (s != ANOVA_OK) return bail(s);
        *out = lr;
        return ANOVA_OK;
    }
    const KernParams kp = kern_params(p);
    double diag = 0.0;
    for (int w = 0; w < p->P; ++w) diag += p->win[w].eta;   // K_ii = sum_l eta_l
    if (!(diag > 0.0)) return bail(fail(ANOVA_ERR_INVALID_ARG, "kernel diagonal is not positive"));
    k_fill<<<nb, 256, 0, st>>>(lr->d, n, diag);
    const long long zero = 0;
    const int minus1 = -1;
    ANOVA_CUDA_TRY(cudaMemcpyAsync(lr->piv_dev, &zero, sizeof(long long), cudaMemcpyHostToDevice, st));
    ANOVA_CUDA_TRY(cudaMemcpyAsync(lr->dpiv, &diag, sizeof(double), cudaMemcpyHostToDevice, st));
    ANOVA_CUDA_TRY(cudaMemcpyAsync(lr->stop, &minus1, sizeof(int), cudaMemcpyHostToDevice, st));
    const double thresh = err_tol * diag;
    // randomly pivoted: contiguous chunks of the residual diagonal for the draws
    const bool random = kind == PCHOL_RANDOM;
    const int rp_chunks = (int)std::min<long long>(1024, std::max<long long>(1, (n + 1023) / 1024));
    const long long rp_chunk = (n + rp_chunks - 1) / rp_chunks;
    double *rp_part = nullptr;
    if (random) {
        if ((e = cudaMalloc(&rp_part, sizeof(double) * rp_chunks)) != cudaSuccess)
            return bail(fail(ANOVA_ERR_OOM, "low-rank allocation failed"));
        k_rp_chunk_sums<<<rp_chunks, 256, 0, st>>>(lr->d, n, rp_chunk, lr->stop, rp_part);
        k_rp_pick<<<1, 32, 0, st>>>(-1, seed, lr->d, n, rp_chunk, rp_chunks, rp_part, nullptr, 0, diag,
                                    (long long *)lr->piv_dev, lr->dpiv, lr->stop, r + 1, thresh);
    }
    struct FreeDev {
        void *p;
        ~FreeDev() {
            if (p) cudaFree(p);
        }
    } free_rp{rp_part};
    for (int j = 0; j < r; ++j) {
        k_pchol_column<<<nb, 256, sizeof(double) * std::max(1, j), st>>>(
            j, p->xw, n, kp, lr->L64, lr->d, (const long long *)lr->piv_dev, lr->dpiv, lr->stop,
            (ValIdx *)lr->partial);
        if (random) {
            k_rp_chunk_sums<<<rp_chunks, 256, 0, st>>>(lr->d, n, rp_chunk, lr->stop, rp_part);
            k_rp_pick<<<1, 32, 0, st>>>(j, seed, lr->d, n, rp_chunk, rp_chunks, rp_part, (const ValIdx *)lr->partial,
                                        nb, diag, (long long *)lr->piv_dev, lr->dpiv, lr->stop, r, thresh);
        } else {
            k_pchol_pick<<<1, 32, 0, st>>>(j, nb, (const ValIdx *)lr->partial, (long long *)lr->piv_dev,
                                           lr->dpiv, lr->stop, r, thresh);
        }
    }
    ANOVA_CUDA_TRY(cudaGetLastError());
    int rank = 0;
    ANOVA_CUDA_TRY(cudaMemcpyAsync(&rank, lr->stop, sizeof(int), cudaMemcpyDeviceToHost, st));
    std::vector<long long> piv(r);
    ANOVA_CUDA_TRY(cudaMemcpyAsync(piv.data(), lr->piv_dev, sizeof(long long) * r, cudaMemcpyDeviceToHost, st));
    ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
    if (rank < 1 || rank > r) return bail(fail(ANOVA_ERR_CUDA, "pivoted Cholesky returned no rank"));
    lr->rank = rank;
    lr->piv.assign(piv.begin(), piv.begin() + rank);
    if (kind == NYSTROM) {
        // classic Nystrom on the pivot set with the L D L^T core (Sec. 4)
        double *C = nullptr;
        if ((e = cudaMalloc(&C, sizeof(double) * rank * rank)) != cudaSuccess)
            return bail(fail(ANOVA_ERR_OOM, "low-rank allocation failed"));
        k_gather_core<<<grid_for((long long)rank * rank, 256), 256, 0, st>>>(p->xw, n, kp,
                                                                            (const long long *)lr->piv_dev, rank, C);
        k_ldl<<<1, 1024, 0, st>>>(C, rank, 1e-10);
        k_nystrom_rows<<<grid_for(n, 128, 152 * 16), 128, 0, st>>>(p->xw, n, kp, (const long long *)lr->piv_dev,
                                                                    C, rank, lr->L64, nullptr);
        e = cudaGetLastError();
        cudaError_t e2 = cudaStreamSynchronize(st);
        cudaFree(C);
        if (e != cudaSuccess) return bail(cuda_fail(e, "Nystrom kernels"));
        if (e2 != cudaSuccess) return bail(cuda_fail(e2, "Nystrom sync"));
    }
    {
        anova_status s = lowrank_finish(lr);
        if (s != ANOVA_OK) return bail(s);
    }
    *out = lr;
    return ANOVA_OK;
}

// FP32 copy of the factor and the Woodbury workspace for rank lr->rank (factor in lr->L64).
static anova_status lowrank_finish(lowrank *lr) {
    anova_plan *p = lr->plan;
    cudaStream_t st = p->stream;
    const long long n = lr->n;
    const int rank = lr->rank;
    if ((cudaMalloc(&lr->L32, sizeof(float) * n * rank)) != cudaSuccess)
        return fail(ANOVA_ERR_OOM, "low-rank allocation failed");
    k_to_float<<<grid_for(n * rank, 256), 256, 0, st>>>(lr->L64, lr->L32, n * rank);
    // Woodbury workspace
    const int nt = (rank + 31) / 32;
    std::vector<int2> tiles;
    for (int a = 0; a < nt; ++a)
        for (int b = 0; b <= a; ++b) tiles.push_back(make_int2(a, b));
    lr->ntiles = (int)tiles.size();
    {
        // row chunks of the core's partial tiles: about 8 CTAs per SM over all tiles, at least
        // 256 rows per chunk (multiples of 32)
        const long long want = std::max<long long>(1, (152LL * 8 + lr->ntiles - 1) / lr->ntiles);
        const long long chunks = std::max<long long>(1, std::min(want, (n + 255) / 256));
        lr->core_rows = (int)(((n + chunks - 1) / chunks + 31) / 32 * 32);
        lr->nchunks = (int)((n + lr->core_rows - 1) / lr->core_rows);
    }
    lr->napply = (int)((n + kApplyRows - 1) / kApplyRows);
    if ((cudaMalloc(&lr->M, sizeof(double) * rank * rank)) != cudaSuccess ||
        (cudaMalloc(&lr->Mcore, sizeof(double) * rank * rank)) != cudaSuccess ||
        (cudaMalloc(&lr->u, sizeof(double) * rank)) != cudaSuccess ||
        (cudaMalloc(&lr->z, sizeof(double) * rank)) != cudaSuccess ||

        (cudaMalloc(&lr->upart, sizeof(double) * rank * lr->napply)) != cudaSuccess ||
        (cudaMalloc(&lr->tiles, sizeof(int2) * tiles.size())) != cudaSuccess ||
        (cudaMalloc(&lr->cpart, sizeof(double) * 1024 * tiles.size() * lr->nchunks)) != cudaSuccess ||
        (cudaMalloc(&lr->info, sizeof(int))) != cudaSuccess ||
        (cudaMalloc(&lr->tmp, sizeof(double) * (n + 1))) != cudaSuccess ||
        (cudaMalloc(&lr->dpart, sizeof(double) * 1024)) != cudaSuccess ||
        (cudaMalloc(&lr->schur, sizeof(double))) != cudaSuccess ||
        (cudaMalloc(&lr->Wl, sizeof(double) * rank * rank)) != cudaSuccess ||
        (cudaMalloc(&lr->Wc, sizeof(double) * rank * rank)) != cudaSuccess ||
        (cudaMalloc(&lr->tmp2, sizeof(double) * rank)) != cudaSuccess ||
        (cudaMalloc(&lr->dinv, sizeof(double) * rank)) != cudaSuccess ||
        (cudaMalloc(&lr->itheta, sizeof(double) * n)) != cudaSuccess ||
        (cudaMalloc(&lr->hbuf, sizeof(double) * n)) != cudaSuccess)
        return fail(ANOVA_ERR_OOM, "low-rank allocation failed");
    ANOVA_CUDA_TRY(cudaMemcpyAsync(lr->tiles, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice, st));
    ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
    return ANOVA_OK;
}

// Randomised Nystrom (Sec. 4): K ~ (K Q)(Q^T K Q)^{-1}(K Q)^T with Q = orth(K G), G the
// k_gauss matrix. Both products with K are multi-RHS matvecs of the plan. Q comes from classical
// Gram-Schmidt with one re-orthogonalisation; a column whose norm falls to 1e-10 of its norm
// before is dropped (the approximation depends only on range(Q), so dropped near-dependent
// directions change it by about their share of K). Q^T K Q (symmetrised) is factored L D L^T
// with D clamped at 1e-10 max D, and Z = (K Q) L^{-T} D^{-1/2}.
static anova_status nystrom_random_build(anova_plan *p, lowrank *lr, int k, uint64_t seed) {
    cudaStream_t st = p->stream;
    const long long n = lr->n;
    struct Bufs {
        double *A = nullptr, *B = nullptr, *part = nullptr, *h = nullptr, *nrm = nullptr, *dpart = nullptr,
               *C = nullptr, *cpart = nullptr;
        ~Bufs() {
            for (double *b : {A, B, part, h, nrm, dpart, C, cpart})
                if (b) cudaFree(b);
        }
    } bf;
    const int nch = (int)((n + kOrthRows - 1) / kOrthRows);
    const int nbd = grid_for(n, 256, 1024);
    if (cudaMalloc(&bf.A, sizeof(double) * n * k) != cudaSuccess ||
        cudaMalloc(&bf.B, sizeof(double) * n * k) != cudaSuccess ||
        cudaMalloc(&bf.part, sizeof(double) * (size_t)nch * k) != cudaSuccess ||
        cudaMalloc(&bf.h, sizeof(double) * k) != cudaSuccess || cudaMalloc(&bf.nrm, sizeof(double) * 2) != cudaSuccess ||
        cudaMalloc(&bf.dpart, sizeof(double) * 1024) != cudaSuccess)
        return fail(ANOVA_ERR_OOM, "low-rank allocation failed");
    k_gauss<<<grid_for(n * k, 256), 256, 0, st>>>(bf.A, n * k, (unsigned long long)seed);
    ANOVA_CUDA_TRY(cudaGetLastError());
    anova_status s = run_matvec_t<double>(p, bf.A, bf.B, k, -1);   // Y = K G
    if (s != ANOVA_OK) return s;
    // Q = orth(Y) in place: kept columns move to the front of B
    int t = 0;
    for (int c = 0; c < k; ++c) {
        double *v = bf.B + (long long)c * n;
        k_dot_partial<<<nbd, 256, 0, st>>>(v, v, n, bf.dpart);
        k_sum_parts<<<1, 32, 0, st>>>(bf.dpart, nbd, bf.nrm);
        for (int pass = 0; pass < 2 && t > 0; ++pass) {
            k_qt_partial<<<dim3(nch, std::min(128, (t + 7) / 8)), 256, 0, st>>>(bf.B, n, t, v, bf.part);
            k_sum_chunks<<<grid_for(t, 128), 128, 0, st>>>(bf.part, nch, t, bf.h);
            k_sub_qh<<<grid_for(n, 256, 152 * 8), 256, sizeof(double) * t, st>>>(bf.B, n, t, bf.h, v);
        }
        k_dot_partial<<<nbd, 256, 0, st>>>(v, v, n, bf.dpart);
        k_sum_parts<<<1, 32, 0, st>>>(bf.dpart, nbd, bf.nrm + 1);
        ANOVA_CUDA_TRY(cudaGetLastError());
        double nr[2];
        ANOVA_CUDA_TRY(cudaMemcpyAsync(nr, bf.nrm, sizeof(nr), cudaMemcpyDeviceToHost, st));
        ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
        if (!(nr[1] > 1e-20 * nr[0]) || !(nr[1] > 0.0)) continue;   // norm ratio <= 1e-10: dependent
        k_scale_to<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(v, n, bf.nrm + 1, bf.B + (long long)t * n);
        ++t;
    }
    if (t < 1) return fail(ANOVA_ERR_BREAKDOWN, "K G has no numerically independent column");
    s = run_matvec_t<double>(p, bf.B, bf.A, t, -1);   // W = K Q
    if (s != ANOVA_OK) return s;
    const int nt = (t + 31) / 32;
    const int nchunks = (int)((n + kCoreRows - 1) / kCoreRows);
    if (cudaMalloc(&bf.C, sizeof(double) * t * t) != cudaSuccess ||
        cudaMalloc(&bf.cpart, sizeof(double) * 1024 * (size_t)nt * nt * nchunks) != cudaSuccess)
        return fail(ANOVA_ERR_OOM, "low-rank allocation failed");
    k_atb_partial<<<dim3(nt * nt, nchunks), 256, 0, st>>>(bf.B, bf.A, n, t, nt, bf.cpart);
    k_atb_sym<<<grid_for((long long)t * t, 256), 256, 0, st>>>(bf.cpart, nchunks, nt, t, bf.C);
    k_ldl<<<1, 1024, 0, st>>>(bf.C, t, 1e-10);
    const KernParams kp = kern_params(p);
    k_nystrom_rows<<<grid_for(n, 128, 152 * 16), 128, 0, st>>>(p->xw, n, kp, nullptr, bf.C, t, lr->L64, bf.A);
    ANOVA_CUDA_TRY(cudaGetLastError());
    ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
    lr->rank = t;
    lr->piv.assign(t, -1);
    return lowrank_finish(lr);
}

// Per-window stacked factors (Sec. 4): sum_l K_l ~ [L_1 ... L_P][L_1 ... L_P]^T with L_l the
// greedy pivoted Cholesky (Algorithm 2) of window l's kernel alone, at rank r / P each (at least
// 1), stacked in the plan's window order; a window that stops early leaves no gap. The stop rule
// of window l is relative to its own diagonal eta_l.
static anova_status per_window_build(anova_plan *p, lowrank *lr, int r, double err_tol, int nb) {
    cudaStream_t st = p->stream;
    const long long n = lr->n;
    const int kw = std::max(1, r / p->P);
    const long long zero = 0;
    const int minus1 = -1;
    int col0 = 0;
    std::vector<long long> piv;
    for (int l = 0; l < p->P; ++l) {
        const double eta = p->win[l].eta;
        const int rl = std::min(kw, r - col0);
        if (!(eta > 0.0) || rl < 1) continue;
        KernParams kp;
        std::memset(&kp, 0, sizeof(kp));
        kp.P = 1;
        kp.dw[0] = p->win[l].dw;
        kp.inv_ell2[0] = 1.0 / (p->win[l].ell * p->win[l].ell);
        kp.eta[0] = eta;
        const double *xw = p->xw + (long long)l * 3 * n;
        double *L = lr->L64 + (long long)col0 * n;
        long long *pv = (long long *)lr->piv_dev + col0;
        double *dp = lr->dpiv + col0;
        k_fill<<<nb, 256, 0, st>>>(lr->d, n, eta);
        ANOVA_CUDA_TRY(cudaMemcpyAsync(pv, &zero, sizeof(long long), cudaMemcpyHostToDevice, st));
        ANOVA_CUDA_TRY(cudaMemcpyAsync(dp, &eta, sizeof(double), cudaMemcpyHostToDevice, st));
        ANOVA_CUDA_TRY(cudaMemcpyAsync(lr->stop, &minus1, sizeof(int), cudaMemcpyHostToDevice, st));
        for (int j = 0; j < rl; ++j) {
            k_pchol_column<<<nb, 256, sizeof(double) * std::max(1, j), st>>>(j, xw, n, kp, L, lr->d, pv, dp,
                                                                           lr->stop, (ValIdx *)lr->partial);
            k_pchol_pick<<<1, 32, 0, st>>>(j, nb, (const ValIdx *)lr->partial, pv, dp, lr->stop, rl,
                                           err_tol * eta);
        }
        ANOVA_CUDA_TRY(cudaGetLastError());
        int rank = 0;
        ANOVA_CUDA_TRY(cudaMemcpyAsync(&rank, lr->stop, sizeof(int), cudaMemcpyDeviceToHost, st));
        ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
        if (rank < 1 || rank > rl) return fail(ANOVA_ERR_CUDA, "pivoted Cholesky returned no rank");
        std::vector<long long> pl(rank);
        ANOVA_CUDA_TRY(cudaMemcpyAsync(pl.data(), pv, sizeof(long long) * rank, cudaMemcpyDeviceToHost, st));
        ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
        piv.insert(piv.end(), pl.begin(), pl.end());
        col0 += rank;
    }
    if (col0 < 1) return fail(ANOVA_ERR_INVALID_ARG, "kernel diagonal is not positive");
    lr->rank = col0;
    lr->piv = piv;
    return lowrank_finish(lr);
}

// Woodbury apply of the (n x n) block: x[0:n] = A^{-1} g[0:n]; if with_schur, x[n] = g[n]/s.
anova_status woodbury_apply(lowrank *lr, const double *theta, const double *y, const double *g, double *x,
                            bool with_schur) {
    (void)theta;  // the reciprocals stored by set_theta (theta must be the array given there)
    anova_plan *p = lr->plan;
    cudaStream_t st = p->stream;
    const long long n = lr->n;
    const int r = lr->rank;
    // hbuf (n doubles) holds the two FP32 parts of y .* g ./ theta
    float *ha = reinterpret_cast<float *>(lr->hbuf), *hb = ha + n;
    k_scaled_rhs_split<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(y, g, lr->itheta, n, ha, hb);
    k_panel_t_pair<<<dim3(lr->napply, (r + 7) / 8), 256, 0, st>>>(lr->L32, ha, hb, n, r, lr->upart);
    k_panel_t_sum_warp<<<(r + 7) / 8, 256, 0, st>>>(lr->upart, lr->napply, r, lr->u);
    // z = M^{-1} u = W^T (W u)
    k_trmv<<<(r + 7) / 8, 256, 0, st>>>(lr->Wl, r, 1, lr->u, lr->tmp2);
    k_trmv<<<(r + 7) / 8, 256, 0, st>>>(lr->Wc, r, 0, lr->tmp2, lr->z);
    k_panel_n_pair<<<(unsigned)((n + 31) / 32), 256, sizeof(float) * (2 * r + 512), st>>>(
        lr->L32, lr->itheta, y, g, lr->z, n, r, x, with_schur ? lr->schur : nullptr);
    ANOVA_CUDA_TRY(cudaGetLastError());
    return ANOVA_OK;
}

anova_status lowrank_set_theta_impl(lowrank *lr, const double *theta, const double *y) {
    anova_plan *p = lr->plan;
    cudaStream_t st = p->stream;
    const long long n = lr->n;
    const int r = lr->rank;
    k_recip<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(theta, n, lr->itheta);
    // M = I + L^T Theta^-1 L: exact-slice products on the tensor cores (csrc/core_tc.cu) where the
    // rank allows it, else FP64 tiles on the FP64 pipe
    const bool tensor = lr->core_path == LOWRANK_CORE_TENSOR ||
                        (lr->core_path == LOWRANK_CORE_AUTO && core_tc_supported(lr));
    if (tensor) {
        if (!core_tc_supported(lr)) return fail(ANOVA_ERR_INVALID_ARG, "tensor-core Woodbury core needs rank <= 256");
        anova_status cs = core_tc(lr);
        if (cs != ANOVA_OK) return cs;
    } else {
        k_core_partial<<<dim3(lr->ntiles, lr->nchunks), 256, 0, st>>>(lr->L32, lr->itheta, n, r, lr->core_rows,
                                                                       (const int2 *)lr->tiles, lr->cpart);
        k_core_sum<<<lr->ntiles, 256, 0, st>>>(lr->cpart, lr->nchunks, lr->ntiles, (const int2 *)lr->tiles, r, lr->M);
    }
    lr->core_used = tensor ? LOWRANK_CORE_TENSOR : LOWRANK_CORE_SIMT;
    ANOVA_CUDA_TRY(cudaMemcpyAsync(lr->Mcore, lr->M, sizeof(double) * r * r, cudaMemcpyDeviceToDevice, st));
    if (r <= kSmemCholMax) {
        static const cudaError_t attr =
            cudaFuncSetAttribute(k_cholesky_smem, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(double) * kSmemCholMax * (kSmemCholMax + 1) / 2));
        if (attr != cudaSuccess) return cuda_fail(attr, "cudaFuncSetAttribute");
        k_cholesky_smem<<<1, 1024, sizeof(double) * r * (r + 1) / 2, st>>>(lr->M, r, lr->info, lr->dinv);
    } else {
        k_cholesky<<<1, 1024, 0, st>>>(lr->M, r, lr->info, lr->dinv);
    }
    ANOVA_CUDA_TRY(cudaGetLastError());
    // the inverse factor and the Schur value are computed before the checks, so that one host
    // synchronisation serves all three (a failed factor only yields values that are discarded)
    k_tri_inv<<<r, 32, sizeof(double) * r, st>>>(lr->M, lr->dinv, r, lr->Wl, lr->Wc);
    ANOVA_CUDA_TRY(cudaGetLastError());
    // Schur complement s = y^T A^{-1} y of the block preconditioner
    anova_status s = woodbury_apply(lr, theta, y, y, lr->tmp, false);
    if (s != ANOVA_OK) return s;
    const int nb = grid_for(n, 256, 1024);
    k_dot_partial<<<nb, 256, 0, st>>>(y, lr->tmp, n, lr->dpart);
    k_sum_parts<<<1, 32, 0, st>>>(lr->dpart, nb, lr->schur);
    ANOVA_CUDA_TRY(cudaGetLastError());
    int info = 0, tc_status = 0;
    double sv = 0.0;
    ANOVA_CUDA_TRY(cudaMemcpyAsync(&info, lr->info, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (tensor) ANOVA_CUDA_TRY(cudaMemcpyAsync(&tc_status, lr->tc_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    ANOVA_CUDA_TRY(cudaMemcpyAsync(&sv, lr->schur, sizeof(double), cudaMemcpyDeviceToHost, st));
    ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
    if (tc_status != 0) return fail(ANOVA_ERR_TIMEOUT, "a bounded tensor-core wait in the Woodbury core ran out");
    if (info != 0) return fail(ANOVA_ERR_BREAKDOWN, "Woodbury core is not positive definite");
    if (!(sv > 0.0) || !std::isfinite(sv)) return fail(ANOVA_ERR_BREAKDOWN, "y^T A^{-1} y is not positive");
    lr->schur_host = sv;
    lr->core_ready = true;
    return ANOVA_OK;
}

anova_status lowrank_apply_impl(lowrank *lr, const double *theta, const double *y, const double *g, double *x) {
    if (!lr->core_ready) return fail(ANOVA_ERR_INVALID_ARG, "call lowrank_precond_set_theta first");
    return woodbury_apply(lr, theta, y, g, x, true);
}

}  // namespace anova
