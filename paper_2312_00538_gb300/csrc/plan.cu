// Plan construction of the ANOVA-NFFT fast summation (arXiv 2312.00538, Sec. 3): per window,
// points are binned by the oversampled-grid cell that holds them and sorted (stable LSD radix
// sort on the device), fractional cell offsets are stored in sorted order, and the host derives
// the cell segments, spread work items, bin tables, grid boxes and FFT line tiles from the
// sorted keys. The host also computes the FP64 plan constants (Fourier coefficients of the
// kernel, window transform, window polynomials, twiddles).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <thread>

// estimated warp instructions of the packed FP32 spread per point, per batch of up to 32 points of
// one segment, and per segment piece: the weights of the cost-balanced warp shares
#ifndef ANOVA_SPLIT_COST_POINT
#define ANOVA_SPLIT_COST_POINT 14.0
#endif
#ifndef ANOVA_SPLIT_COST_BATCH
#define ANOVA_SPLIT_COST_BATCH 170.0
#endif
#ifndef ANOVA_SPLIT_COST_PIECE
#define ANOVA_SPLIT_COST_PIECE 100.0
#endif

#include "anova_internal.h"

namespace anova {

namespace {

constexpr int kSortTile = 1024;  // keys per histogram tile (one scatter warp each)

__global__ void k_keys(const double *__restrict__ X, long long n, int d, const int *__restrict__ feat,
                       const int *__restrict__ dws, int P, int n_os, int B, int NB, int KB,
                       uint32_t *__restrict__ keys, int *__restrict__ vals) {
    const long long total = n * P;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int w = (int)(q / n);
        const long long i = q - (long long)w * n;
        const int dw = dws[w];
        uint32_t bin = 0, loc = 0;
        for (int k = 0; k < dw; ++k) {
            const double s = (X[i * d + feat[3 * w + k]] + 0.5) * n_os;
            int c = (int)floor(s);
            c = min(max(c, 0), n_os - 1);
            bin = bin * NB + (uint32_t)(c / B);
            loc = loc * B + (uint32_t)(c % B);
        }
        uint32_t bvol = 1;
        for (int k = 0; k < dw; ++k) bvol *= (uint32_t)B;
        keys[q] = ((uint32_t)w << KB) | (bin * bvol + loc);
        vals[q] = (int)i;
    }
}

__global__ void k_radix_hist(const uint32_t *__restrict__ keys, long long cnt, int shift,
                             int *__restrict__ hist, int nblk) {
    __shared__ int h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const long long b0 = (long long)blockIdx.x * kSortTile;
    const long long b1 = min(cnt, b0 + kSortTile);
    for (long long i = b0 + threadIdx.x; i < b1; i += blockDim.x)
        atomicAdd(&h[(keys[i] >> shift) & 255u], 1);
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[(long long)i * nblk + blockIdx.x] = h[i];
}

// exclusive scan of len ints in place over tiles of kScanTile, two launches: per-tile sums, then
// every tile scans itself after adding the sums of the tiles before it (at most a few hundred)
constexpr int kScanTile = 8192;   // 1024 threads x 8 consecutive ints

__device__ __forceinline__ int block_sum_1024(int v, int *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    int s = lane < 32 ? red[lane] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

__global__ void __launch_bounds__(1024) k_scan_tile_sums(const int *__restrict__ data, long long len,
                                                         int *__restrict__ tsum) {
    __shared__ int red[32];
    const long long b0 = (long long)blockIdx.x * kScanTile;
    int s = 0;
    for (int k = 0; k < 8; ++k) {
        const long long i = b0 + threadIdx.x + 1024LL * k;  // coalesced
        if (i < len) s += data[i];
    }
    s = block_sum_1024(s, red);
    if (threadIdx.x == 0) tsum[blockIdx.x] = s;
}

// exclusive scan of the tile sums in place: one block, 1024 at a time with a running carry
__global__ void __launch_bounds__(1024) k_scan_tile_prefix(int *__restrict__ tsum, int cnt) {
    __shared__ int wsum[32];
    __shared__ int carry_s;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) carry_s = 0;
    __syncthreads();
    for (int b = 0; b < cnt; b += 1024) {
        const int own = b + t < cnt ? tsum[b + t] : 0;
        int inc = own;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += u;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            int w = wsum[lane], wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += u;
            }
            wsum[lane] = wi - w;
        }
        __syncthreads();
        const int carry = carry_s;
        if (b + t < cnt) tsum[b + t] = carry + wsum[warp] + inc - own;
        __syncthreads();
        if (t == 1023) carry_s = carry + wsum[warp] + inc;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) k_scan_tiles(int *__restrict__ data, long long len,
                                                     const int *__restrict__ tprefix) {
    __shared__ int wsum[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int carry = tprefix[blockIdx.x];  // sum of all earlier tiles
    const long long i0 = (long long)blockIdx.x * kScanTile + 8LL * t;
    int v[8];
    int own = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        v[k] = i0 + k < len ? data[i0 + k] : 0;
        own += v[k];
    }
    // exclusive scan of the per-thread sums: within the warp, then across warps
    int inc = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int w = wsum[lane], wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += u;
        }
        wsum[lane] = wi - w;
    }
    __syncthreads();
    int run = carry + wsum[warp] + inc - own;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (i0 + k < len) data[i0 + k] = run;
        run += v[k];
    }
}

// stable scatter: one warp per tile, items taken in order 32 at a time
__global__ void k_radix_scatter(const uint32_t *__restrict__ kin, const int *__restrict__ vin,
                                uint32_t *__restrict__ kout, int *__restrict__ vout, long long cnt,
                                int shift, const int *__restrict__ offs, int nblk) {
    __shared__ int base[256];
    const int lane = threadIdx.x;
    for (int i = lane; i < 256; i += 32) base[i] = offs[(long long)i * nblk + blockIdx.x];
    __syncwarp();
    const long long b0 = (long long)blockIdx.x * kSortTile;
    const long long b1 = min(cnt, b0 + kSortTile);
    const unsigned lt = (1u << lane) - 1u;
    for (long long c = b0; c < b1; c += 32) {
        const long long i = c + lane;
        const bool valid = i < b1;
        const uint32_t key = valid ? kin[i] : 0u;
        const int dig = valid ? (int)((key >> shift) & 255u) : 256 + lane;
        const unsigned mask = __match_any_sync(0xffffffffu, dig);
        const int rank = __popc(mask & lt);
        int pos = 0;
        if (valid) pos = base[dig] + rank;
        __syncwarp();
        if (valid) {
            kout[pos] = key;
            vout[pos] = vin[i];
            if ((mask & lt) == 0) base[dig] += __popc(mask);
        }
        __syncwarp();
    }
}

template <typename T>
__global__ void k_gather(const uint32_t *__restrict__ keys, const int *__restrict__ vals,
                         const double *__restrict__ X, long long n, int d,
                         const int *__restrict__ feat, const int *__restrict__ dws, int P, int n_os,
                         int KB, T *__restrict__ frac, int *__restrict__ perm) {
    const long long total = n * P;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int w = (int)(keys[q] >> KB);
        const int i = vals[q];
        const int dw = dws[w];
        for (int k = 0; k < 3; ++k) {
            T f = T(0);
            if (k < dw) {
                const double s = (X[(long long)i * d + feat[3 * w + k]] + 0.5) * n_os;
                double c = floor(s);
                c = fmin(fmax(c, 0.0), (double)(n_os - 1));
                f = (T)(s - c);
            }
            frac[(long long)k * total + q] = f;
        }
        perm[q] = i;
    }
}

// FP64 window coordinates in original point order, structure of arrays (window, feature, point)
__global__ void k_window_coords(const double *__restrict__ X, long long n, int d,
                                const int *__restrict__ feat, const int *__restrict__ dws, int P,
                                double *__restrict__ xw) {
    const long long total = n * P;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int w = (int)(q / n);
        const long long i = q - (long long)w * n;
        for (int k = 0; k < 3; ++k)
            xw[((long long)w * 3 + k) * n + i] = k < dws[w] ? X[i * d + feat[3 * w + k]] : 0.0;
    }
}

int ilog2(int x) {
    int l = 0;
    while ((1 << l) < x) ++l;
    return l;
}

int bitrev(int x, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((x >> b) & 1) << (bits - 1 - b);
    return r;
}

template <typename T>
void free_dev(T *&p) {
    if (p) cudaFree(p);
    p = nullptr;
}

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

// f(t, nt) on nt host threads (t = 0 .. nt - 1; the calling thread runs t = 0); nt is capped by the
// hardware threads and by `items`, so small inputs stay on one thread
template <typename F>
void parallel_for_threads(long long items, long long min_per_thread, F f) {
    const long long hw = std::max(1u, std::thread::hardware_concurrency());
    const int nt = (int)std::max(1LL, std::min({hw, 16LL, items / std::max(1LL, min_per_thread)}));
    std::vector<std::thread> th;
    for (int t = 1; t < nt; ++t) th.emplace_back(f, t, nt);
    f(0, nt);
    for (auto &x : th) x.join();
}

// cell index inside its bin of every sorted point: the low digits of its sort key
__global__ void k_cellloc(const uint32_t *__restrict__ keys, long long total, int KB, int B,
                          const int *__restrict__ dws, unsigned char *__restrict__ loc) {
    const uint32_t kmask = KB >= 32 ? 0xffffffffu : ((1u << KB) - 1u);
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const uint32_t key = keys[q];
        const int w = (int)(key >> KB);
        uint32_t bvol = 1;
        for (int k = 0; k < dws[w]; ++k) bvol *= (uint32_t)B;
        loc[q] = (unsigned char)((key & kmask) % bvol);
    }
}

}  // namespace

size_t elem_size(const anova_plan *p) { return p->prec == ANOVA_FP64 ? sizeof(double) : sizeof(float); }

void release_workspace(anova_plan *p) {
    if (p->grids || p->tiles || p->part) ++p->ws_gen;
    if (p->grids) cudaFree(p->grids);
    if (p->tiles) cudaFree(p->tiles);
    if (p->part) cudaFree(p->part);
    p->grids = p->tiles = p->part = nullptr;
    p->ws_rhs = 0;
    p->ws_bytes = 0;
}

anova_status ensure_workspace(anova_plan *p, int nrhs) {
    if (nrhs <= p->ws_rhs) return ANOVA_OK;
    // the old buffers may still be in use by a batch graph launched on another stream, so the
    // whole device is waited for before they are freed
    cudaError_t e = (p->grids || p->tiles || p->part) ? cudaDeviceSynchronize() : cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    release_workspace(p);
    const size_t es = elem_size(p);
    const int B = p->B;
    const int tw = B + 2 * p->m - 1;
    const size_t tv = (size_t)tw * tw * tw;
    const size_t gbytes = es * 4 * (size_t)nrhs * p->grid_total;
    const size_t tbytes = es * std::max<size_t>(1, (size_t)p->nwi * nrhs * tv);
    const size_t pbytes = es * (size_t)p->P * nrhs * p->n;
    if ((e = cudaMalloc(&p->grids, gbytes)) != cudaSuccess ||
        (e = cudaMalloc(&p->tiles, tbytes)) != cudaSuccess ||
        (e = cudaMalloc(&p->part, pbytes)) != cudaSuccess) {
        release_workspace(p);
        return fail(ANOVA_ERR_OOM, std::string("workspace allocation failed: ") + cudaGetErrorString(e));
    }
    e = cudaMemsetAsync(p->grids, 0, gbytes, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    p->ws_rhs = nrhs;
    p->ws_bytes = (int64_t)(gbytes + tbytes + pbytes);
    return ANOVA_OK;
}

void destroy_plan(anova_plan *p) {
    if (!p) return;
    cudaStreamSynchronize(p->stream);
    for (int k = 0; k < 3; ++k) {
        if (p->aux[k]) {
            cudaStreamSynchronize(p->aux[k]);
            cudaStreamDestroy(p->aux[k]);
        }
        if (p->join_evt[k]) cudaEventDestroy(p->join_evt[k]);
    }
    if (p->fork_evt) cudaEventDestroy(p->fork_evt);
    if (p->host_exec) cudaGraphExecDestroy(p->host_exec);
    if (p->host_cap) cudaStreamDestroy(p->host_cap);
    release_workspace(p);
    void *bufs[] = {p->frac, p->xw, p->perm, p->cellloc, p->segs, p->wis, p->chunks, p->wi_chunk, p->wsplit, p->wi_order, p->wi_gorder, p->bins, p->mbins, p->ftiles, p->ftiles_full, p->dwin,
                    p->D1br, p->tw, p->dv, p->dkv, p->dev_status};
    for (void *b : bufs)
        if (b) cudaFree(b);
    delete p;
}

anova_status create_plan(const double *points, int64_t n, int d, const int32_t *windows, int P,
                         const double *ell, const double *eta, int N, int m, int flags,
                         void *stream, anova_plan_t *out) {
    return create_plan_shaped(points, n, d, windows, P, ell, eta, N, m, flags, stream, PlanShape(), out);
}

anova_status create_plan_shaped(const double *points, int64_t n, int d, const int32_t *windows, int P,
                                const double *ell, const double *eta, int N, int m, int flags, void *stream,
                                const PlanShape &shape, anova_plan_t *out) {
    // ------------------------------------------------------------------ validation
    if (!out) return fail(ANOVA_ERR_INVALID_ARG, "out is NULL");
    const int wi_max = shape.wi_max;
    if (wi_max < kSegMax || wi_max > (1 << 16)) return fail(ANOVA_ERR_INVALID_ARG, "work-item cap out of range");
    if (shape.conv_lines != 8 && shape.conv_lines != 16 && shape.conv_lines != 32)
        return fail(ANOVA_ERR_INVALID_ARG, "FFT lines per CTA must be 8, 16 or 32");
    *out = nullptr;
    if (!points || !windows || !ell) return fail(ANOVA_ERR_INVALID_ARG, "NULL input pointer");
    if (n < 1 || n > (int64_t)1 << 30) return fail(ANOVA_ERR_INVALID_ARG, "n must be in [1, 2^30]");
    if (d < 1) return fail(ANOVA_ERR_INVALID_ARG, "d must be >= 1");
    if (P < 1 || P > kMaxWindows) return fail(ANOVA_ERR_INVALID_ARG, "P must be in [1, 64]");
    if ((int64_t)n * P > ((int64_t)1 << 31) - 1) return fail(ANOVA_ERR_INVALID_ARG, "n * P exceeds 2^31 - 1");
    const int prec = flags & 1;
    if (flags & ~7) return fail(ANOVA_ERR_INVALID_ARG, "unknown flag bits");
    if ((flags & 6) == 6) return fail(ANOVA_ERR_INVALID_ARG, "ANOVA_INTERP_TENSOR and ANOVA_INTERP_SIMT both set");
    if (N != 16 && N != 32 && N != 64 && N != 128)
        return fail(ANOVA_ERR_INVALID_ARG, "N must be an even power of two in {16, 32, 64, 128}");
    if (prec == ANOVA_FP32 ? (m < 2 || m > 6) : (m < 3 || m > 6))
        return fail(ANOVA_ERR_INVALID_ARG, "m out of range (FP32: 2..6, FP64: 3..6)");
    for (int l = 0; l < P; ++l) {
        if (!(ell[l] > 0.0) || !std::isfinite(ell[l]))
            return fail(ANOVA_ERR_INVALID_ARG, "kernel length scale must be positive and finite");
        if (eta && !std::isfinite(eta[l])) return fail(ANOVA_ERR_NONFINITE, "window weight not finite");
        int cnt = 0;
        bool ended = false;
        for (int k = 0; k < 3; ++k) {
            const int f = windows[3 * l + k];
            if (f < 0) {
                if (f != -1) return fail(ANOVA_ERR_INVALID_ARG, "window padding must be -1");
                ended = true;
                continue;
            }
            if (ended) return fail(ANOVA_ERR_INVALID_ARG, "window padding must follow valid entries");
            if (f >= d) return fail(ANOVA_ERR_INVALID_ARG, "window feature index >= d");
            for (int k2 = 0; k2 < k; ++k2)
                if (windows[3 * l + k2] == f) return fail(ANOVA_ERR_INVALID_ARG, "repeated feature in a window");
            ++cnt;
        }
        if (cnt == 0) return fail(ANOVA_ERR_INVALID_ARG, "empty window");
    }
    {
        std::vector<char> used(d, 0);
        for (int l = 0; l < P; ++l)
            for (int k = 0; k < 3; ++k)
                if (windows[3 * l + k] >= 0) used[windows[3 * l + k]] = 1;
        // rows split over host threads; each records the kind of the first bad value it meets
        std::vector<int> bad(16, 0);  // 1: not finite, 2: outside the box
        parallel_for_threads(n, 1 << 16, [&](int t, int nt) {
            const int64_t i0 = n * t / nt, i1 = n * (t + 1) / nt;
            for (int64_t i = i0; i < i1 && !bad[t]; ++i)
                for (int k = 0; k < d; ++k) {
                    const double x = points[i * d + k];
                    if (!std::isfinite(x)) { bad[t] = 1; break; }
                    if (used[k] && (x < -kBoxHalf - 1e-12 || x > kBoxHalf + 1e-12)) { bad[t] = 2; break; }
                }
        });
        for (int b : bad) {
            if (b == 1) return fail(ANOVA_ERR_NONFINITE, "points hold NaN or Inf");
            if (b == 2) return fail(ANOVA_ERR_OUT_OF_RANGE, "a point coordinate lies outside [-0.2, 0.2]");
        }
    }
    std::unique_ptr<anova_plan, void (*)(anova_plan *)> plan(new (std::nothrow) anova_plan(),
                                                            destroy_plan);
    if (!plan) return fail(ANOVA_ERR_OOM, "host allocation failed");
    anova_plan *p = plan.get();
    p->n = n;
    p->d = d;
    p->P = P;
    p->N = N;
    p->m = m;
    p->n_os = 2 * N;
    p->prec = prec;
    p->interp_flags = flags & 6;
    p->wi_max = wi_max;
    p->conv_lines = shape.conv_lines;
    p->B = prec == ANOVA_FP64 ? kBinF64 : kBinF32;
    p->NB = p->n_os / p->B;
    p->tile_w = p->B + 2 * m - 1;
    p->stream = reinterpret_cast<cudaStream_t>(stream);
    ANOVA_CUDA_TRY(cudaGetDevice(&p->device));
    const int nos = p->n_os;
    const size_t es = elem_size(p);

    // ------------------------------------------------------------------ windows (grouped by dw)
    std::vector<int> order(P);
    for (int l = 0; l < P; ++l) order[l] = l;
    auto dw_of = [&](int l) {
        int c = 0;
        for (int k = 0; k < 3; ++k) c += windows[3 * l + k] >= 0;
        return c;
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return dw_of(a) > dw_of(b); });
    p->win.resize(P);
    p->user_to_internal.assign(P, 0);
    for (int w = 0; w < P; ++w) {
        const int l = order[w];
        p->user_to_internal[l] = w;
        WindowInfo &wi = p->win[w];
        wi.dw = dw_of(l);
        for (int k = 0; k < 3; ++k) wi.feat[k] = windows[3 * l + k];
        wi.ell = ell[l];
        wi.eta = eta ? eta[l] : 1.0;
    }

    // ------------------------------------------------------------------ host constants
    if (!window_poly(m, kPolyDeg, p->poly) || !window_poly(m, kPolyDeg64, p->poly64))
        return fail(ANOVA_ERR_INVALID_ARG, "window polynomial fit failed");
    const int lb = ilog2(nos);
    // deconvolution diagonal per window and axis, bit-reversed; eta_l scales the axis-0 copy
    std::vector<double> d1br((size_t)P * 3 * nos, 0.0);
    std::vector<std::pair<double, std::vector<double>>> d1_cache;  // windows with the same ell share it
    for (int w = 0; w < P; ++w) {
        std::vector<double> D1;
        bool cached = false;
        for (auto &c : d1_cache)
            if (c.first == p->win[w].ell) {
                D1 = c.second;
                cached = true;
                break;
            }
        if (!cached) {
            if (!deconv_diag(p->win[w].ell, N, m, nos, D1))
                return fail(ANOVA_ERR_INVALID_ARG, "kernel coefficient fit failed");
            d1_cache.emplace_back(p->win[w].ell, D1);
        }
        for (int ax = 0; ax < 3; ++ax)
            for (int e = 0; e < nos; ++e)
                d1br[((size_t)w * 3 + ax) * nos + e] = D1[bitrev(e, lb)] * (ax == 0 ? p->win[w].eta : 1.0);
    }
    std::vector<double> twid(nos);
    for (int k = 0; k < nos / 2; ++k) {
        twid[2 * k] = std::cos(-2.0 * M_PI * k / nos);
        twid[2 * k + 1] = std::sin(-2.0 * M_PI * k / nos);
    }

    // ------------------------------------------------------------------ device sort
    const long long total = (long long)n * P;
    DevBuf dX, dfeat, ddws, dk0, dv0, dk1, dv1, dhist;
    ANOVA_CUDA_TRY(cudaMalloc(&dX.p, sizeof(double) * n * d));
    ANOVA_CUDA_TRY(cudaMalloc(&dfeat.p, sizeof(int) * 3 * P));
    ANOVA_CUDA_TRY(cudaMalloc(&ddws.p, sizeof(int) * P));
    ANOVA_CUDA_TRY(cudaMalloc(&dk0.p, sizeof(uint32_t) * total));
    ANOVA_CUDA_TRY(cudaMalloc(&dv0.p, sizeof(int) * total));
    ANOVA_CUDA_TRY(cudaMalloc(&dk1.p, sizeof(uint32_t) * total));
    ANOVA_CUDA_TRY(cudaMalloc(&dv1.p, sizeof(int) * total));
    std::vector<int> hfeat(3 * P), hdws(P);
    for (int w = 0; w < P; ++w) {
        hdws[w] = p->win[w].dw;
        for (int k = 0; k < 3; ++k) hfeat[3 * w + k] = p->win[w].feat[k] < 0 ? 0 : p->win[w].feat[k];
    }
    cudaStream_t st = p->stream;
    ANOVA_CUDA_TRY(cudaMemcpyAsync(dX.p, points, sizeof(double) * n * d, cudaMemcpyHostToDevice, st));
    ANOVA_CUDA_TRY(cudaMemcpyAsync(dfeat.p, hfeat.data(), sizeof(int) * 3 * P, cudaMemcpyHostToDevice, st));
    ANOVA_CUDA_TRY(cudaMemcpyAsync(ddws.p, hdws.data(), sizeof(int) * P, cudaMemcpyHostToDevice, st));
    const int KB = 3 * lb;  // bits of the in-window key (enough for d_W <= 3)
    const int keybits = KB + ilog2(P);
    {
        const int nb = (int)std::min<long long>((total + 255) / 256, 152LL * 32);
        k_keys<<<nb, 256, 0, st>>>((const double *)dX.p, n, d, (const int *)dfeat.p, (const int *)ddws.p,
                                   P, nos, p->B, p->NB, KB, (uint32_t *)dk0.p, (int *)dv0.p);
        ANOVA_CUDA_TRY(cudaGetLastError());
    }
    const int nblk = (int)((total + kSortTile - 1) / kSortTile);
    const long long hlen = 256LL * nblk;
    const int nscan = (int)((hlen + kScanTile - 1) / kScanTile);
    ANOVA_CUDA_TRY(cudaMalloc(&dhist.p, sizeof(int) * ((size_t)hlen + nscan)));
    int *dtsum = (int *)dhist.p + hlen;
    uint32_t *kin = (uint32_t *)dk0.p, *kout = (uint32_t *)dk1.p;
    int *vin = (int *)dv0.p, *vout = (int *)dv1.p;
    for (int shift = 0; shift < keybits; shift += 8) {
        k_radix_hist<<<nblk, 256, 0, st>>>(kin, total, shift, (int *)dhist.p, nblk);
        k_scan_tile_sums<<<nscan, 1024, 0, st>>>((const int *)dhist.p, hlen, dtsum);
        k_scan_tile_prefix<<<1, 1024, 0, st>>>(dtsum, nscan);
        k_scan_tiles<<<nscan, 1024, 0, st>>>((int *)dhist.p, hlen, dtsum);
        k_radix_scatter<<<nblk, 32, 0, st>>>(kin, vin, kout, vout, total, shift, (const int *)dhist.p, nblk);
        ANOVA_CUDA_TRY(cudaGetLastError());
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    // sorted keys/values now in kin/vin
    ANOVA_CUDA_TRY(cudaMalloc(&p->frac, es * 3 * total));
    ANOVA_CUDA_TRY(cudaMalloc(&p->perm, sizeof(int) * total));
    {
        const int nb = (int)std::min<long long>((total + 255) / 256, 152LL * 32);
        if (prec == ANOVA_FP64)
            k_gather<double><<<nb, 256, 0, st>>>(kin, vin, (const double *)dX.p, n, d, (const int *)dfeat.p,
                                                 (const int *)ddws.p, P, nos, KB, (double *)p->frac, p->perm);
        else
            k_gather<float><<<nb, 256, 0, st>>>(kin, vin, (const double *)dX.p, n, d, (const int *)dfeat.p,
                                                (const int *)ddws.p, P, nos, KB, (float *)p->frac, p->perm);
        ANOVA_CUDA_TRY(cudaGetLastError());
    }
    ANOVA_CUDA_TRY(cudaMalloc(&p->xw, sizeof(double) * 3 * total));
    {
        const int nb = (int)std::min<long long>((total + 255) / 256, 152LL * 32);
        k_window_coords<<<nb, 256, 0, st>>>((const double *)dX.p, n, d, (const int *)dfeat.p,
                                            (const int *)ddws.p, P, p->xw);
        ANOVA_CUDA_TRY(cudaGetLastError());
    }
    std::vector<uint32_t> hkeys(total);
    ANOVA_CUDA_TRY(cudaMemcpyAsync(hkeys.data(), kin, sizeof(uint32_t) * total, cudaMemcpyDeviceToHost, st));
    ANOVA_CUDA_TRY(cudaStreamSynchronize(st));

    // ------------------------------------------------------------------ host tables
    const int B = p->B, NB = p->NB;
    const uint32_t kmask = (KB >= 32) ? 0xffffffffu : ((1u << KB) - 1u);
    std::vector<int4> segs, wis, ftiles;
    std::vector<int2> bins;
    int64_t goff = 0;
    // groups of consecutive windows with equal dw
    for (int w = 0; w < P; ++w) {
        if (p->groups.empty() || p->groups.back().dw != p->win[w].dw) {
            Group g;
            g.dw = p->win[w].dw;
            g.w_begin = w;
            p->groups.push_back(g);
        }
        p->groups.back().w_end = w + 1;
    }
    // per-window tables built on host threads (windows are independent), then concatenated
    struct WinTables {
        std::vector<int4> segs, wis;  // segment indices relative to the window's first segment
        std::vector<int2> bins;       // work-item indices relative to the window's first work item
        int cmin[3] = {0, 0, 0}, cmax[3] = {-1, -1, -1};
        bool bad = false;             // a bin tile would leave the grid (N too small for m)
    };
    std::vector<WinTables> wt(P);
    auto build_window = [&](int w) {
        WindowInfo &wi = p->win[w];
        WinTables &o = wt[w];
        const int dw = wi.dw;
        int bvol = 1, nbins = 1;
        for (int k = 0; k < dw; ++k) { bvol *= B; nbins *= NB; }
        o.bins.assign(nbins, make_int2(0, 0));
        int cmin[3] = {nos, nos, nos}, cmax[3] = {-1, -1, -1};
        const long long q0 = (long long)w * n, q1 = q0 + n;
        uint32_t prev = 0xffffffffu;
        int cur_bin = -1, wi_pts = 0;
        for (long long q = q0; q < q1; ++q) {
            const uint32_t key = hkeys[q] & kmask;
            const bool new_cell = key != prev;
            if (new_cell || o.segs.back().z >= kSegMax) {
                const uint32_t bin = key / bvol, loc = key % bvol;
                int c[3] = {0, 0, 0};
                uint32_t bb = bin, ll = loc;
                for (int k = dw - 1; k >= 0; --k) {
                    c[k] = (int)(bb % NB) * B + (int)(ll % B);
                    bb /= NB;
                    ll /= B;
                }
                for (int k = 0; k < dw; ++k) {
                    cmin[k] = std::min(cmin[k], c[k]);
                    cmax[k] = std::max(cmax[k], c[k]);
                }
                const int packed = c[0] | (c[1] << 10) | (c[2] << 20);
                o.segs.push_back(make_int4(packed, (int)q, 0, w));
                // work items: runs of one bin's segments, at most wi_max points
                if ((int)bin != cur_bin || wi_pts + kSegMax > p->wi_max) {
                    int bc[3] = {0, 0, 0};
                    uint32_t b2 = bin;
                    for (int k = dw - 1; k >= 0; --k) { bc[k] = (int)(b2 % NB); b2 /= NB; }
                    o.wis.push_back(make_int4(w, (int)o.segs.size() - 1, (int)o.segs.size(),
                                              bc[0] | (bc[1] << 10) | (bc[2] << 20)));
                    if ((int)bin != cur_bin) {
                        o.bins[bin] = make_int2((int)o.wis.size() - 1, 0);
                        cur_bin = (int)bin;
                    }
                    o.bins[bin].y += 1;
                    wi_pts = 0;
                    // tile of this bin must stay inside the grid
                    for (int k = 0; k < dw; ++k) {
                        const int lo = bc[k] * B - m + 1, hi = bc[k] * B + B + m - 1;
                        if (lo < 0 || hi >= nos) o.bad = true;
                    }
                    if (o.bad) return;
                }
                o.wis.back().z = (int)o.segs.size();
                prev = key;
            }
            o.segs.back().z += 1;
            wi_pts += 1;
        }
        for (int k = 0; k < 3; ++k) { o.cmin[k] = cmin[k]; o.cmax[k] = cmax[k]; }
    };
    parallel_for_threads(P, 1, [&](int t, int nt) {
        for (int w = t; w < P; w += nt) build_window(w);
    });
    for (int w = 0; w < P; ++w) {
        WindowInfo &wi = p->win[w];
        const WinTables &o = wt[w];
        if (o.bad) return fail(ANOVA_ERR_INVALID_ARG, "bandwidth N too small for this window cut-off m");
        const int dw = wi.dw;
        const int s0 = (int)segs.size(), x0 = (int)wis.size();
        wi.seg_begin = s0;
        wi.wi_begin = x0;
        wi.bin_off = (int)bins.size();
        segs.insert(segs.end(), o.segs.begin(), o.segs.end());
        for (int4 t : o.wis) wis.push_back(make_int4(t.x, t.y + s0, t.z + s0, t.w));
        for (int2 b : o.bins) bins.push_back(b.y > 0 ? make_int2(b.x + x0, b.y) : b);
        wi.seg_end = (int)segs.size();
        wi.wi_end = (int)wis.size();
        for (int k = 0; k < dw; ++k) {
            wi.box_lo[k] = o.cmin[k] - m + 1;
            wi.box_hi[k] = o.cmax[k] + m + 1;
        }
        wi.grid_off = goff;
        int64_t gsz = 1;
        for (int k = 0; k < dw; ++k) gsz *= nos;
        goff += gsz;
    }
    p->grid_total = goff;
    // FFT tiles: group -> pass -> window
    for (Group &g : p->groups) {
        for (int pass = 0; pass < g.dw; ++pass) {
            for (int w = g.w_begin; w < g.w_end; ++w) {
                WindowInfo &wi = p->win[w];
                wi.tile_begin[pass] = (int)ftiles.size();
                int plo = 0, phi = 1, qlo = 0, qhi = 1;
                // a pass transforms full lines along its axis for the box of the other axes: the
                // input is zero outside the box on axes not yet transformed, and only the box is
                // read on axes already transformed (by the later passes and the interpolation)
                if (g.dw == 3) {
                    if (pass == 0) { plo = wi.box_lo[1]; phi = wi.box_hi[1]; qlo = wi.box_lo[2]; qhi = wi.box_hi[2]; }
                    if (pass == 1) { plo = wi.box_lo[0]; phi = wi.box_hi[0]; qlo = wi.box_lo[2]; qhi = wi.box_hi[2]; }
                    if (pass == 2) { plo = wi.box_lo[0]; phi = wi.box_hi[0]; qlo = wi.box_lo[1]; qhi = wi.box_hi[1]; }
                } else if (g.dw == 2) {
                    if (pass == 0) { qlo = wi.box_lo[1]; qhi = wi.box_hi[1]; }
                    if (pass == 1) { qlo = wi.box_lo[0]; qhi = wi.box_hi[0]; }
                }
                for (int pp = plo; pp < phi; ++pp)
                    for (int q = qlo; q < qhi; q += p->conv_lines)
                        ftiles.push_back(make_int4(w, pp, q, pass | (std::min(p->conv_lines, qhi - q) << 8)));
                wi.tile_end[pass] = (int)ftiles.size();
            }
        }
    }
    // FFT tiles over whole grids, for products from grids summed over several plans' points
    // (the sum is not confined to this plan's box)
    std::vector<int4> ftiles_full;
    for (Group &g : p->groups) {
        for (int pass = 0; pass < g.dw; ++pass) {
            for (int w = g.w_begin; w < g.w_end; ++w) {
                WindowInfo &wi = p->win[w];
                wi.full_begin[pass] = (int)ftiles_full.size();
                const int phi = g.dw == 3 ? nos : 1, qhi = g.dw >= 2 ? nos : 1;
                for (int pp = 0; pp < phi; ++pp)
                    for (int q = 0; q < qhi; q += p->conv_lines)
                        ftiles_full.push_back(make_int4(w, pp, q, pass | (std::min(p->conv_lines, qhi - q) << 8)));
                wi.full_end[pass] = (int)ftiles_full.size();
            }
        }
    }
    // bins holding several work items (their partial tiles are summed before the grid gather)
    std::vector<int4> mbins;
    for (int w = 0; w < P; ++w) {
        WindowInfo &wi = p->win[w];
        int nbins = 1, tv = 1;
        for (int k = 0; k < wi.dw; ++k) { nbins *= NB; tv *= (B + 2 * m - 1); }
        wi.mb_begin = (int)mbins.size();
        for (int b = 0; b < nbins; ++b) {
            const int2 be = bins[wi.bin_off + b];
            if (be.y > 1) mbins.push_back(make_int4(be.x, be.y, tv, 0));
        }
        wi.mb_end = (int)mbins.size();
    }
    p->nmbins = (int)mbins.size();
    // chunks of the tensor-core interpolation: a work item's points are sorted by cell, so the
    // cells of one column (l0, l1) of its bin are consecutive; each column is cut into runs of
    // at most kTcChunkRows points
    std::vector<int4> chunks;
    std::vector<int> wi_chunk(wis.size() + 1, 0);
    for (size_t x = 0; x < wis.size(); ++x) {
        const int4 t = wis[x];
        wi_chunk[x] = (int)chunks.size();
        int cur_col = -1;
        for (int s2 = t.y; s2 < t.z; ++s2) {
            const int4 sg = segs[s2];
            const int l0 = ((sg.x >> 0) & 1023) - ((t.w >> 0) & 1023) * B;
            const int l1 = ((sg.x >> 10) & 1023) - ((t.w >> 10) & 1023) * B;
            const int col = l0 | (l1 << 8);
            int q = sg.y, left = sg.z;
            while (left > 0) {
                if (col != cur_col || chunks.back().y == kTcChunkRows) {
                    chunks.push_back(make_int4(q, 0, col, 0));
                    cur_col = col;
                }
                const int take = std::min(left, kTcChunkRows - chunks.back().y);
                chunks.back().y += take;
                q += take;
                left -= take;
            }
        }
    }
    wi_chunk[wis.size()] = (int)chunks.size();
    // point ranges of the packed FP32 spread's warps: each work item cut into kSpreadSplit
    // contiguous ranges of about equal estimated cost. A warp pays per point (its footprint's
    // multiply-adds, ~14 warp instructions), per batch of up to 32 points of one segment (the
    // batch's window weights and staging, ~170) and per segment piece (adding the footprint
    // into its tile, ~100), so a run of sparse cells costs more per point than a full cell; cut
    // at equal point counts, the slowest warp of a work item averaged ~12 % above the mean.
    std::vector<int> wsplit(wis.size() * (kSpreadSplit + 1));
    for (size_t x = 0; x < wis.size(); ++x) {
        const int4 t = wis[x];
        int *o = &wsplit[x * (kSpreadSplit + 1)];
        auto seg_cost = [](int sz) {
            return ANOVA_SPLIT_COST_POINT * sz + ANOVA_SPLIT_COST_BATCH * ((sz + 31) / 32) + ANOVA_SPLIT_COST_PIECE;
        };
        double total_cost = 0.0;
        for (int s2 = t.y; s2 < t.z; ++s2) total_cost += seg_cost(segs[s2].z);
        o[0] = segs[t.y].y;
        o[kSpreadSplit] = segs[t.z - 1].y + segs[t.z - 1].z;
        int k = 1;
        double acc = 0.0;
        for (int s2 = t.y; s2 < t.z && k < kSpreadSplit; ++s2) {
            const int sz = segs[s2].z;
            const double c = seg_cost(sz);
            while (k < kSpreadSplit && acc + c >= total_cost * k / kSpreadSplit) {
                const double f = (total_cost * k / kSpreadSplit - acc) / c;
                o[k] = segs[s2].y + (int)std::lround(std::min(1.0, std::max(0.0, f)) * sz);
                ++k;
            }
            acc += c;
        }
        for (; k < kSpreadSplit; ++k) o[k] = o[kSpreadSplit];
        for (k = 1; k <= kSpreadSplit; ++k) o[k] = std::max(o[k], o[k - 1]);
    }
    p->nseg = (int)segs.size();
    p->nwi = (int)wis.size();
    p->ntiles = (int)ftiles.size();

    // ------------------------------------------------------------------ table invariants
    // Every kernel index is derived from these tables; check them once here so that a table
    // that would send a kernel outside its buffers is reported instead of launched.
    {
        std::vector<int> hperm(total);
        ANOVA_CUDA_TRY(cudaMemcpyAsync(hperm.data(), p->perm, sizeof(int) * total, cudaMemcpyDeviceToHost, st));
        ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
        // windows checked on host threads: 1 = not a permutation, 2 = not sorted, 3 = window order
        std::vector<int> perr(P, 0);
        parallel_for_threads(P, 1, [&](int t, int nt) {
            std::vector<char> seen(n);
            for (int w = t; w < P; w += nt) {
                std::fill(seen.begin(), seen.end(), 0);
                for (long long q = (long long)w * n; q < (long long)(w + 1) * n; ++q) {
                    const int i = hperm[q];
                    if (i < 0 || i >= n || seen[i]) { perr[w] = 1; break; }
                    seen[i] = 1;
                    if (q > (long long)w * n && hkeys[q] < hkeys[q - 1]) { perr[w] = 2; break; }
                    if ((int)(hkeys[q] >> KB) != w) { perr[w] = 3; break; }
                }
            }
        });
        for (int e : perr) {
            if (e == 1) return fail(ANOVA_ERR_CUDA, "plan check: sort did not produce a permutation");
            if (e == 2) return fail(ANOVA_ERR_CUDA, "plan check: keys not sorted");
            if (e == 3) return fail(ANOVA_ERR_CUDA, "plan check: window order");
        }
        const int tw = B + 2 * m - 1;
        for (int w = 0; w < P; ++w) {
            const WindowInfo &wi = p->win[w];
            int npts = 0;
            for (int s2 = wi.seg_begin; s2 < wi.seg_end; ++s2) {
                const int4 sg = segs[s2];
                if (sg.w != w || sg.z < 1 || sg.z > kSegMax || sg.y < (long long)w * n ||
                    (long long)sg.y + sg.z > (long long)(w + 1) * n)
                    return fail(ANOVA_ERR_CUDA, "plan check: bad segment");
                npts += sg.z;
                for (int k = 0; k < 3; ++k) {
                    const int c = (sg.x >> (10 * k)) & 1023;
                    if (k < wi.dw ? (c - m + 1 < 0 || c + m > nos - 1) : c != 0)
                        return fail(ANOVA_ERR_INVALID_ARG, "plan check: footprint leaves the grid");
                }
            }
            if (npts != n) return fail(ANOVA_ERR_CUDA, "plan check: segments do not cover the points");
            for (int x = wi.wi_begin; x < wi.wi_end; ++x) {
                const int4 t = wis[x];
                if (t.x != w || t.y < wi.seg_begin || t.z > wi.seg_end || t.y >= t.z)
                    return fail(ANOVA_ERR_CUDA, "plan check: bad work item");
                int pts = 0;
                for (int s2 = t.y; s2 < t.z; ++s2) {
                    pts += segs[s2].z;
                    for (int k = 0; k < 3; ++k) {
                        const int c = (segs[s2].x >> (10 * k)) & 1023, b = (t.w >> (10 * k)) & 1023;
                        const int lc = c - b * B;
                        if (k < wi.dw ? (lc < 0 || lc >= B || b * B - m + 1 < 0 || b * B + B + m - 1 > nos - 1)
                                      : (c != 0 || b != 0))
                            return fail(ANOVA_ERR_CUDA, "plan check: segment outside its bin");
                    }
                }
                if (pts > p->wi_max) return fail(ANOVA_ERR_CUDA, "plan check: work item too large");
            }
            int nbins = 1;
            for (int k = 0; k < wi.dw; ++k) nbins *= NB;
            for (int b = 0; b < nbins; ++b) {
                const int2 be = bins[wi.bin_off + b];
                if (be.y == 0) continue;
                if (be.x < wi.wi_begin || be.x + be.y > wi.wi_end) return fail(ANOVA_ERR_CUDA, "plan check: bin table");
            }
            for (int k = 0; k < wi.dw; ++k)
                if (wi.box_lo[k] < 0 || wi.box_hi[k] > nos || wi.box_lo[k] >= wi.box_hi[k])
                    return fail(ANOVA_ERR_CUDA, "plan check: grid box");
            (void)tw;
        }
        for (size_t x = 0; x < wis.size(); ++x) {
            // a work item's chunks cover its points in order, each inside one column of its bin
            const int4 t = wis[x];
            long long q = segs[t.y].y;
            if (wi_chunk[x] > wi_chunk[x + 1]) return fail(ANOVA_ERR_CUDA, "plan check: chunk table");
            for (int c = wi_chunk[x]; c < wi_chunk[x + 1]; ++c) {
                const int4 ch = chunks[c];
                const int l0 = ch.z & 255, l1 = ch.z >> 8;
                if (ch.x != q || ch.y < 1 || ch.y > kTcChunkRows || l0 < 0 || l0 >= B || l1 < 0 || l1 >= B)
                    return fail(ANOVA_ERR_CUDA, "plan check: chunk table");
                q += ch.y;
            }
            if (q != (long long)segs[t.z - 1].y + segs[t.z - 1].z) return fail(ANOVA_ERR_CUDA, "plan check: chunk table");
            // the warps' ranges start and end with the item's points and do not decrease
            const int *o = &wsplit[x * (kSpreadSplit + 1)];
            if (o[0] != segs[t.y].y || o[kSpreadSplit] != segs[t.z - 1].y + segs[t.z - 1].z)
                return fail(ANOVA_ERR_CUDA, "plan check: spread split table");
            for (int k = 1; k <= kSpreadSplit; ++k)
                if (o[k] < o[k - 1]) return fail(ANOVA_ERR_CUDA, "plan check: spread split table");
        }
        for (const std::vector<int4> *tl : {&ftiles, &ftiles_full})
        for (const int4 &t : *tl) {
            const int ax = t.w & 255, lines = t.w >> 8;
            if (t.x < 0 || t.x >= P || t.y < 0 || t.y >= nos || t.z < 0 || lines < 1 || lines > p->conv_lines ||
                t.z + lines > nos || ax >= p->win[t.x].dw)
                return fail(ANOVA_ERR_CUDA, "plan check: FFT tile");
        }
    }

    // ------------------------------------------------------------------ upload tables
    std::vector<DevWindow> hdw(P);
    for (int w = 0; w < P; ++w) {
        const WindowInfo &wi = p->win[w];
        DevWindow &x = hdw[w];
        std::memset(&x, 0, sizeof(x));
        x.dw = wi.dw;
        for (int k = 0; k < 3; ++k) { x.box_lo[k] = wi.box_lo[k]; x.box_hi[k] = wi.box_hi[k]; }
        x.grid_off = wi.grid_off;
        x.bin_off = wi.bin_off;
    }
    auto upload = [&](void **dst, const void *src, size_t bytes) -> anova_status {
        if (bytes == 0) bytes = 16;
        cudaError_t e = cudaMalloc(dst, bytes);
        if (e != cudaSuccess) return fail(ANOVA_ERR_OOM, "device allocation failed");
        p->static_bytes += (int64_t)bytes;
        if (src) {
            e = cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
        }
        return ANOVA_OK;
    };
    anova_status s;
    if ((s = upload((void **)&p->segs, segs.data(), sizeof(int4) * segs.size())) != ANOVA_OK) return s;
    if ((s = upload((void **)&p->wis, wis.data(), sizeof(int4) * wis.size())) != ANOVA_OK) return s;
    if ((s = upload((void **)&p->chunks, chunks.data(), sizeof(int4) * chunks.size())) != ANOVA_OK) return s;
    if ((s = upload((void **)&p->wi_chunk, wi_chunk.data(), sizeof(int) * wi_chunk.size())) != ANOVA_OK) return s;
    if ((s = upload((void **)&p->wsplit, wsplit.data(), sizeof(int) * wsplit.size())) != ANOVA_OK) return s;
    {
        // each window's work items by decreasing point count (ties by index): persistent kernels
        // that take items in this order finish on the smallest ones
        std::vector<int> order(wis.size());
        for (int w = 0; w < P; ++w) {
            const int b0 = p->win[w].wi_begin, b1 = p->win[w].wi_end;
            std::vector<std::pair<int, int>> sz;
            sz.reserve(b1 - b0);
            for (int x = b0; x < b1; ++x) {
                int cnt = 0;
                for (int sgi = wis[x].y; sgi < wis[x].z; ++sgi) cnt += segs[sgi].z;
                sz.emplace_back(-cnt, x);
            }
            std::sort(sz.begin(), sz.end());
            for (int i = 0; i < b1 - b0; ++i) order[b0 + i] = sz[i].second;
        }
        if ((s = upload((void **)&p->wi_order, order.data(), sizeof(int) * order.size())) != ANOVA_OK) return s;
        // the same over each dimension group (launches that cover a whole group)
        for (const Group &gr : p->groups) {
            std::vector<std::pair<int, int>> sz;
            sz.reserve(gr.wi_end - gr.wi_begin);
            for (int x = gr.wi_begin; x < gr.wi_end; ++x) {
                int cnt = 0;
                for (int sgi = wis[x].y; sgi < wis[x].z; ++sgi) cnt += segs[sgi].z;
                sz.emplace_back(-cnt, x);
            }
            std::sort(sz.begin(), sz.end());
            for (int i = 0; i < gr.wi_end - gr.wi_begin; ++i) order[gr.wi_begin + i] = sz[i].second;
        }
        if ((s = upload((void **)&p->wi_gorder, order.data(), sizeof(int) * order.size())) != ANOVA_OK) return s;
    }
    if ((s = upload((void **)&p->bins, bins.data(), sizeof(int2) * bins.size())) != ANOVA_OK) return s;
    if ((s = upload((void **)&p->mbins, mbins.data(), sizeof(int4) * mbins.size())) != ANOVA_OK) return s;
    {
        // cell index inside its bin for every sorted point (the low digits of the sort key), from
        // the sorted keys still on the device
        if ((s = upload((void **)&p->cellloc, nullptr, (size_t)total)) != ANOVA_OK) return s;
        const int nb = (int)std::min<long long>((total + 255) / 256, 152LL * 32);
        k_cellloc<<<nb, 256, 0, st>>>(kin, total, KB, B, (const int *)ddws.p, p->cellloc);
        ANOVA_CUDA_TRY(cudaGetLastError());
    }
    if ((s = upload((void **)&p->ftiles, ftiles.data(), sizeof(int4) * ftiles.size())) != ANOVA_OK) return s;
    if ((s = upload((void **)&p->ftiles_full, ftiles_full.data(), sizeof(int4) * ftiles_full.size())) != ANOVA_OK)
        return s;
    if ((s = upload((void **)&p->dwin, hdw.data(), sizeof(DevWindow) * P)) != ANOVA_OK) return s;
    if ((s = upload((void **)&p->dev_status, nullptr, sizeof(int) * kStatusAlloc)) != ANOVA_OK) return s;
    ANOVA_CUDA_TRY(cudaMemsetAsync(p->dev_status, 0, sizeof(int) * kStatusAlloc, st));
    for (int k = 0; k < 3; ++k) {
        ANOVA_CUDA_TRY(cudaStreamCreateWithFlags(&p->aux[k], cudaStreamNonBlocking));
        ANOVA_CUDA_TRY(cudaEventCreateWithFlags(&p->join_evt[k], cudaEventDisableTiming));
    }
    ANOVA_CUDA_TRY(cudaEventCreateWithFlags(&p->fork_evt, cudaEventDisableTiming));
    ANOVA_CUDA_TRY(cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device));
    std::vector<float> f32;
    if (prec == ANOVA_FP64) {
        if ((s = upload(&p->D1br, d1br.data(), sizeof(double) * d1br.size())) != ANOVA_OK) return s;
        if ((s = upload(&p->tw, twid.data(), sizeof(double) * twid.size())) != ANOVA_OK) return s;
        ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
    } else {
        f32.assign(d1br.begin(), d1br.end());
        if ((s = upload(&p->D1br, f32.data(), sizeof(float) * f32.size())) != ANOVA_OK) return s;
        ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
        f32.assign(twid.begin(), twid.end());
        if ((s = upload(&p->tw, f32.data(), sizeof(float) * f32.size())) != ANOVA_OK) return s;
        ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
    }
    p->static_bytes += (int64_t)(es * 3 * total + sizeof(int) * total + sizeof(double) * 3 * total);
    ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
    *out = plan.release();
    return ANOVA_OK;
}

}  // namespace anova
