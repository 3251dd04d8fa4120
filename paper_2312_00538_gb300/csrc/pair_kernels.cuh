// FP64 plans' 3-D spread and interpolation with their multiply-adds in FP32 pairs (arXiv
// 2312.00538, Sec. 3: the same sums as k_spread and k_interp_direct; only the arithmetic differs).
#pragma once

#include "nfft_kernels.cuh"

namespace anova {

// ------------------------------------------------------------------ FP64 3-D spread in FP32 pairs
// The FP64 plans' 3-D spread with the footprint's multiply-adds on the FP32 pipe (GB300's FP64
// pipe runs at 1/64 of FP32, and the generic kernel keeps it ~80 % busy). A value is a pair
// (hi, lo) of FP32 numbers; a product of pairs keeps the exact error of hi * hi (fma) and the
// cross terms; sums carry the rounding error of every addition to hi exactly in lo (two-sum);
// all with explicitly rounded operations so that no contraction changes them. The window
// weights are evaluated in FP64 as in k_spread and stored as pairs; tiles are pairs in shared
// memory; the partial tile is written in FP64. Relative accuracy ~2^-44 of the sums of the terms'
// magnitudes. Same work split and shared-memory layout as k_spread (DW = 3). Cheaper than the
// renormalised pair type of pair_arith.cuh (used by the FFT passes): a product is left as
// (hi * hi, its error plus the cross terms) and only the accumulators' hi parts take the two-sum.
struct fpair {
    float hi, lo;
};
__device__ __forceinline__ fpair fpair_of(double d) {
    const float h = __double2float_rn(d);
    return {h, __double2float_rn(d - (double)h)};
}
__device__ __forceinline__ fpair fpair_mul(fpair a, fpair b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return {p, e};
}
// acc += x (x not normalised: |x.lo| small against |x.hi|)
__device__ __forceinline__ void fpair_acc(fpair &acc, fpair x) {
    const float t = __fadd_rn(acc.hi, x.hi);
    const float bp = __fsub_rn(t, acc.hi);
    const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(t, bp)), __fsub_rn(x.hi, bp));
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(err, x.lo));
    acc.hi = t;
}

template <int M, int B, int NWARP>
__global__ void __launch_bounds__(NWARP * 32) k_spread3_pair(SpreadArgs a) {
    pdl_wait();
    pdl_trigger();
    using C = SpreadCfg<double, 3, M, B, NWARP>;
    using G = typename C::G;
    constexpr int W2 = G::W2, RPL = G::RPL, WS = G::WS, PS = G::PSTRIDE, TW = C::TW;
    constexpr int RCH = RPL < 2 ? RPL : 2;
    constexpr int PD = PolyDegOf<double>::D;
    static_assert(sizeof(fpair) == sizeof(double), "pairs take the FP64 layout's slots");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    fpair *tiles_s = reinterpret_cast<fpair *>(smem_raw);
    fpair *wts_s = tiles_s + NWARP * C::TVP;
    double *coef_s = reinterpret_cast<double *>(wts_s + NWARP * 32 * PS);

    const int wi_idx = a.wi_begin + blockIdx.x;
    if (wi_idx >= a.wi_end) return;
    const int r = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int4 wi = a.wis[wi_idx];
    const int bin[3] = {cell_coord(wi.w, 0), cell_coord(wi.w, 1), cell_coord(wi.w, 2)};

    for (int i = threadIdx.x; i < NWARP * C::TVP; i += NWARP * 32) tiles_s[i] = {0.0f, 0.0f};
    for (int i = threadIdx.x; i < M * (PD + 1); i += NWARP * 32)
        coef_s[(i / (PD + 1)) * C::CS + i % (PD + 1)] = window_coef<double>(a.wp, i / (PD + 1), i % (PD + 1));
    __syncthreads();

    const int4 s_first = a.segs[wi.y];
    const int4 s_last = a.segs[wi.z - 1];
    const int p0 = s_first.y, p1 = s_last.y + s_last.z;
    const int len = p1 - p0;
    const int pw0 = p0 + (int)(((long long)len * warp) / NWARP);
    const int pw1 = p0 + (int)(((long long)len * (warp + 1)) / NWARP);

    const double *frac = reinterpret_cast<const double *>(a.frac);
    const double *vr = reinterpret_cast<const double *>(a.v) + (size_t)r * a.n;
    fpair *tile = tiles_s + warp * C::TVP;
    fpair *wts = wts_s + warp * 32 * PS;

    // rows owned by this lane: row = lane + 32 t, (ra, rb) = (row / W2, row % W2); rows past the
    // footprint are clamped (their products are computed and dropped)
    int ra[RPL], rb[RPL];
    bool rvalid[RPL];
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
        const int row = lane + 32 * t;
        rvalid[t] = row < G::ROWS;
        ra[t] = min(row / W2, W2 - 1);
        rb[t] = row % W2;
    }

    if (pw0 < pw1) {
        int lo = wi.y, hi = wi.z - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.segs[mid].y <= pw0) lo = mid; else hi = mid - 1;
        }
        for (int s = lo; s < wi.z; ++s) {
            const int4 sg = a.segs[s];
            if (sg.y >= pw1) break;
            const int q0 = max(sg.y, pw0), q1 = min(sg.y + sg.z, pw1);
            if (q0 >= q1) continue;
            int lc[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) lc[k] = cell_coord(sg.x, k) - bin[k] * B;
            for (int qb = q0; qb < q1; qb += 32) {
                const int cnt = min(32, q1 - qb);
                // the batch's weights in FP64 (one (point, axis, pair of offsets) per lane and
                // round), stored as pairs
                for (int t = lane; t < cnt * 3 * M; t += 32) {
                    const int pl = t / (3 * M);
                    const int rem = t - pl * (3 * M);
                    const int k = rem / M, j = rem - k * M;
                    const int q = qb + pl;
                    double wlo, whi;
                    window_pair<double, PD>(frac[(size_t)k * a.total + q], coef_s + j * C::CS, wlo, whi);
                    if (k == 2) {
                        const double vv = vr[a.perm[q]];
                        wlo *= vv;
                        whi *= vv;
                    }
                    wts[pl * PS + k * WS + j] = fpair_of(wlo);
                    wts[pl * PS + k * WS + W2 - 1 - j] = fpair_of(whi);
                }
                __syncwarp();
#pragma unroll
                for (int t0 = 0; t0 < RPL; t0 += RCH) {
                    fpair acc[RCH][W2];
#pragma unroll
                    for (int tt = 0; tt < RCH; ++tt)
#pragma unroll
                        for (int c = 0; c < W2; ++c) acc[tt][c] = {0.0f, 0.0f};
                    for (int j = 0; j < cnt; ++j) {
                        const fpair *pw = wts + j * PS;
                        fpair wz[W2];
#pragma unroll
                        for (int c = 0; c < W2; c += 2) {
                            const float4 q4 = *reinterpret_cast<const float4 *>(pw + 2 * WS + c);
                            wz[c] = {q4.x, q4.y};
                            wz[c + 1] = {q4.z, q4.w};
                        }
#pragma unroll
                        for (int tt = 0; tt < RCH; ++tt) {
                            const int t = t0 + tt;
                            if (t < RPL) {
                                const fpair rw = fpair_mul(pw[ra[t]], pw[WS + rb[t]]);
#pragma unroll
                                for (int c = 0; c < W2; ++c) fpair_acc(acc[tt][c], fpair_mul(rw, wz[c]));
                            }
                        }
                    }
#pragma unroll
                    for (int tt = 0; tt < RCH; ++tt) {
                        const int t = t0 + tt;
                        if (t < RPL && rvalid[t]) {
                            fpair *dst = tile + ((lc[0] + ra[t]) * TW + (lc[1] + rb[t])) * TW + lc[2];
#pragma unroll
                            for (int c = 0; c < W2; ++c) {
                                fpair v = dst[c];
                                fpair_acc(v, acc[tt][c]);
                                dst[c] = v;
                            }
                        }
                    }
                }
                __syncwarp();
            }
        }
    }
    __syncthreads();
    double *out = reinterpret_cast<double *>(a.tiles) + ((size_t)wi_idx * a.nrhs + r) * C::TV;
    for (int i = threadIdx.x; i < C::TV; i += NWARP * 32) {
        fpair sum = tiles_s[i];
#pragma unroll
        for (int w = 1; w < NWARP; ++w) fpair_acc(sum, tiles_s[w * C::TVP + i]);
        out[i] = (double)sum.hi + (double)sum.lo;
    }
}

// ------------------------------------------------------------------ FP64 3-D interpolation in FP32 pairs
// k_interp_direct for the FP64 plans' 3-D windows with the multiply-adds on the FP32 pipe: the
// convolved grid's box is first converted to pairs (hi = fl32(g), lo = fl32(g - hi)) in a free
// workspace buffer, then every point's (2M)^3 block is summed as in k_interp_direct, the weights
// evaluated in FP64 and split into pairs. Same pair arithmetic as k_spread3_pair.
struct GridPairArgs {
    const double *grid;
    fpair *pairs;                 // same layout as grid
    const DevWindow *dwin;
    long long grid_stride;
    long long box_cum[kMaxWindows + 1];  // cumulative box volumes of windows w_begin..
    int w_begin, w_end, n_os;
};

template <int DW>
__global__ void __launch_bounds__(256) k_grid_pairs(GridPairArgs a) {
    static_assert(DW == 3, "3-D windows");
    pdl_wait();
    pdl_trigger();
    const int r = blockIdx.y;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int nw = a.w_end - a.w_begin;
    if (idx >= a.box_cum[nw]) return;
    int wl = 0;
    while (idx >= a.box_cum[wl + 1]) ++wl;
    const DevWindow dw = a.dwin[a.w_begin + wl];
    long long loc = idx - a.box_cum[wl];
    int u[3];
    for (int k = 2; k >= 0; --k) {
        const int ext = dw.box_hi[k] - dw.box_lo[k];
        u[k] = dw.box_lo[k] + (int)(loc % ext);
        loc /= ext;
    }
    const size_t g = (size_t)r * a.grid_stride + dw.grid_off + ((size_t)u[0] * a.n_os + u[1]) * a.n_os + u[2];
    a.pairs[g] = fpair_of(a.grid[g]);
}

template <int M>
__global__ void __launch_bounds__(128) k_interp_pair(InterpDirectArgs<double> a, const fpair *__restrict__ pairs) {
    pdl_wait();
    pdl_trigger();
    constexpr int W2 = 2 * M;
    const int r = blockIdx.y;
    const long long q = a.q_begin + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= a.q_end) return;
    int lo = a.seg_begin, hi = a.seg_end - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.segs[mid].y <= q) lo = mid; else hi = mid - 1;
    }
    const int4 sg = a.segs[lo];
    const int w = sg.w;
    const DevWindow dw = a.dwin[w];
    const fpair *grid = pairs + (size_t)r * a.grid_stride_rhs + dw.grid_off;
    int c0[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) c0[k] = cell_coord(sg.x, k) - M + 1;
    fpair wt[3][W2];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double wd[W2];
        Weights<double, M>::eval(a.frac[(size_t)k * a.total + q], a.wp, wd);
#pragma unroll
        for (int c = 0; c < W2; ++c) wt[k][c] = fpair_of(wd[c]);
    }
    fpair f = {0.0f, 0.0f};
    const long long n2 = (long long)a.n_os * a.n_os;
#pragma unroll 1
    for (int aa = 0; aa < W2; ++aa) {
        fpair sa = {0.0f, 0.0f};
        for (int bb = 0; bb < W2; ++bb) {
            const float2 *row = reinterpret_cast<const float2 *>(grid + (long long)(c0[0] + aa) * n2 +
                                                                 (long long)(c0[1] + bb) * a.n_os + c0[2]);
            fpair sb = {0.0f, 0.0f};
#pragma unroll
            for (int cc = 0; cc < W2; ++cc) {
                const float2 gv = __ldg(row + cc);
                fpair_acc(sb, fpair_mul({gv.x, gv.y}, wt[2][cc]));
            }
            fpair wyb = wt[1][0];
#pragma unroll
            for (int k = 1; k < W2; ++k)
                if (k == bb) wyb = wt[1][k];
            fpair_acc(sa, fpair_mul(wyb, sb));
        }
        fpair wxa = wt[0][0];
#pragma unroll
        for (int k = 1; k < W2; ++k)
            if (k == aa) wxa = wt[0][k];
        fpair_acc(f, fpair_mul(wxa, sa));
    }
    a.part[((size_t)(w - a.part_w0) * a.nrhs + r) * a.n + a.perm[q]] = (double)f.hi + (double)f.lo;
}

}  // namespace anova
