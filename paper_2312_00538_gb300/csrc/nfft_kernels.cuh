// Spread (adjoint-NFFT step), tile reduction, gather interpolation (NFFT step) and window sum
// of the ANOVA fast summation (arXiv 2312.00538, Sec. 3: inner sum over i, outer sum over J).
//
// Points of every window are sorted by cell, cells grouped into bins of B^d cells. A spread
// work item is a run of one bin's cells (at most the plan's work-item cap of points, 2048 by
// default). Each warp of the work item's CTA accumulates a contiguous share of its points cell by
// cell: lanes own rows of the (2M)^d footprint of
// the current cell in registers, the window weights of 32 points at a time are staged in shared
// memory and broadcast, and the footprint is added into the warp's own tile of the bin
// neighbourhood ((B + 2M - 1)^d cells) -- no atomics anywhere. The CTA then sums its warp
// tiles and writes one partial tile per work item; the bin reduction adds the partial tiles of
// each bin, and the grid gather the (at most 3^d) bin tiles covering each grid point, both in a
// fixed order, so the grid is bit-for-bit reproducible.
#pragma once

#include <type_traits>

#include "kernels_common.cuh"
#include "tcgen05.cuh"

#ifndef ANOVA_TC_INTERP_MINB
#define ANOVA_TC_INTERP_MINB 4  // resident CTAs per SM the tensor-core interpolation is compiled for
#endif
#ifndef ANOVA_SPREAD_MINB
#define ANOVA_SPREAD_MINB 3  // resident CTAs per SM the packed FP32 spread is compiled for
#endif
#ifndef ANOVA_EPI_PAIR
#define ANOVA_EPI_PAIR 1  // tensor-core interpolation: b-sums of the epilogue with paired FMAs
#endif
#ifndef ANOVA_SPREAD_UNROLL
#define ANOVA_SPREAD_UNROLL 8  // points per unrolled group of the packed FP32 spread's inner loop
#endif

namespace anova {

struct SpreadArgs {
    int packed;             // FP32 3-D windows, m = 2 or 4: the packed kernel may be used
    const int4 *wis;        // {window, seg_begin, seg_end, bin packed}
    const int4 *segs;       // {cell packed, sorted start, count, window}
    const void *frac;       // T[3][total]
    const int *perm;        // [total]
    const void *v;          // T[nrhs][n]
    void *tiles;            // T[nwi][nrhs][TV]
    long long n, total;
    int nrhs, wi_begin, wi_end;
    WinParams wp;
    const int *order;       // packed kernel: CTA k takes work item order[wi_begin + k] (null: identity)
    const int *wsplit = nullptr;  // packed kernel: per work item, wsplit_n + 1 bounds of its warps'
    int wsplit_n = 0;             // sorted-point ranges (null or a different warp count: equal points)
};

template <typename T, int DW, int M, int B, int NWARP>
struct SpreadCfg {
    using G = Geo<DW, M>;
    static constexpr int TW = B + 2 * M - 1;
    static constexpr int TV = ipow(TW, DW);
    static constexpr int TVP = (TV + 3) / 4 * 4;
    static constexpr int CS = 16;  // coefficients per window pair in shared memory (>= degree + 1)
    // warp tiles, staged weights, window coefficients
    static constexpr size_t smem =
        sizeof(T) * ((size_t)NWARP * TVP + (size_t)NWARP * 32 * G::PSTRIDE + (size_t)M * CS);
};

template <typename T, int DW, int M, int B, int NWARP>
__global__ void __launch_bounds__(NWARP * 32) k_spread(SpreadArgs a) {
    pdl_wait();
    pdl_trigger();
    using C = SpreadCfg<T, DW, M, B, NWARP>;
    using G = typename C::G;
    constexpr int W2 = G::W2, RPL = G::RPL, WS = G::WS, PS = G::PSTRIDE, TW = C::TW;
    constexpr int RCH = RPL < 2 ? RPL : 2;  // rows per lane held in registers at once
    constexpr int PD = PolyDegOf<T>::D;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *tiles_s = reinterpret_cast<T *>(smem_raw);
    T *wts_s = tiles_s + NWARP * C::TVP;
    T *coef_s = wts_s + NWARP * 32 * PS;

    const int wi_idx = a.wi_begin + blockIdx.x;
    if (wi_idx >= a.wi_end) return;
    const int r = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int4 wi = a.wis[wi_idx];
    const int bin_packed = wi.w;
    int bin[3] = {cell_coord(bin_packed, 0), cell_coord(bin_packed, 1), cell_coord(bin_packed, 2)};

    for (int i = threadIdx.x; i < NWARP * C::TVP; i += NWARP * 32) tiles_s[i] = T(0);
    for (int i = threadIdx.x; i < M * (PD + 1); i += NWARP * 32)
        coef_s[(i / (PD + 1)) * C::CS + i % (PD + 1)] = window_coef<T>(a.wp, i / (PD + 1), i % (PD + 1));
    __syncthreads();

    const int4 s_first = a.segs[wi.y];
    const int4 s_last = a.segs[wi.z - 1];
    const int p0 = s_first.y, p1 = s_last.y + s_last.z;
    const int len = p1 - p0;
    const int pw0 = p0 + (int)(((long long)len * warp) / NWARP);
    const int pw1 = p0 + (int)(((long long)len * (warp + 1)) / NWARP);

    const T *frac = reinterpret_cast<const T *>(a.frac);
    const T *vr = reinterpret_cast<const T *>(a.v) + (size_t)r * a.n;
    T *tile = tiles_s + warp * C::TVP;
    T *wts = wts_s + warp * 32 * PS;

    // rows owned by this lane: row = lane + 32 t; DW=3: (ra, rb) = (row / W2, row % W2)
    int ra[RPL], rb[RPL];
    bool rvalid[RPL];
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
        const int row = lane + 32 * t;
        rvalid[t] = row < G::ROWS;
        // indices of rows past the footprint are clamped so that their (discarded) products
        // only read this point's staged weights
        ra[t] = min(DW == 3 ? row / W2 : row, W2 - 1);
        rb[t] = DW == 3 ? row % W2 : 0;
    }

    if (pw0 < pw1) {
        // first segment overlapping [pw0, pw1): binary search on the sorted starts
        int lo = wi.y, hi = wi.z - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.segs[mid].y <= pw0) lo = mid; else hi = mid - 1;
        }
        if constexpr (DW == 3) {
            for (int s = lo; s < wi.z; ++s) {
                const int4 sg = a.segs[s];
                if (sg.y >= pw1) break;
                const int q0 = max(sg.y, pw0), q1 = min(sg.y + sg.z, pw1);
                if (q0 >= q1) continue;
                int lc[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) lc[k] = cell_coord(sg.x, k) - bin[k] * B;  // in [0, B)
                for (int qb = q0; qb < q1; qb += 32) {
                    const int cnt = min(32, q1 - qb);
                    // the batch's weights, one (point, axis, pair of offsets) per lane and round: a
                    // batch of few points (sparse cells) still keeps the warp's lanes busy
                    for (int t = lane; t < cnt * DW * M; t += 32) {
                        const int pl = t / (DW * M);
                        const int rem = t - pl * (DW * M);
                        const int k = rem / M, j = rem - k * M;
                        const int q = qb + pl;
                        T lo, hi;
                        window_pair<T, PD>(frac[(size_t)k * a.total + q], coef_s + j * C::CS, lo, hi);
                        if (k == DW - 1) {
                            const T vv = vr[a.perm[q]];
                            lo *= vv;
                            hi *= vv;
                        }
                        wts[pl * PS + k * WS + j] = lo;
                        wts[pl * PS + k * WS + W2 - 1 - j] = hi;
                    }
                    __syncwarp();
                    if (cnt == 1) {
                        // a lone point (sparse cells, typical of FP64 plans): its products go
                        // straight into the tile, one multiply-add per value instead of a product
                        // and a separate add
                        const T *pw = wts;
                        T wz[W2];
                        lds_vec<T, W2>(pw + (DW - 1) * WS, wz);
#pragma unroll
                        for (int t = 0; t < RPL; ++t) {
                            if (!rvalid[t]) continue;
                            const T rw = pw[ra[t]] * pw[WS + rb[t]];
                            T *dst = tile + ((lc[0] + ra[t]) * TW + (lc[1] + rb[t])) * TW + lc[2];
#pragma unroll
                            for (int c = 0; c < W2; ++c) dst[c] = fma(rw, wz[c], dst[c]);
                        }
                        __syncwarp();
                        continue;
                    }
#pragma unroll
                    for (int t0 = 0; t0 < RPL; t0 += RCH) {
                        T acc[RCH][W2];
#pragma unroll
                        for (int tt = 0; tt < RCH; ++tt)
#pragma unroll
                            for (int c = 0; c < W2; ++c) acc[tt][c] = T(0);
                        for (int j = 0; j < cnt; ++j) {
                            const T *pw = wts + j * PS;
                            T wz[W2];
                            lds_vec<T, W2>(pw + (DW - 1) * WS, wz);
#pragma unroll
                            for (int tt = 0; tt < RCH; ++tt) {
                                const int t = t0 + tt;
                                if (t < RPL) {
                                    T rw;
                                    if (DW == 3) rw = pw[ra[t]] * pw[WS + rb[t]];
                                    else if (DW == 2) rw = pw[ra[t]];
                                    else rw = T(1);
#pragma unroll
                                    for (int c = 0; c < W2; ++c) acc[tt][c] = fma(rw, wz[c], acc[tt][c]);
                                }
                            }
                        }
#pragma unroll
                        for (int tt = 0; tt < RCH; ++tt) {
                            const int t = t0 + tt;
                            if (t < RPL && rvalid[t]) {
                                int base;
                                if (DW == 3) base = ((lc[0] + ra[t]) * TW + (lc[1] + rb[t])) * TW + lc[2];
                                else if (DW == 2) base = (lc[0] + ra[t]) * TW + lc[1];
                                else base = lc[0];
#pragma unroll
                                for (int c = 0; c < W2; ++c) tile[base + c] += acc[tt][c];
                            }
                        }
                    }
                    __syncwarp();
                }
            }
        } else {
            // 1-D and 2-D footprints: a lane owns one footprint row (2-D: row a, 1-D: the single
            // row) for every PPS-th point of the batch; the PPS point slots keep their sums over
            // the cell's batches and are folded in a fixed order when the cell ends
            constexpr int LR = DW == 2 ? W2 : 1;  // lanes per point
            constexpr int PPS = 32 / LR;          // point slots per warp
            const int slot = lane / LR, row = lane % LR;
            const bool lane_ok = slot < PPS;
            for (int s = lo; s < wi.z; ++s) {
                const int4 sg = a.segs[s];
                if (sg.y >= pw1) break;
                const int q0 = max(sg.y, pw0), q1 = min(sg.y + sg.z, pw1);
                if (q0 >= q1) continue;
                int lc[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) lc[k] = cell_coord(sg.x, k) - bin[k] * B;  // in [0, B)
                T acc[W2];
#pragma unroll
                for (int c = 0; c < W2; ++c) acc[c] = T(0);
                for (int qb = q0; qb < q1; qb += 32) {
                    const int cnt = min(32, q1 - qb);
                    for (int t = lane; t < cnt * DW * M; t += 32) {
                        const int pl = t / (DW * M);
                        const int rem = t - pl * (DW * M);
                        const int k = rem / M, j = rem - k * M;
                        const int q = qb + pl;
                        T lo_w, hi_w;
                        window_pair<T, PD>(frac[(size_t)k * a.total + q], coef_s + j * C::CS, lo_w, hi_w);
                        if (k == DW - 1) {
                            const T vv = vr[a.perm[q]];
                            lo_w *= vv;
                            hi_w *= vv;
                        }
                        wts[pl * PS + k * WS + j] = lo_w;
                        wts[pl * PS + k * WS + W2 - 1 - j] = hi_w;
                    }
                    __syncwarp();
                    if (lane_ok)
                        for (int jp = slot; jp < cnt; jp += PPS) {
                            const T *pw = wts + jp * PS;
                            const T rw = DW == 2 ? pw[row] : T(1);
                            T wz[W2];
                            lds_vec<T, W2>(pw + (DW - 1) * WS, wz);
#pragma unroll
                            for (int c = 0; c < W2; ++c) acc[c] = fma(rw, wz[c], acc[c]);
                        }
                    __syncwarp();
                }
                // tree fold of the slots into slot 0 (lanes past the slots hold zeros)
#pragma unroll
                for (int k = 1; k < PPS; k <<= 1) {
#pragma unroll
                    for (int c = 0; c < W2; ++c) {
                        const T other = __shfl_down_sync(0xffffffffu, acc[c], k * LR);
                        if (lane_ok && slot % (2 * k) == 0 && slot + k < PPS) acc[c] += other;
                    }
                }
                if (slot == 0) {
                    const int base = DW == 2 ? (lc[0] + row) * TW + lc[1] : lc[0];
#pragma unroll
                    for (int c = 0; c < W2; ++c) tile[base + c] += acc[c];
                }
                __syncwarp();
            }
        }
    }
    __syncthreads();
    T *out = reinterpret_cast<T *>(a.tiles) + ((size_t)wi_idx * a.nrhs + r) * C::TV;
    for (int i = threadIdx.x; i < C::TV; i += NWARP * 32) {
        T s = T(0);
#pragma unroll
        for (int w = 0; w < NWARP; ++w) s += tiles_s[w * C::TVP + i];
        out[i] = s;
    }
}

// ------------------------------------------------------------------ FP32 3-D spread, packed
// Specialisation of k_spread for FP32 3-D windows whose footprint edge 2M divides 16 (M = 2, 4):
// LPP lanes share a point (32, the default: the warp takes one point per step; 16: two points per
// step), each lane holding (2M)^2 / LPP rows (a, b) of the footprint, 2M values each, as f32x2
// pairs along c for fma.rn.f32x2. The staged weights are laid out so that every load is a
// 32- to 128-bit broadcast: X permuted so that a lane's rows are contiguous, Y and Z (times v)
// in order.
template <int M, int B, int NWARP, int LPP = 16>
struct SpreadX2Cfg {
    static constexpr int W2 = 2 * M;
    static constexpr int RPL = W2 * W2 / LPP;        // rows per lane (LPP lanes share a point)
    static constexpr int S = LPP / W2;               // a-stride between a lane's rows
    static constexpr int TW = B + W2 - 1;
    static constexpr int TV = TW * TW * TW;
    static constexpr int TVP = (TV + 3) / 4 * 4;
    static constexpr int XO = 0, YO = W2, ZO = 2 * W2, PS = 3 * W2;      // staged floats per point
    static constexpr int SEG_CACHE = 128;                               // segments kept in shared memory
    // warp tiles, staged weights, the item's segments
    static constexpr size_t smem = sizeof(float) * ((size_t)NWARP * TVP + (size_t)NWARP * 32 * PS) + 16 * SEG_CACHE;
};

template <int M, int B, int NWARP, int LPP>
__global__ void __launch_bounds__(NWARP * 32, ANOVA_SPREAD_MINB) k_spread3_x2(SpreadArgs a) {
    pdl_wait();
    pdl_trigger();
    using C = SpreadX2Cfg<M, B, NWARP, LPP>;
    constexpr int W2 = C::W2, RPL = C::RPL, S = C::S, TW = C::TW, PS = C::PS;
    constexpr int PPS = 32 / LPP;  // points per warp step
    constexpr int SPREAD_UNROLL = ANOVA_SPREAD_UNROLL / PPS > 0 ? ANOVA_SPREAD_UNROLL / PPS : 1;
    static_assert(32 % (PPS * SPREAD_UNROLL) == 0, "unrolled steps stay inside the staged batch");
    static_assert(LPP % W2 == 0 && RPL * LPP == W2 * W2, "2M must divide the lanes per point");
    static_assert(W2 % 4 == 0, "vector staging layout");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *tiles_s = reinterpret_cast<float *>(smem_raw);
    float *wts_s = tiles_s + NWARP * C::TVP;

    if (a.wi_begin + (int)blockIdx.x >= a.wi_end) return;
    const int wi_idx = a.order ? a.order[a.wi_begin + blockIdx.x] : a.wi_begin + blockIdx.x;
    const int r = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int half = lane / LPP, lh = lane % LPP;
    const int4 wi = a.wis[wi_idx];
    const int bin[3] = {cell_coord(wi.w, 0), cell_coord(wi.w, 1), cell_coord(wi.w, 2)};

    for (int i = threadIdx.x; i < NWARP * C::TVP; i += NWARP * 32) tiles_s[i] = 0.0f;
    // the item's segments in shared memory (each warp searches them for its first point and
    // walks them in order)
    int4 *segs_s = reinterpret_cast<int4 *>(wts_s + NWARP * 32 * PS);
    const bool seg_cached = wi.z - wi.y <= C::SEG_CACHE;
    if (seg_cached)
        for (int i = threadIdx.x; i < wi.z - wi.y; i += NWARP * 32) segs_s[i] = a.segs[wi.y + i];
    __syncthreads();
    auto seg_at = [&](int i) -> int4 { return seg_cached ? segs_s[i - wi.y] : a.segs[i]; };

    // each warp takes a contiguous share of the item's points, of about equal cost by the plan's
    // split table (else of equal size); a cell may be split between two warps, each adds its
    // part into its own tile
    int pw0, pw1;
    if (a.wsplit && a.wsplit_n == NWARP) {
        pw0 = a.wsplit[(size_t)wi_idx * (NWARP + 1) + warp];
        pw1 = a.wsplit[(size_t)wi_idx * (NWARP + 1) + warp + 1];
    } else {
        const int4 s_first = seg_at(wi.y);
        const int4 s_last = seg_at(wi.z - 1);
        const int p0 = s_first.y, p1 = s_last.y + s_last.z;
        const int len = p1 - p0;
        pw0 = p0 + (int)(((long long)len * warp) / NWARP);
        pw1 = p0 + (int)(((long long)len * (warp + 1)) / NWARP);
    }

    const float *fr0 = reinterpret_cast<const float *>(a.frac);
    const float *fr1 = fr0 + a.total, *fr2 = fr0 + 2 * a.total;
    // v is read through the permutation: the permutation streams in sorted order and v (4 bytes
    // per point) stays in L2, so no sorted copy of v is written first
    const float *vr = reinterpret_cast<const float *>(a.v) + (size_t)r * a.n;
    auto vsorted_at = [&](int q) { return vr[a.perm[q]]; };
    float *tile = tiles_s + warp * C::TVP;
    float *wts = wts_s + warp * 32 * PS;
    const int g = lh / W2;           // this lane's rows: a = g + S k, b = lh % W2
    const int rb = lh % W2;

    if (pw0 < pw1) {
        int s;
        {
            int lo = wi.y, hi = wi.z - 1;  // last segment starting at or before pw0
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (seg_at(mid).y <= pw0) lo = mid; else hi = mid - 1;
            }
            s = lo;
        }
        int4 sg = seg_at(s);
        int4 sg_next = (s + 1 < wi.z) ? seg_at(s + 1) : sg;
        int q = pw0;
        int send = min(sg.y + sg.z, pw1);
        int cnt = min(32, send - q);
        // per-point inputs of the current batch (prefetched one batch ahead)
        float fx = 0.f, fy = 0.f, fz = 0.f, vv = 0.f;
        if (lane < cnt) {
            fx = fr0[q + lane];
            fy = fr1[q + lane];
            fz = fr2[q + lane];
            vv = vsorted_at(q + lane);
        }
        f32x2 acc[RPL][W2 / 2];
#pragma unroll
        for (int k = 0; k < RPL; ++k)
#pragma unroll
            for (int c = 0; c < W2 / 2; ++c) acc[k][c] = zero2();
        while (true) {
            // next batch: same piece, or the first batch of the next segment in range
            const int qn = q + cnt;
            bool newpiece = false, done = false;
            int sn = s, sendn = send;
            int4 sgn = sg;
            if (qn >= send) {
                newpiece = true;
                if (qn < pw1 && s + 1 < wi.z) {
                    sn = s + 1;
                    sgn = sg_next;
                    sendn = min(sgn.y + sgn.z, pw1);
                } else {
                    done = true;
                }
            }
            const int cntn = done ? 0 : min(32, sendn - qn);
            float nfx = 0.f, nfy = 0.f, nfz = 0.f, nvv = 0.f;
            if (lane < cntn) {
                nfx = fr0[qn + lane];
                nfy = fr1[qn + lane];
                nfz = fr2[qn + lane];
                nvv = vsorted_at(qn + lane);
            }
            int4 sg_next2 = sg_next;
            if (newpiece && !done && sn + 1 < wi.z) sg_next2 = seg_at(sn + 1);
            // stage the current batch's weights (zeros for lanes past the batch)
            {
                float wx[W2], wy[W2], wz[W2];
                Weights<float, M>::eval(fx, a.wp, wx);
                Weights<float, M>::eval(fy, a.wp, wy);
                Weights<float, M>::eval(fz, a.wp, wz);
                const float vl = lane < cnt ? vv : 0.0f;
#pragma unroll
                for (int j = 0; j < W2; ++j) wz[j] *= vl;
                float4 *dst = reinterpret_cast<float4 *>(wts + lane * PS);
                // X at permuted positions a -> (a % S) * RPL + a / S, so a lane's rows are adjacent
#pragma unroll
                for (int pos = 0; pos < W2; pos += 4) {
                    float xv[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) xv[t] = wx[((pos + t) % RPL) * S + (pos + t) / RPL];
                    dst[(C::XO + pos) / 4] = make_float4(xv[0], xv[1], xv[2], xv[3]);
                }
#pragma unroll
                for (int b = 0; b < W2; b += 4) dst[(C::YO + b) / 4] = make_float4(wy[b], wy[b + 1], wy[b + 2], wy[b + 3]);
#pragma unroll
                for (int c = 0; c < W2; c += 4) dst[(C::ZO + c) / 4] = make_float4(wz[c], wz[c + 1], wz[c + 2], wz[c + 3]);
            }
            __syncwarp();
            // steps in groups of SPREAD_UNROLL: lanes past the batch staged zero Z weights, so
            // the padded steps add zeros and the unrolled group needs no remainder loop
            const int nstep = (cnt + PPS - 1) / PPS;
            for (int j0 = 0; j0 < nstep; j0 += SPREAD_UNROLL)
#pragma unroll
            for (int ju = 0; ju < SPREAD_UNROLL; ++ju) {
                const int jj = j0 + ju;
                const float *pw = wts + (PPS * jj + half) * PS;
                float xr[RPL];
                f32x2 z2[W2 / 2];
                const float yb = pw[C::YO + rb];
                if constexpr (RPL % 4 == 0) {
#pragma unroll
                    for (int k = 0; k < RPL; k += 4) {
                        const float4 t = *reinterpret_cast<const float4 *>(pw + C::XO + g * RPL + k);
                        xr[k] = t.x;
                        xr[k + 1] = t.y;
                        xr[k + 2] = t.z;
                        xr[k + 3] = t.w;
                    }
                } else if constexpr (RPL == 2) {
                    const float2 t = *reinterpret_cast<const float2 *>(pw + C::XO + g * RPL);
                    xr[0] = t.x;
                    xr[1] = t.y;
                } else {
#pragma unroll
                    for (int k = 0; k < RPL; ++k) xr[k] = pw[C::XO + g * RPL + k];
                }
#pragma unroll
                for (int c = 0; c < W2 / 2; c += 2) lds_pairs(pw + C::ZO + 2 * c, z2[c], z2[c + 1]);
#pragma unroll
                for (int k = 0; k < RPL; ++k) {
                    const float rs = xr[k] * yb;
                    const f32x2 rw = make_float2(rs, rs);
#pragma unroll
                    for (int c = 0; c < W2 / 2; ++c) acc[k][c] = fma2(rw, z2[c], acc[k][c]);
                }
            }
            __syncwarp();
            if (newpiece) {
                // the two half-warps hold the same rows: fold the upper half into the lower,
                // which adds the cell's footprint into the warp's tile
                int lc[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) lc[k] = cell_coord(sg.x, k) - bin[k] * B;
                if constexpr (PPS == 2) {
#pragma unroll
                    for (int k = 0; k < RPL; ++k)
#pragma unroll
                        for (int c = 0; c < W2 / 2; ++c) {
                            f32x2 o;
                            o.x = __shfl_down_sync(0xffffffffu, acc[k][c].x, 16);
                            o.y = __shfl_down_sync(0xffffffffu, acc[k][c].y, 16);
                            acc[k][c] = add2(acc[k][c], o);
                        }
                }
                if (half == 0) {
#pragma unroll
                    for (int k = 0; k < RPL; ++k) {
                        const int ra = g + S * k;
                        float *dst = tile + ((lc[0] + ra) * TW + (lc[1] + rb)) * TW + lc[2];
#pragma unroll
                        for (int c = 0; c < W2 / 2; ++c) {
                            dst[2 * c] += acc[k][c].x;
                            dst[2 * c + 1] += acc[k][c].y;
                        }
                    }
                }
#pragma unroll
                for (int k = 0; k < RPL; ++k)
#pragma unroll
                    for (int c = 0; c < W2 / 2; ++c) acc[k][c] = zero2();
                __syncwarp();
            }
            if (done) break;
            s = sn;
            q = qn;
            send = sendn;
            if (newpiece) {
                sg = sgn;
                sg_next = sg_next2;
            }
            cnt = cntn;
            fx = nfx;
            fy = nfy;
            fz = nfz;
            vv = nvv;
        }
    }
    __syncthreads();
    float *out = reinterpret_cast<float *>(a.tiles) + ((size_t)wi_idx * a.nrhs + r) * C::TV;
    for (int i = threadIdx.x; i < C::TV; i += NWARP * 32) {
        float s2 = 0.0f;
#pragma unroll
        for (int w = 0; w < NWARP; ++w) s2 += tiles_s[w * C::TVP + i];
        out[i] = s2;
    }
}

// ------------------------------------------------------------------ work-item tiles -> bin tile
// A bin split into several work items has several partial tiles; they are summed, in work-item
// order, into the slot of the bin's first work item, so the grid gather reads one tile per bin.
struct BinReduceArgs {
    void *tiles;
    const int4 *mbins;           // {first work item, count, tile volume, 0} of multi-item bins
    int nmbins, nrhs, mb_begin;
    int tv_max;                  // largest tile volume among these bins (sets the chunk count)
};

// One CTA per (bin, chunk of 128 tile elements): warp k sums the work items k, k+8, k+16, ... of
// its chunk (four elements per lane, 32 apart, so four independent loads per item), then warps
// 0-3 each add the eight partial sums of 32 elements in a fixed order.
constexpr int kBinReduceChunk = 128;

template <typename T>
__global__ void __launch_bounds__(256) k_bin_reduce(BinReduceArgs a) {
    pdl_wait();
    pdl_trigger();
    constexpr int EPL = kBinReduceChunk / 32;  // elements per lane
    __shared__ T part[8][kBinReduceChunk];
    const int chunks = (a.tv_max + kBinReduceChunk - 1) / kBinReduceChunk;
    const int b = a.mb_begin + blockIdx.x / chunks;
    const int c = blockIdx.x % chunks;
    const int r = blockIdx.y;
    const int4 mb = a.mbins[b];
    const int tv = mb.z;
    const int lane = threadIdx.x & 31;
    const int slice = threadIdx.x >> 5;
    const int e0 = c * kBinReduceChunk + lane;
    if (c * kBinReduceChunk >= tv) return;  // whole CTA: this bin's tile is shorter
    T *tiles = reinterpret_cast<T *>(a.tiles);
    T s[EPL];
#pragma unroll
    for (int i = 0; i < EPL; ++i) s[i] = T(0);
    for (int k = slice; k < mb.y; k += 8) {
        const T *tk = tiles + ((size_t)(mb.x + k) * a.nrhs + r) * tv;
#pragma unroll
        for (int i = 0; i < EPL; ++i)
            if (e0 + 32 * i < tv) s[i] += tk[e0 + 32 * i];
    }
#pragma unroll
    for (int i = 0; i < EPL; ++i) part[slice][lane + 32 * i] = s[i];
    __syncthreads();
    if (slice < EPL) {
        const int e = e0 + 32 * slice;
        if (e < tv) {
            T t = part[0][lane + 32 * slice];
#pragma unroll
            for (int k = 1; k < 8; ++k) t += part[k][lane + 32 * slice];
            tiles[((size_t)mb.x * a.nrhs + r) * tv + e] = t;
        }
    }
}

// ------------------------------------------------------------------ bin tiles -> grid
struct ReduceArgs {
    const void *tiles;
    void *grid0;                 // T[nrhs][grid_total]
    const DevWindow *dwin;
    const int2 *bins;            // {first work item, count} per window per bin
    long long grid_total;
    long long box_cum[kMaxWindows + 1];  // cumulative box volumes of windows w_begin..
    int w_begin, w_end, nrhs, n_os, NB, M, B;
    int zero_offset;             // 1: grid0 is one window's grid (ignore its grid offset)
};

template <typename T, int DW>
__global__ void __launch_bounds__(256) k_reduce(ReduceArgs a) {
    pdl_wait();
    pdl_trigger();
    const int r = blockIdx.y;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int nw = a.w_end - a.w_begin;
    if (idx >= a.box_cum[nw]) return;
    int wl = 0;
    while (idx >= a.box_cum[wl + 1]) ++wl;
    const int w = a.w_begin + wl;
    const DevWindow dw = a.dwin[w];
    long long loc = idx - a.box_cum[wl];
    int u[3] = {0, 0, 0};
    for (int k = DW - 1; k >= 0; --k) {
        const int ext = dw.box_hi[k] - dw.box_lo[k];
        u[k] = dw.box_lo[k] + (int)(loc % ext);
        loc /= ext;
    }
    const int TW = a.B + 2 * a.M - 1;
    int TV = TW;
    for (int k = 1; k < DW; ++k) TV *= TW;
    int blo[3] = {0, 0, 0}, bhi[3] = {0, 0, 0};
    for (int k = 0; k < DW; ++k) {
        // bin b covers grid points [b B - M + 1, b B + B + M - 1]
        const int lo_num = u[k] - a.B - a.M + 1;  // b >= ceil(lo_num / B)
        int lo = lo_num >= 0 ? (lo_num + a.B - 1) / a.B : -((-lo_num) / a.B);
        int hi = (u[k] + a.M - 1) >= 0 ? (u[k] + a.M - 1) / a.B : -1;
        blo[k] = max(lo, 0);
        bhi[k] = min(hi, a.NB - 1);
    }
    const T *tiles = reinterpret_cast<const T *>(a.tiles);
    T s = T(0);
    for (int b0 = blo[0]; b0 <= bhi[0]; ++b0) {
        for (int b1 = (DW > 1 ? blo[1] : 0); b1 <= (DW > 1 ? bhi[1] : 0); ++b1) {
            for (int b2 = (DW > 2 ? blo[2] : 0); b2 <= (DW > 2 ? bhi[2] : 0); ++b2) {
                const int l0 = u[0] - (b0 * a.B - a.M + 1);
                const int l1 = DW > 1 ? u[1] - (b1 * a.B - a.M + 1) : 0;
                const int l2 = DW > 2 ? u[2] - (b2 * a.B - a.M + 1) : 0;
                if (l0 < 0 || l0 >= TW || l1 < 0 || l1 >= TW || l2 < 0 || l2 >= TW) continue;
                int lin = b0, l = l0;
                if (DW > 1) { lin = lin * a.NB + b1; l = l * TW + l1; }
                if (DW > 2) { lin = lin * a.NB + b2; l = l * TW + l2; }
                const int2 be = a.bins[dw.bin_off + lin];
                if (be.y > 0) s += tiles[((size_t)be.x * a.nrhs + r) * TV + l];
            }
        }
    }
    long long g = u[0];
    if (DW > 1) g = g * a.n_os + u[1];
    if (DW > 2) g = g * a.n_os + u[2];
    reinterpret_cast<T *>(a.grid0)[(size_t)r * a.grid_total + (a.zero_offset ? 0 : dw.grid_off) + g] = s;
}

// ------------------------------------------------------------------ gather interpolation
struct InterpArgs {
    const int4 *segs;
    const void *frac;
    const int *perm;
    const void *grid;            // T[nrhs][grid_total] (grid_stride_rhs between RHS)
    const DevWindow *dwin;
    void *part;                  // T[P][nrhs][n] (indexed by internal window)
    long long n, total, grid_stride_rhs;
    int nrhs, seg_begin, seg_end, n_os;
    int zero_offset;             // 1: grid is one window's grid (ignore its grid offset)
    int part_w0;                 // part holds windows part_w0, part_w0 + 1, ...
    WinParams wp;
};

template <typename T, int DW, int M, int NWARP>
struct InterpCfg {
    using G = Geo<DW, M>;
    static constexpr int VOLP = (G::VOL + 3) / 4 * 4;
    static constexpr size_t smem = sizeof(T) * (size_t)NWARP * VOLP;
};

template <typename T, int DW, int M, int NWARP>
__global__ void __launch_bounds__(NWARP * 32) k_interp(InterpArgs a) {
    pdl_wait();
    pdl_trigger();
    using C = InterpCfg<T, DW, M, NWARP>;
    using G = typename C::G;
    constexpr int W2 = G::W2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s = a.seg_begin + blockIdx.x * NWARP + warp;
    if (s >= a.seg_end) return;
    const int r = blockIdx.y;
    T *blk = reinterpret_cast<T *>(smem_raw) + warp * C::VOLP;
    const int4 sg = a.segs[s];
    const int w = sg.w;
    const DevWindow dw = a.dwin[w];
    const T *grid = reinterpret_cast<const T *>(a.grid) + (size_t)r * a.grid_stride_rhs +
                    (a.zero_offset ? 0 : dw.grid_off);
    int c0[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) c0[k] = cell_coord(sg.x, k) - M + 1;
    for (int o = lane; o < G::VOL; o += 32) {
        long long g;
        if (DW == 3) {
            const int aa = o / (W2 * W2), bb = (o / W2) % W2, cc = o % W2;
            g = ((long long)(c0[0] + aa) * a.n_os + (c0[1] + bb)) * a.n_os + (c0[2] + cc);
        } else if (DW == 2) {
            const int aa = o / W2, bb = o % W2;
            g = (long long)(c0[0] + aa) * a.n_os + (c0[1] + bb);
        } else {
            g = c0[0] + o;
        }
        blk[o] = grid[g];
    }
    __syncwarp();
    const T *frac = reinterpret_cast<const T *>(a.frac);
    T *out = reinterpret_cast<T *>(a.part) + ((size_t)(w - a.part_w0) * a.nrhs + r) * a.n;
    for (int qb = 0; qb < sg.z; qb += 32) {
        const bool valid = qb + lane < sg.z;
        const int q = sg.y + min(qb + lane, sg.z - 1);
        T wt[DW][W2];
#pragma unroll
        for (int k = 0; k < DW; ++k) Weights<T, M>::eval(frac[(size_t)k * a.total + q], a.wp, wt[k]);
        T f = T(0);
        if (DW == 3) {
            // a-loop kept rolled (the block is re-read from shared memory, not hoisted into
            // registers); the x weights rotate through registers instead of dynamic indexing
            T wx[W2];
#pragma unroll
            for (int k = 0; k < W2; ++k) wx[k] = wt[0][k];
#pragma unroll 1
            for (int aa = 0; aa < W2; ++aa) {
                const T *plane = blk + aa * W2 * W2;
                T sa = T(0);
                if constexpr (sizeof(T) == 4 && W2 % 4 == 0) {
                    // inner products along c on f32x2 pairs (two FMAs per instruction)
                    f32x2 wz2[W2 / 2];
#pragma unroll
                    for (int cc = 0; cc < W2 / 2; ++cc) wz2[cc] = pack2(wt[2][2 * cc], wt[2][2 * cc + 1]);
#pragma unroll
                    for (int bb = 0; bb < W2; ++bb) {
                        f32x2 sb2 = zero2();
#pragma unroll
                        for (int cc = 0; cc < W2 / 2; cc += 2) {
                            f32x2 t0, t1;
                            lds_pairs(plane + bb * W2 + 2 * cc, t0, t1);
                            sb2 = fma2(t0, wz2[cc], sb2);
                            sb2 = fma2(t1, wz2[cc + 1], sb2);
                        }
                        float lo, hi;
                        unpack2(sb2, lo, hi);
                        sa = fma(wt[1][bb], lo + hi, sa);
                    }
                } else {
#pragma unroll
                    for (int bb = 0; bb < W2; ++bb) {
                        T row[W2];
                        lds_vec<T, W2>(plane + bb * W2, row);
                        T sb = T(0);
#pragma unroll
                        for (int cc = 0; cc < W2; ++cc) sb = fma(row[cc], wt[2][cc], sb);
                        sa = fma(wt[1][bb], sb, sa);
                    }
                }
                f = fma(wx[0], sa, f);
#pragma unroll
                for (int k = 0; k < W2 - 1; ++k) wx[k] = wx[k + 1];
            }
        } else if (DW == 2) {
#pragma unroll
            for (int aa = 0; aa < W2; ++aa) {
                T row[W2];
                lds_vec<T, W2>(blk + aa * W2, row);
                T sb = T(0);
#pragma unroll
                for (int cc = 0; cc < W2; ++cc) sb = fma(row[cc], wt[1][cc], sb);
                f = fma(wt[0][aa], sb, f);
            }
        } else {
#pragma unroll
            for (int cc = 0; cc < W2; ++cc) f = fma(blk[cc], wt[0][cc], f);
        }
        if (valid) out[a.perm[q]] = f;
    }
}

// ------------------------------------------------------------------ FP32 3-D interpolation
// One CTA per spread work item (one bin's run of cells). The bin's grid neighbourhood is staged in
// shared memory as B shifted copies: copy s holds, for every (x, y) of the neighbourhood, the 2M
// values along the last axis that a cell with last local coordinate s needs, 16-byte aligned.
// Any lane can then read its own cell's rows with 128-bit loads, so a warp evaluates 32
// consecutive points per batch (one per lane) whatever cells they fall in; lanes of one cell
// share addresses (broadcast). Per-point inputs of the next batch load while the current batch
// computes; inner products along the last axis use f32x2 pairs.
struct InterpWiArgs {
    const int4 *wis;
    const int4 *segs;
    const float *frac;
    const int *perm;
    const unsigned char *cellloc;  // cell index inside its bin, (l0 B + l1) B + l2, per sorted point
    const float *grid;       // [nrhs][grid_total]
    const DevWindow *dwin;
    float *part;             // [P][nrhs][n] by internal window (offset by part_w0)
    long long n, total, grid_stride_rhs;
    int nrhs, wi_begin, wi_end, n_os, part_w0;
    WinParams wp;
    int *status;             // error bits (tensor-core path: a bounded wait ran out)
    unsigned wait_polls;     // tensor-core path: polls of each chunk's completion wait before it
                             // gives up (the drain before the accumulators are freed always
                             // uses the full limit)
    const int *order;        // persistent kernels: work items of each window, largest first
    int *counters;           // persistent kernels: per-RHS work counters (zeroed before the launch)
    const int4 *chunks;      // tensor-core path: chunks {sorted start, count, l0 | l1 << 8, 0}
    const int *wi_chunk;     // tensor-core path: chunks of work item x: [wi_chunk[x], wi_chunk[x + 1])
};

template <int M, int B, int NWARP>
struct InterpX2Cfg {
    static constexpr int W2 = 2 * M;
    static constexpr int TW = B + W2 - 1;
    static constexpr int ROWS = TW * TW;
    static constexpr size_t smem = sizeof(float) * (size_t)B * ROWS * W2;
};

template <int M, int B, int NWARP>
__global__ void __launch_bounds__(NWARP * 32) k_interp3_x2(InterpWiArgs a) {
    pdl_wait();
    pdl_trigger();
    using C = InterpX2Cfg<M, B, NWARP>;
    constexpr int W2 = C::W2, TW = C::TW, ROWS = C::ROWS;
    static_assert(W2 % 4 == 0, "pairs along the last axis");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *cp = reinterpret_cast<float *>(smem_raw);

    const int wi_idx = a.wi_begin + blockIdx.x;
    if (wi_idx >= a.wi_end) return;
    const int r = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int4 wi = a.wis[wi_idx];
    const int w = wi.x;
    const int bin[3] = {cell_coord(wi.w, 0), cell_coord(wi.w, 1), cell_coord(wi.w, 2)};
    const DevWindow dw = a.dwin[w];
    const float *grid = a.grid + (size_t)r * a.grid_stride_rhs + dw.grid_off;
    {
        const int o0 = bin[0] * B - M + 1, o1 = bin[1] * B - M + 1, o2 = bin[2] * B - M + 1;
        for (int e = threadIdx.x; e < B * ROWS * W2; e += NWARP * 32) {
            const int c = e % W2, row = (e / W2) % ROWS, sh = e / (W2 * ROWS);
            const int x = row / TW, y = row % TW;
            cp[e] = grid[((long long)(o0 + x) * a.n_os + (o1 + y)) * a.n_os + (o2 + sh + c)];
        }
    }
    __syncthreads();
    const int4 s_first = a.segs[wi.y];
    const int4 s_last = a.segs[wi.z - 1];
    const int p0 = s_first.y, p1 = s_last.y + s_last.z;
    const int len = p1 - p0;
    const int pw0 = p0 + (int)(((long long)len * warp) / NWARP);
    const int pw1 = p0 + (int)(((long long)len * (warp + 1)) / NWARP);
    if (pw0 >= pw1) return;
    const float *fr0 = a.frac, *fr1 = a.frac + a.total, *fr2 = a.frac + 2 * a.total;
    float *out = a.part + ((size_t)(w - a.part_w0) * a.nrhs + r) * a.n;

    // current batch inputs (lanes past the range keep a valid point's data and do not write)
    int q = pw0 + min(lane, pw1 - pw0 - 1);
    float fx = fr0[q], fy = fr1[q], fz = fr2[q];
    int pi = a.perm[q];
    int loc = a.cellloc[q];
    for (int qb = pw0; qb < pw1; qb += 32) {
        const bool valid = qb + lane < pw1;
        const int qbn = qb + 32;
        float nfx = fx, nfy = fy, nfz = fz;
        int npi = pi, nloc = loc;
        if (qbn < pw1) {
            const int qn = qbn + min(lane, pw1 - qbn - 1);
            nfx = fr0[qn];
            nfy = fr1[qn];
            nfz = fr2[qn];
            npi = a.perm[qn];
            nloc = a.cellloc[qn];
        }
        float wx[W2], wy[W2], wz[W2];
        Weights<float, M>::eval(fx, a.wp, wx);
        Weights<float, M>::eval(fy, a.wp, wy);
        Weights<float, M>::eval(fz, a.wp, wz);
        f32x2 wz2[W2 / 2];
#pragma unroll
        for (int cc = 0; cc < W2 / 2; ++cc) wz2[cc] = make_float2(wz[2 * cc], wz[2 * cc + 1]);
        const int l2 = loc % B, l1 = (loc / B) % B, l0 = loc / (B * B);
        const float *base = cp + ((size_t)l2 * ROWS + l0 * TW + l1) * W2;
        float f = 0.0f;
#pragma unroll 1
        for (int aa = 0; aa < W2; ++aa) {
            const float *plane = base + aa * TW * W2;
            float sa = 0.0f;
#pragma unroll
            for (int bb = 0; bb < W2; ++bb) {
                f32x2 sb2 = zero2();
#pragma unroll
                for (int cc = 0; cc < W2 / 2; cc += 2) {
                    f32x2 t0, t1;
                    lds_pairs(plane + bb * W2 + 2 * cc, t0, t1);
                    sb2 = fma2(t0, wz2[cc], sb2);
                    sb2 = fma2(t1, wz2[cc + 1], sb2);
                }
                sa = fmaf(wy[bb], sb2.x + sb2.y, sa);
            }
            f = fmaf(wx[0], sa, f);
#pragma unroll
            for (int k = 0; k < W2 - 1; ++k) wx[k] = wx[k + 1];
        }
        if (valid) out[pi] = f;
        fx = nfx;
        fy = nfy;
        fz = nfz;
        pi = npi;
        loc = nloc;
    }
}

// ------------------------------------------------------------------ FP32 3-D interpolation, tensor cores
// For points p whose cells share the first two cell coordinates (a "column" of up to B cells
// along the last axis, consecutive in sorted order), the inner sums along the last axis,
// h_p[a, b] = sum_c z_p[c] g[l0 + a, l1 + b, l2_p + c], are one matrix product: the points' window
// weights placed at their cell's offset l2_p in a row of 16 (the column's 11 grid values padded)
// times the column's 64 x 16 block of the bin neighbourhood. A CTA of four warps takes up to 128
// points of one column at a time (a chunk, cut once in the plan's chunk table) and has the tensor
// cores form all their 64 inner sums
// (tcgen05.mma kind::tf32, M = 128, N = 64, K = 2 x 8; both operands split into a tf32 high part
// and an FP32 remainder so that hi*hi + hi*lo + lo*hi carries ~22 significant bits; FP32
// accumulation in tensor memory). Each thread then reads its point's 64 sums from tensor memory
// and finishes sum_a x_a sum_b y_b h[a, b] on the FP32 pipe. Chunks are software-pipelined over two
// operand buffers and two accumulators (the product of one chunk runs while the previous chunk's
// sums are finished and the next chunk's inputs load). CTAs are persistent and take work items
// from a counter. Every completion wait is bounded and reports through a.status.
template <int M, int B>
struct InterpTcCfg {
    static constexpr int W2 = 2 * M;
    static constexpr int TW = B + W2 - 1;
    static constexpr int TV = TW * TW * TW;
    static constexpr int TVP = (TV + 3) / 4 * 4;
    static constexpr int ROWS = 128;                 // points per chunk (MMA M)
    static constexpr int NCOL = W2 * W2;             // rows (a, b) of the column block (MMA N)
    static constexpr int KC = 16;                    // column length TW padded to two K = 8 steps
    static constexpr uint32_t A_BYTES = ROWS * KC * 4, B_BYTES = NCOL * KC * 4;
    // two buffers of {A hi, A lo} and of {B hi, B lo}, the neighbourhood, the work item's chunks,
    // barriers, TMEM slot, work
    static constexpr int CHUNK_CACHE = 128;          // chunks of a work item kept in shared memory
    static constexpr uint32_t A0 = 0, B0 = 4 * A_BYTES, TILE = B0 + 4 * B_BYTES, CHUNKS = TILE + TVP * 4,
                              MBAR = CHUNKS + CHUNK_CACHE * 16, SLOT = MBAR + 16, WORK = SLOT + 4;
    static constexpr size_t smem = SLOT + 16;
    static constexpr uint32_t kMaxPolls = 1u << 22;
    static constexpr uint32_t TMEM_COLS = 2 * NCOL;  // two accumulators
    static_assert(TW <= KC, "a column fits in two K = 8 steps");
};

// per-RHS counters of the persistent tensor-core kernels live after the status word, in blocks
// of kStatusCounters ints: 16 work counters (next work item per RHS), then 16 exit counters
// (CTAs that have finished, per RHS). The last CTA of a RHS to finish puts both back to zero,
// so every launch finds them zeroed without a memset in the stream.
constexpr int kStatusCounters = 32;
constexpr int kStatusInts = 1 + 3 * kStatusCounters;
static_assert(kStatusInts <= kStatusAlloc, "status block holds three counter blocks");

// PARAM_WAIT: the chunk completion waits take their poll bound from a.wait_polls (the
// failure-detection hook) instead of the compile-time bound. Only launched when the bound was
// lowered: a runtime bound in the hot loop measured about 11 % slower.
template <int M, int B, bool PARAM_WAIT>
__global__ void __launch_bounds__(128, ANOVA_TC_INTERP_MINB) k_interp3_tc(InterpWiArgs a) {
    pdl_wait();
    pdl_trigger();
    using C = InterpTcCfg<M, B>;
    constexpr int W2 = C::W2, TW = C::TW, ROWS = C::ROWS, KC = C::KC;
    static_assert(W2 == 8 && C::NCOL == 64 && B <= 8, "layout written for m = 4, bins of at most 8 cells");
    static_assert(ROWS == kTcChunkRows, "chunk table cut for this chunk size");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *tile = reinterpret_cast<float *>(smem_raw + C::TILE);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem_raw + C::MBAR);
    uint32_t *slot = reinterpret_cast<uint32_t *>(smem_raw + C::SLOT);
    int *work_s = reinterpret_cast<int *>(smem_raw + C::WORK);
    int4 *chunks_s = reinterpret_cast<int4 *>(smem_raw + C::CHUNKS);

    const int r = blockIdx.y;
    const int t = threadIdx.x, warp = t >> 5;
    if (warp == 0) tc::tmem_alloc(slot, C::TMEM_COLS);
    if (t == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        tc::mbar_init_fence();
    }
    // operand rows past a chunk's end (and the pad of B) are read by the product: keep them finite
    for (int i = t; i < (int)(C::TILE / 4); i += 128) reinterpret_cast<float *>(smem_raw)[i] = 0.0f;
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot;
    const uint32_t sbase = tc::smem_u32(smem_raw);
    constexpr uint32_t idesc = tc::idesc_tf32(ROWS, C::NCOL);
    const float *fr0 = a.frac, *fr1 = a.frac + a.total, *fr2 = a.frac + 2 * a.total;
    int *counter = a.counters + r;
    const int nwork = a.wi_end - a.wi_begin;
    // this thread's B entries: row n = t / 2 (a = n / 8, b = n % 8), K half t % 2 (8 values)
    const int bn = t >> 1, bkh = t & 1;
    const int ba = bn >> 3, bb = bn & 7;

    uint32_t parity = 0u;   // bit b: phase parity of barrier b
    uint32_t pending = 0u;  // bit b: a product committed to barrier b is not yet waited for
    int buf = 0;
    bool alive = true;
    bool failed = false;    // this thread's bounded wait ran out

    struct Chunk {
        int q0, cnt, l0, l1;
    };
    // per-thread inputs of one chunk
    struct Raw {
        float f[3];
        int pi, l2;
    };

    while (alive) {
        if (t == 0) *work_s = atomicAdd(counter, 1);
        if (__syncthreads_or(failed)) {
            alive = false;
            if (t == 0) atomicOr(a.status, 1);
            break;
        }
        const int k = *work_s;
        if (k >= nwork) break;
        const int wi_idx = a.order[a.wi_begin + k];
        const int4 wi = a.wis[wi_idx];
        const int w = wi.x;
        const int bin[3] = {cell_coord(wi.w, 0), cell_coord(wi.w, 1), cell_coord(wi.w, 2)};
        const DevWindow dw = a.dwin[w];
        const float *grid = a.grid + (size_t)r * a.grid_stride_rhs + dw.grid_off;
        float *out = a.part + ((size_t)(w - a.part_w0) * a.nrhs + r) * a.n;
        {
            const int o0 = bin[0] * B - M + 1, o1 = bin[1] * B - M + 1, o2 = bin[2] * B - M + 1;
            for (int e = t; e < C::TV; e += 128) {
                const int z = e % TW, y = (e / TW) % TW, x = e / (TW * TW);
                tile[e] = grid[((long long)(o0 + x) * a.n_os + (o1 + y)) * a.n_os + (o2 + z)];
            }
        }
        // the item's chunks (up to ROWS consecutive points of one column; the plan's chunk
        // table) in shared memory
        const int ch0 = a.wi_chunk[wi_idx], ch1 = a.wi_chunk[wi_idx + 1];
        const bool ch_cached = ch1 - ch0 <= C::CHUNK_CACHE;
        if (ch_cached)
            for (int i = t; i < ch1 - ch0; i += 128) chunks_s[i] = a.chunks[ch0 + i];
        __syncthreads();
        int cc = ch0;
        auto form = [&](Chunk &ch) {
            ch.cnt = 0;
            if (cc >= ch1) return;
            const int4 d = ch_cached ? chunks_s[cc - ch0] : a.chunks[cc];
            ++cc;
            ch.q0 = d.x;
            ch.cnt = d.y;
            ch.l0 = d.z & 255;
            ch.l1 = d.z >> 8;
        };
        auto load_raw = [&](const Chunk &ch, Raw &rw) {
            if (t < ch.cnt) {
                const int q = ch.q0 + t;
                rw.f[0] = fr0[q];
                rw.f[1] = fr1[q];
                rw.f[2] = fr2[q];
                rw.pi = a.perm[q];
                rw.l2 = a.cellloc[q] % B;
            }
        };
        // both operands of one chunk: the points' last-axis weights (A) and the column block (B)
        auto stage = [&](int bf, const Chunk &ch, const Raw &rw) {
            unsigned char *abuf = smem_raw + C::A0 + bf * 2 * C::A_BYTES;
            unsigned char *bbuf = smem_raw + C::B0 + bf * 2 * C::B_BYTES;
            if (t < ch.cnt) {
                float wz[W2];
                Weights<float, M>::eval(rw.f[2], a.wp, wz);
                float hi[W2], lo[W2];
#pragma unroll
                for (int j = 0; j < W2; ++j) tc::split_tf32(wz[j], hi[j], lo[j]);
                // the row holds z at positions l2 .. l2 + 7 of 16 (the rest zero)
                auto put = [&](auto shift_tag) {
                    constexpr int SH = decltype(shift_tag)::value;
                    float vh[KC], vl[KC];
#pragma unroll
                    for (int c = 0; c < KC; ++c) {
                        vh[c] = (c >= SH && c < SH + W2) ? hi[c - SH] : 0.0f;
                        vl[c] = (c >= SH && c < SH + W2) ? lo[c - SH] : 0.0f;
                    }
#pragma unroll
                    for (int c4 = 0; c4 < KC; c4 += 4) {
                        *reinterpret_cast<float4 *>(abuf + tc::operand_offset16(t, c4)) =
                            make_float4(vh[c4], vh[c4 + 1], vh[c4 + 2], vh[c4 + 3]);
                        *reinterpret_cast<float4 *>(abuf + C::A_BYTES + tc::operand_offset16(t, c4)) =
                            make_float4(vl[c4], vl[c4 + 1], vl[c4 + 2], vl[c4 + 3]);
                    }
                };
                switch (rw.l2) {
                    case 0: put(std::integral_constant<int, 0>()); break;
                    case 1: if constexpr (B > 1) put(std::integral_constant<int, 1>()); break;
                    case 2: if constexpr (B > 2) put(std::integral_constant<int, 2>()); break;
                    case 3: if constexpr (B > 3) put(std::integral_constant<int, 3>()); break;
                    case 4: if constexpr (B > 4) put(std::integral_constant<int, 4>()); break;
                    case 5: if constexpr (B > 5) put(std::integral_constant<int, 5>()); break;
                    case 6: if constexpr (B > 6) put(std::integral_constant<int, 6>()); break;
                    default: if constexpr (B > 7) put(std::integral_constant<int, 7>()); break;
                }
            }
            const float *src = tile + ((ch.l0 + ba) * TW + (ch.l1 + bb)) * TW;
            float hi[8], lo[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int c = 8 * bkh + j;
                tc::split_tf32(c < TW ? src[c < TW ? c : 0] : 0.0f, hi[j], lo[j]);
            }
#pragma unroll
            for (int j4 = 0; j4 < 8; j4 += 4) {
                *reinterpret_cast<float4 *>(bbuf + tc::operand_offset16(bn, 8 * bkh + j4)) =
                    make_float4(hi[j4], hi[j4 + 1], hi[j4 + 2], hi[j4 + 3]);
                *reinterpret_cast<float4 *>(bbuf + C::B_BYTES + tc::operand_offset16(bn, 8 * bkh + j4)) =
                    make_float4(lo[j4], lo[j4 + 1], lo[j4 + 2], lo[j4 + 3]);
            }
        };
        auto issue = [&](int bf) {
            const uint32_t ab = sbase + C::A0 + bf * 2 * C::A_BYTES, bbase = sbase + C::B0 + bf * 2 * C::B_BYTES;
            const uint32_t d = tmem + (uint32_t)(bf * C::NCOL);
            tc::fence_after_sync();
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                const uint32_t ko = 256u * ks;
                const uint64_t ahi = tc::smem_desc(ab + ko, 128, 512), alo = tc::smem_desc(ab + C::A_BYTES + ko, 128, 512);
                const uint64_t bhi = tc::smem_desc(bbase + ko, 128, 512), blo = tc::smem_desc(bbase + C::B_BYTES + ko, 128, 512);
                tc::mma_tf32(d, ahi, bhi, idesc, ks > 0);
                tc::mma_tf32(d, ahi, blo, idesc, true);
                tc::mma_tf32(d, alo, bhi, idesc, true);
            }
            tc::mma_commit(&mbar[bf]);
        };
        // finish chunk `ch` whose product went to accumulator bf
        // (the first two axes' weights are evaluated here, while the product runs). A thread whose
        // bounded wait runs out marks itself failed and skips the dependent work; the block agrees
        // on failures at the next barrier.
        auto finish = [&](int bf, const Chunk &ch, const Raw &rw) {
            float wx[W2], wy[W2];
            Weights<float, M>::eval(rw.f[0], a.wp, wx);
            Weights<float, M>::eval(rw.f[1], a.wp, wy);
            if (!tc::mbar_wait_bounded(&mbar[bf], (parity >> bf) & 1u, PARAM_WAIT ? a.wait_polls : C::kMaxPolls)) {
                failed = true;
                return;
            }
            parity ^= 1u << bf;
            pending &= ~(1u << bf);
            tc::fence_after_sync();
            const uint32_t col = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(bf * C::NCOL);
            float f = 0.0f;
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4) {
                float h[16];
                tc::tmem_ld16(col + (uint32_t)(16 * q4), h);
#pragma unroll
                for (int aa = 0; aa < 2; ++aa) {
#if ANOVA_EPI_PAIR
                    // b-sums in pairs (even and odd b), the two halves added at the end
                    f32x2 sp = zero2();
#pragma unroll
                    for (int b2 = 0; b2 < W2; b2 += 2)
                        sp = fma2(make_float2(wy[b2], wy[b2 + 1]), make_float2(h[aa * W2 + b2], h[aa * W2 + b2 + 1]), sp);
                    const float sb = sp.x + sp.y;
#else
                    float sb = 0.0f;
#pragma unroll
                    for (int b2 = 0; b2 < W2; ++b2) sb = fmaf(wy[b2], h[aa * W2 + b2], sb);
#endif
                    f = fmaf(wx[2 * q4 + aa], sb, f);
                }
            }
            if (t < ch.cnt) out[rw.pi] = f;
            tc::fence_before_sync();
        };
        // one pipeline step: stage and start chunk `nx` (if any) into buffer bf ^ 1, load the
        // inputs of the chunk after it, finish chunk `cu` from buffer bf
        auto step = [&](Chunk &cu, Raw &rcu, Chunk &nx, Raw &rnx, Chunk &nn, Raw &rnn) -> int {
            const bool have_next = nx.cnt > 0;
            if (have_next) stage(buf ^ 1, nx, rnx);
            form(nn);
            load_raw(nn, rnn);
            tc::fence_proxy_async();
            if (__syncthreads_or(failed)) return -1;
            if (have_next) {
                if (t == 0) issue(buf ^ 1);
                pending |= 1u << (buf ^ 1);
            }
            finish(buf, cu, rcu);
            buf ^= 1;
            return have_next ? 1 : 0;
        };

        Chunk c0, c1, c2;
        Raw r0, r1, r2;
        form(c0);
        load_raw(c0, r0);
        stage(buf, c0, r0);
        form(c1);
        load_raw(c1, r1);
        tc::fence_proxy_async();
        __syncthreads();
        if (t == 0) issue(buf);
        pending |= 1u << buf;
        // ping-pong between the two register sets; c2/r2 receive the chunk after next
        int st;
        while (true) {
            st = step(c0, r0, c1, r1, c2, r2);
            if (st <= 0) break;
            c0 = c2;
            r0 = r2;
            st = step(c1, r1, c0, r0, c2, r2);
            if (st <= 0) break;
            c1 = c2;
            r1 = r2;
        }
        if (st < 0) {
            if (t == 0) atomicOr(a.status, 1);
            alive = false;
        }
    }
    if (!alive) {
        // a completion that never arrived: one more bounded wait on each barrier's pending
        // phase before the accumulator columns are released
#pragma unroll
        for (int b = 0; b < 2; ++b)
            if ((pending >> b) & 1u) tc::mbar_wait_bounded(&mbar[b], (parity >> b) & 1u, C::kMaxPolls);
    }
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, C::TMEM_COLS);
    if (t == 0) {
        // every CTA has taken its last work item before it counts itself out; the last one out
        // resets this RHS's counters for the next launch
        __threadfence();
        if (atomicAdd(&a.counters[16 + r], 1) == (int)gridDim.x - 1) {
            atomicExch(&a.counters[r], 0);
            atomicExch(&a.counters[16 + r], 0);
        }
    }
}

// ------------------------------------------------------------------ interpolation, any dims
// The general form of the per-bin interpolation (any precision, 1-3 dims, any cut-off): one CTA
// per work item stages the bin's grid neighbourhood ((B + 2M - 1)^d values) in shared memory,
// warps split the item's points evenly, one point per lane, scalar shared-memory reads.
template <typename T>
struct InterpBinArgs {
    const int4 *wis;
    const int4 *segs;
    const T *frac;
    const int *perm;
    const unsigned char *cellloc;
    const T *grid;
    const DevWindow *dwin;
    T *part;
    long long n, total, grid_stride_rhs;
    int nrhs, wi_begin, wi_end, n_os, part_w0;
    WinParams wp;
};

template <typename T, int DW, int M, int B, int NWARP>
struct InterpBinCfg {
    static constexpr int W2 = 2 * M;
    static constexpr int TW = B + W2 - 1;
    static constexpr int TV = ipow(TW, DW);
    static constexpr size_t smem = sizeof(T) * (size_t)TV;
};

template <typename T, int DW, int M, int B, int NWARP>
__global__ void __launch_bounds__(NWARP * 32) k_interp_bin(InterpBinArgs<T> a) {
    pdl_wait();
    pdl_trigger();
    using C = InterpBinCfg<T, DW, M, B, NWARP>;
    constexpr int W2 = C::W2, TW = C::TW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *bt = reinterpret_cast<T *>(smem_raw);
    const int wi_idx = a.wi_begin + blockIdx.x;
    if (wi_idx >= a.wi_end) return;
    const int r = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int4 wi = a.wis[wi_idx];
    const int w = wi.x;
    const int bin[3] = {cell_coord(wi.w, 0), cell_coord(wi.w, 1), cell_coord(wi.w, 2)};
    const DevWindow dw = a.dwin[w];
    const T *grid = a.grid + (size_t)r * a.grid_stride_rhs + dw.grid_off;
    for (int e = threadIdx.x; e < C::TV; e += NWARP * 32) {
        int rem = e;
        long long g = 0;
        int l[3] = {0, 0, 0};
        for (int k = DW - 1; k >= 0; --k) {
            l[k] = rem % TW;
            rem /= TW;
        }
        for (int k = 0; k < DW; ++k) g = g * a.n_os + (bin[k] * B - M + 1 + l[k]);
        bt[e] = grid[g];
    }
    __syncthreads();
    const int4 s_first = a.segs[wi.y];
    const int4 s_last = a.segs[wi.z - 1];
    const int p0 = s_first.y, p1 = s_last.y + s_last.z;
    const int len = p1 - p0;
    const int pw0 = p0 + (int)(((long long)len * warp) / NWARP);
    const int pw1 = p0 + (int)(((long long)len * (warp + 1)) / NWARP);
    T *out = a.part + ((size_t)(w - a.part_w0) * a.nrhs + r) * a.n;
    for (int qb = pw0; qb < pw1; qb += 32) {
        const bool valid = qb + lane < pw1;
        const int q = qb + min(lane, pw1 - qb - 1);
        int loc = a.cellloc[q];
        int lc[3] = {0, 0, 0};
        for (int k = DW - 1; k >= 0; --k) {
            lc[k] = loc % B;
            loc /= B;
        }
        T wt[DW][W2];
#pragma unroll
        for (int k = 0; k < DW; ++k) Weights<T, M>::eval(a.frac[(size_t)k * a.total + q], a.wp, wt[k]);
        T f = T(0);
        if (DW == 3) {
#pragma unroll 1
            for (int aa = 0; aa < W2; ++aa) {
                T sa = T(0);
                for (int bb = 0; bb < W2; ++bb) {
                    const T *row = bt + ((lc[0] + aa) * TW + (lc[1] + bb)) * TW + lc[2];
                    T sb = T(0);
#pragma unroll
                    for (int cc = 0; cc < W2; ++cc) sb = fma(row[cc], wt[2][cc], sb);
                    sa = fma(wt[1][bb], sb, sa);
                }
                T wxa = wt[0][0];
#pragma unroll
                for (int k = 1; k < W2; ++k)
                    if (k == aa) wxa = wt[0][k];
                f = fma(wxa, sa, f);
            }
        } else if (DW == 2) {
#pragma unroll
            for (int aa = 0; aa < W2; ++aa) {
                const T *row = bt + (lc[0] + aa) * TW + lc[1];
                T sb = T(0);
#pragma unroll
                for (int cc = 0; cc < W2; ++cc) sb = fma(row[cc], wt[1][cc], sb);
                f = fma(wt[0][aa], sb, f);
            }
        } else {
#pragma unroll
            for (int cc = 0; cc < W2; ++cc) f = fma(bt[lc[0] + cc], wt[0][cc], f);
        }
        if (valid) out[a.perm[q]] = f;
    }
}

// ------------------------------------------------------------------ interpolation, direct reads
// One thread per point reading its (2M)^d grid block straight from the (L2-resident) grid. Used
// where staging a bin's neighbourhood costs more than it saves: the FP64 plan, whose bins hold
// few points (n_os = 128, B = 2) and whose FMA rate is low.
template <typename T>
struct InterpDirectArgs {
    const T *frac;
    const int *perm;
    const int4 *segs;
    const T *grid;
    const DevWindow *dwin;
    T *part;
    long long n, total, grid_stride_rhs;
    int nrhs, seg_begin, seg_end, n_os, part_w0;
    long long q_begin, q_end;  // sorted points of the windows handled
    WinParams wp;
};

template <typename T, int DW, int M>
__global__ void __launch_bounds__(128) k_interp_direct(InterpDirectArgs<T> a) {
    pdl_wait();
    pdl_trigger();
    constexpr int W2 = 2 * M;
    const int r = blockIdx.y;
    const long long q = a.q_begin + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= a.q_end) return;
    // the segment holding q gives its cell and window (binary search over segment starts)
    int lo = a.seg_begin, hi = a.seg_end - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.segs[mid].y <= q) lo = mid; else hi = mid - 1;
    }
    const int4 sg = a.segs[lo];
    const int w = sg.w;
    const DevWindow dw = a.dwin[w];
    const T *grid = a.grid + (size_t)r * a.grid_stride_rhs + dw.grid_off;
    int c0[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) c0[k] = cell_coord(sg.x, k) - M + 1;
    T wt[DW][W2];
#pragma unroll
    for (int k = 0; k < DW; ++k) Weights<T, M>::eval(a.frac[(size_t)k * a.total + q], a.wp, wt[k]);
    T f = T(0);
    if (DW == 3) {
        const long long n2 = (long long)a.n_os * a.n_os;
#pragma unroll 1
        for (int aa = 0; aa < W2; ++aa) {
            T sa = T(0);
            for (int bb = 0; bb < W2; ++bb) {
                const T *row = grid + (long long)(c0[0] + aa) * n2 + (long long)(c0[1] + bb) * a.n_os + c0[2];
                T sb = T(0);
#pragma unroll
                for (int cc = 0; cc < W2; ++cc) sb = fma(__ldg(row + cc), wt[2][cc], sb);
                sa = fma(wt[1][bb], sb, sa);
            }
            T wxa = wt[0][0];
#pragma unroll
            for (int k = 1; k < W2; ++k)
                if (k == aa) wxa = wt[0][k];
            f = fma(wxa, sa, f);
        }
    } else if (DW == 2) {
#pragma unroll
        for (int aa = 0; aa < W2; ++aa) {
            const T *row = grid + (long long)(c0[0] + aa) * a.n_os + c0[1];
            T sb = T(0);
#pragma unroll
            for (int cc = 0; cc < W2; ++cc) sb = fma(__ldg(row + cc), wt[1][cc], sb);
            f = fma(wt[0][aa], sb, f);
        }
    } else {
#pragma unroll
        for (int cc = 0; cc < W2; ++cc) f = fma(__ldg(grid + c0[0] + cc), wt[0][cc], f);
    }
    a.part[((size_t)(w - a.part_w0) * a.nrhs + r) * a.n + a.perm[q]] = f;
}

// ------------------------------------------------------------------ sum over windows
// Kv[r][j] = sum over windows w (in order) of part[w][r][j]; blockIdx.y = r. VEC = 4: four
// consecutive j per thread with 16-byte loads (n a multiple of 4 and Kv 16-byte aligned).
template <typename T, int VEC>
__global__ void k_window_sum(const T *__restrict__ part, T *__restrict__ Kv, long long n, int nrhs,
                             int P) {
    pdl_wait();
    pdl_trigger();
    const int r = blockIdx.y;
    const long long nv = n / VEC;
    T *out = Kv + (size_t)r * n;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nv;
         i += (long long)gridDim.x * blockDim.x) {
        if constexpr (VEC == 4) {
            float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int w = 0; w < P; ++w) {
                const float4 t = reinterpret_cast<const float4 *>(part + ((size_t)w * nrhs + r) * n)[i];
                s.x += t.x;
                s.y += t.y;
                s.z += t.z;
                s.w += t.w;
            }
            reinterpret_cast<float4 *>(out)[i] = s;
        } else {
            T s = T(0);
            for (int w = 0; w < P; ++w) s += part[((size_t)w * nrhs + r) * n + i];
            out[i] = s;
        }
    }
}

// Launches k_window_sum with 16-byte loads where the sizes and alignment allow it (FP32).
template <typename T>
cudaError_t launch_window_sum(const T *part, T *Kv, long long n, int nrhs, int P, cudaStream_t st) {
    auto blocks = [](long long items) {
        return (int)std::max<long long>(1, std::min<long long>((items + 255) / 256, 152LL * 8));
    };
    if constexpr (sizeof(T) == 4) {
        if (n % 4 == 0 && reinterpret_cast<uintptr_t>(Kv) % 16 == 0 && reinterpret_cast<uintptr_t>(part) % 16 == 0) {
            return launch_k(k_window_sum<T, 4>, dim3(blocks(n / 4), nrhs), dim3(256), 0, st, part, Kv, n, nrhs, P);
        }
    }
    return launch_k(k_window_sum<T, 1>, dim3(blocks(n), nrhs), dim3(256), 0, st, part, Kv, n, nrhs, P);
}

}  // namespace anova
