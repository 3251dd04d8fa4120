// Spread (adjoint-NFFT step), tile reduction, gather interpolation (NFFT step) and window sum
// of the ANOVA fast summation (arXiv 2312.00538, Sec. 3: inner sum over i, outer sum over J).
//
// Points of every window are sorted by cell, cells grouped into bins of B^d cells. A spread
// work item is a run of one bin's cells (at most kWiMax points). Each warp of the work item's
// CTA accumulates its share of points cell by cell: lanes own rows of the (2M)^d footprint of
// the current cell in registers, the window weights of 32 points at a time are staged in shared
// memory and broadcast, and the footprint is added into the warp's own tile of the bin
// neighbourhood ((B + 2M - 1)^d cells) -- no atomics anywhere. The CTA then sums its warp
// tiles and writes one partial tile per work item; a reduction kernel adds the (at most 3^d
// bins x work items) partial tiles covering each grid point in a fixed order, so the grid is
// bit-for-bit reproducible.
#pragma once

#include "kernels_common.cuh"

namespace anova {

struct SpreadArgs {
    const int4 *wis;        // {window, seg_begin, seg_end, bin packed}
    const int4 *segs;       // {cell packed, sorted start, count, window}
    const void *frac;       // T[3][total]
    const int *perm;        // [total]
    const void *v;          // T[nrhs][n]
    void *tiles;            // T[nwi][nrhs][TV]
    long long n, total;
    int nrhs, wi_begin, wi_end;
    WinParams wp;
};

template <typename T, int DW, int M, int B, int NWARP>
struct SpreadCfg {
    using G = Geo<DW, M>;
    static constexpr int TW = B + 2 * M - 1;
    static constexpr int TV = ipow(TW, DW);
    static constexpr int TVP = (TV + 3) / 4 * 4;
    static constexpr size_t smem = sizeof(T) * ((size_t)NWARP * TVP + (size_t)NWARP * 32 * G::PSTRIDE);
};

template <typename T, int DW, int M, int B, int NWARP>
__global__ void __launch_bounds__(NWARP * 32) k_spread(SpreadArgs a) {
    using C = SpreadCfg<T, DW, M, B, NWARP>;
    using G = typename C::G;
    constexpr int W2 = G::W2, RPL = G::RPL, WS = G::WS, PS = G::PSTRIDE, TW = C::TW;
    constexpr int RCH = RPL < 2 ? RPL : 2;  // rows per lane held in registers at once
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *tiles_s = reinterpret_cast<T *>(smem_raw);
    T *wts_s = tiles_s + NWARP * C::TVP;

    const int wi_idx = a.wi_begin + blockIdx.x;
    if (wi_idx >= a.wi_end) return;
    const int r = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int4 wi = a.wis[wi_idx];
    const int bin_packed = wi.w;
    int bin[3] = {cell_coord(bin_packed, 0), cell_coord(bin_packed, 1), cell_coord(bin_packed, 2)};

    for (int i = threadIdx.x; i < NWARP * C::TVP; i += NWARP * 32) tiles_s[i] = T(0);
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
                if (lane < cnt) {
                    const int q = qb + lane;
                    const T vv = vr[a.perm[q]];
                    T w[W2];
#pragma unroll
                    for (int k = 0; k < DW; ++k) {
                        Weights<T, M>::eval(frac[(size_t)k * a.total + q], a.wp, w);
                        if (k == DW - 1) {
#pragma unroll
                            for (int j = 0; j < W2; ++j) w[j] *= vv;
                        }
#pragma unroll
                        for (int j = 0; j < W2; ++j) wts[lane * PS + k * WS + j] = w[j];
                    }
                }
                __syncwarp();
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

// ------------------------------------------------------------------ work-item tiles -> bin tile
// A bin split into several work items has several partial tiles; they are summed, in work-item
// order, into the slot of the bin's first work item, so the grid gather reads one tile per bin.
struct BinReduceArgs {
    void *tiles;
    const int4 *mbins;           // {first work item, count, tile volume, 0} of multi-item bins
    int nmbins, nrhs, mb_begin;
};

template <typename T>
__global__ void __launch_bounds__(256) k_bin_reduce(BinReduceArgs a) {
    const int b = a.mb_begin + blockIdx.x;
    const int r = blockIdx.y;
    if (b >= a.mb_begin + a.nmbins) return;
    const int4 mb = a.mbins[b];
    const int tv = mb.z;
    T *tiles = reinterpret_cast<T *>(a.tiles);
    for (int e = threadIdx.x; e < tv; e += blockDim.x) {
        T acc[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = T(0);
        int k = 0;
        for (; k + 8 <= mb.y; k += 8) {
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u] += tiles[((size_t)(mb.x + k + u) * a.nrhs + r) * tv + e];
        }
        for (int u = 0; k + u < mb.y; ++u) acc[u] += tiles[((size_t)(mb.x + k + u) * a.nrhs + r) * tv + e];
        T s = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
        tiles[((size_t)mb.x * a.nrhs + r) * tv + e] = s;
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
#pragma unroll
                for (int bb = 0; bb < W2; ++bb) {
                    T row[W2];
                    lds_vec<T, W2>(plane + bb * W2, row);
                    T sb = T(0);
#pragma unroll
                    for (int cc = 0; cc < W2; ++cc) sb = fma(row[cc], wt[2][cc], sb);
                    sa = fma(wt[1][bb], sb, sa);
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

// ------------------------------------------------------------------ sum over windows
template <typename T>
__global__ void k_window_sum(const T *__restrict__ part, T *__restrict__ Kv, long long n, int nrhs,
                             int P) {
    const long long total = n * nrhs;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / n, j = i - r * n;
        T s = T(0);
        for (int w = 0; w < P; ++w) s += part[((size_t)w * nrhs + r) * n + j];
        Kv[i] = s;
    }
}

}  // namespace anova
