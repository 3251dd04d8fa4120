// Host-side launch sequence of one fast-summation matvec (spread -> reduce -> per-axis
// FFT/scale/IFFT -> interpolation -> window sum), templated on the element type.
#pragma once

#include <algorithm>
#include <type_traits>

#include "conv_kernels.cuh"
#include "nfft_kernels.cuh"
#include "pair_kernels.cuh"

namespace anova {

#ifndef ANOVA_SPREAD_WARPS
#define ANOVA_SPREAD_WARPS 8  // warps per CTA of the packed FP32 spread
#endif
// Work order knobs, both off: measured at n = 1e6 (three 3-D windows), largest-first spread CTAs
// made the spread 2 % slower and the group-wide order changed the interpolation by under 1 %.
#ifndef ANOVA_SPREAD_ORDER
#define ANOVA_SPREAD_ORDER 0  // packed spread: CTAs take work items largest first
#endif
#ifndef ANOVA_GROUP_ORDER
#define ANOVA_GROUP_ORDER 0   // largest-first order over a whole dimension group (else per window)
#endif
constexpr int kAuxStreams = 3;           // concurrent window chains of one matvec
#ifndef ANOVA_INTERP_VARIANT
// FP32 3-D interpolation with m = 4: 2 = tensor cores where chosen, 0 = always one point per lane
#define ANOVA_INTERP_VARIANT 2
#endif
#ifndef ANOVA_SPREAD_LPP
#define ANOVA_SPREAD_LPP 32  // lanes per point in the packed FP32 spread (16 or 32)
#endif

template <typename T>
struct Prec;
template <>
struct Prec<float> {
    static constexpr int B = kBinF32;
    static constexpr int SPREAD_WARPS = ANOVA_SPREAD_WARPS;
    static constexpr int INTERP_WARPS = 8;
};
#ifndef ANOVA_F64_SPREAD_WARPS
#define ANOVA_F64_SPREAD_WARPS 4
#endif
template <>
struct Prec<double> {
    static constexpr int B = kBinF64;
    static constexpr int SPREAD_WARPS = ANOVA_F64_SPREAD_WARPS;
    static constexpr int INTERP_WARPS = 4;
};

#ifndef ANOVA_F64_PAIR
#define ANOVA_F64_PAIR 1  // FP64 3-D spread and interpolation: multiply-adds in FP32 pairs
#endif

template <typename T, int DW, int M>
cudaError_t launch_spread_t(const SpreadArgs &a, int nblocks, int nrhs, cudaStream_t st) {
    constexpr int B = Prec<T>::B, NW = Prec<T>::SPREAD_WARPS;
    using C = SpreadCfg<T, DW, M, B, NW>;
    if constexpr (sizeof(T) == 8 && DW == 3 && ANOVA_F64_PAIR) {
        auto kp = k_spread3_pair<M, B, NW>;
        static const cudaError_t configured_p =
            cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
        if (configured_p != cudaSuccess) return configured_p;
        return launch_k(kp, dim3(nblocks, nrhs), dim3(NW * 32), C::smem, st, a);
    }
    auto kern = k_spread<T, DW, M, B, NW>;
    static const cudaError_t configured =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
    if (configured != cudaSuccess) return configured;
    return launch_k(kern, dim3(nblocks, nrhs), dim3(NW * 32), C::smem, st, a);
}

template <typename T, int DW, int M>
cudaError_t launch_interp_t(const InterpArgs &a, int nseg, int nrhs, cudaStream_t st) {
    constexpr int NW = Prec<T>::INTERP_WARPS;
    using C = InterpCfg<T, DW, M, NW>;
    auto kern = k_interp<T, DW, M, NW>;
    static const cudaError_t configured =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
    if (configured != cudaSuccess) return configured;
    return launch_k(kern, dim3((nseg + NW - 1) / NW, nrhs), dim3(NW * 32), C::smem, st, a);
}

#ifndef ANOVA_F64_PAIR_FFT
#define ANOVA_F64_PAIR_FFT 1  // FP64 grids: FFT passes in FP32 pairs
#endif
template <typename T>
struct ConvArith {
    using type = T;
};
template <>
struct ConvArith<double> {
    using type = std::conditional_t<ANOVA_F64_PAIR_FFT != 0, pf, double>;
};

template <typename T, int NOS, int DW, int LINES>
cudaError_t launch_conv_t(const ConvArgs &a, int ntiles, int nrhs, cudaStream_t st) {
    using C = ConvCfg<T, NOS, LINES>;
    auto kern = k_conv<T, NOS, DW, LINES, typename ConvArith<T>::type>;
    static const cudaError_t configured =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
    if (configured != cudaSuccess) return configured;
    return launch_k(kern, dim3(ntiles, nrhs), dim3(256), C::smem, st, a);
}

// CTAs of `kern` (threads per CTA, dynamic shared memory) that fit on one SM at once, from its
// registers and shared memory, at most `cap`
template <typename K>
cudaError_t resident_ctas(K kern, int threads, size_t smem, int cap, int *out) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    int dev = 0, regs_sm = 0, smem_sm = 0, smem_res = 0, thr_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_res, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    const int by_regs = regs_sm / std::max(1, (fa.numRegs + 7) / 8 * 8 * threads);
    const int by_smem = smem_sm / std::max(1, (int)(smem + fa.sharedSizeBytes) + smem_res);
    const int by_thr = thr_sm / std::max(1, threads);
    *out = std::max(1, std::min(std::min(std::min(by_regs, by_smem), by_thr), cap));
    return cudaSuccess;
}

template <int M, int LPP>
cudaError_t launch_spread3_x2(const SpreadArgs &a, int nblocks, int nrhs, cudaStream_t st) {
    constexpr int B = Prec<float>::B, NW = Prec<float>::SPREAD_WARPS;
    using C = SpreadX2Cfg<M, B, NW, LPP>;
    auto kern = k_spread3_x2<M, B, NW, LPP>;
    static const cudaError_t configured =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
    if (configured != cudaSuccess) return configured;
    return launch_k(kern, dim3(nblocks, nrhs), dim3(NW * 32), C::smem, st, a);
}

template <int M>
cudaError_t launch_interp3_x2(const InterpWiArgs &a, int nblocks, int nrhs, cudaStream_t st) {
    constexpr int B = Prec<float>::B, NW = Prec<float>::INTERP_WARPS;
    using C = InterpX2Cfg<M, B, NW>;
    auto kern = k_interp3_x2<M, B, NW>;
    static const cudaError_t configured =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
    if (configured != cudaSuccess) return configured;
    return launch_k(kern, dim3(nblocks, nrhs), dim3(NW * 32), C::smem, st, a);
}

template <int M, bool PARAM_WAIT>
cudaError_t launch_interp3_tc_t(const InterpWiArgs &a, int nwork, int nrhs, int sm_count, cudaStream_t st) {
    using C = InterpTcCfg<M, Prec<float>::B>;
    auto kern = k_interp3_tc<M, Prec<float>::B, PARAM_WAIT>;
    static const cudaError_t configured =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
    if (configured != cudaSuccess) return configured;
    // resident CTAs per SM, capped by tensor memory (512 columns per SM): a CTA beyond the cap
    // would wait in its allocation until others exit
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaError_t e = resident_ctas(kern, 128, C::smem, (int)(512 / C::TMEM_COLS), &per_sm);
        if (e != cudaSuccess) return e;
    }
    // persistent CTAs take work items from the per-RHS counters a.counters[r] (zero at every
    // launch: the kernel's last CTA resets them)
    const int nblocks = std::max(1, std::min(nwork, per_sm * std::max(sm_count, 1)));
    return launch_k(kern, dim3(nblocks, nrhs), dim3(128), C::smem, st, a);
}

template <int M>
cudaError_t launch_interp3_tc(const InterpWiArgs &a, int nwork, int nrhs, int sm_count, cudaStream_t st) {
    return a.wait_polls == InterpTcCfg<M, Prec<float>::B>::kMaxPolls
               ? launch_interp3_tc_t<M, false>(a, nwork, nrhs, sm_count, st)
               : launch_interp3_tc_t<M, true>(a, nwork, nrhs, sm_count, st);
}

template <typename T, int DW, int M>
cudaError_t launch_interp_bin_t(const InterpBinArgs<T> &a, int nblocks, int nrhs, cudaStream_t st) {
    constexpr int B = Prec<T>::B, NW = 4;
    using C = InterpBinCfg<T, DW, M, B, NW>;
    auto kern = k_interp_bin<T, DW, M, B, NW>;
    static const cudaError_t configured =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
    if (configured != cudaSuccess) return configured;
    return launch_k(kern, dim3(nblocks, nrhs), dim3(NW * 32), C::smem, st, a);
}

template <typename T, int DW>
cudaError_t dispatch_interp_bin_m(int m, const InterpBinArgs<T> &a, int nb, int nrhs, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        switch (m) {
            case 2: return launch_interp_bin_t<T, DW, 2>(a, nb, nrhs, st);
            case 3: return launch_interp_bin_t<T, DW, 3>(a, nb, nrhs, st);
            case 4: return launch_interp_bin_t<T, DW, 4>(a, nb, nrhs, st);
            case 5: return launch_interp_bin_t<T, DW, 5>(a, nb, nrhs, st);
            case 6: return launch_interp_bin_t<T, DW, 6>(a, nb, nrhs, st);
        }
    } else {
        switch (m) {
            case 3: return launch_interp_bin_t<T, DW, 3>(a, nb, nrhs, st);
            case 4: return launch_interp_bin_t<T, DW, 4>(a, nb, nrhs, st);
            case 5: return launch_interp_bin_t<T, DW, 5>(a, nb, nrhs, st);
            case 6: return launch_interp_bin_t<T, DW, 6>(a, nb, nrhs, st);
        }
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t dispatch_interp_bin(int dw, int m, const InterpBinArgs<T> &a, int nb, int nrhs, cudaStream_t st) {
    switch (dw) {
        case 1: return dispatch_interp_bin_m<T, 1>(m, a, nb, nrhs, st);
        case 2: return dispatch_interp_bin_m<T, 2>(m, a, nb, nrhs, st);
        case 3: return dispatch_interp_bin_m<T, 3>(m, a, nb, nrhs, st);
    }
    return cudaErrorInvalidValue;
}

template <typename T, int DW>
cudaError_t dispatch_interp_direct_m(int m, const InterpDirectArgs<T> &a, int nrhs, cudaStream_t st) {
    const long long cnt = a.q_end - a.q_begin;
    const dim3 grid((unsigned)((cnt + 127) / 128), nrhs);
    switch (m) {
        case 3: return launch_k(k_interp_direct<T, DW, 3>, grid, dim3(128), 0, st, a);
        case 4: return launch_k(k_interp_direct<T, DW, 4>, grid, dim3(128), 0, st, a);
        case 5: return launch_k(k_interp_direct<T, DW, 5>, grid, dim3(128), 0, st, a);
        case 6: return launch_k(k_interp_direct<T, DW, 6>, grid, dim3(128), 0, st, a);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t dispatch_interp_direct(int dw, int m, const InterpDirectArgs<T> &a, int nrhs, cudaStream_t st) {
    switch (dw) {
        case 1: return dispatch_interp_direct_m<T, 1>(m, a, nrhs, st);
        case 2: return dispatch_interp_direct_m<T, 2>(m, a, nrhs, st);
        case 3: return dispatch_interp_direct_m<T, 3>(m, a, nrhs, st);
    }
    return cudaErrorInvalidValue;
}

// the FP32 3-D paths with a packed kernel (footprint edge 2m divides 16)
inline bool packed_path(int prec_bytes, int dw, int m) { return prec_bytes == 4 && dw == 3 && (m == 2 || m == 4); }

// runtime (dw, m) -> template dispatch
template <typename T, int DW>
cudaError_t dispatch_spread_m(int m, const SpreadArgs &a, int nb, int nrhs, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        switch (m) {
            case 2: return launch_spread_t<T, DW, 2>(a, nb, nrhs, st);
            case 3: return launch_spread_t<T, DW, 3>(a, nb, nrhs, st);
            case 4: return launch_spread_t<T, DW, 4>(a, nb, nrhs, st);
            case 5: return launch_spread_t<T, DW, 5>(a, nb, nrhs, st);
            case 6: return launch_spread_t<T, DW, 6>(a, nb, nrhs, st);
        }
    } else {
        switch (m) {
            case 3: return launch_spread_t<T, DW, 3>(a, nb, nrhs, st);
            case 4: return launch_spread_t<T, DW, 4>(a, nb, nrhs, st);
            case 5: return launch_spread_t<T, DW, 5>(a, nb, nrhs, st);
            case 6: return launch_spread_t<T, DW, 6>(a, nb, nrhs, st);
        }
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t dispatch_spread(int dw, int m, const SpreadArgs &a, int nb, int nrhs, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        // the packed kernel reads v in sorted order; callers without that copy use the generic one
        if (a.packed && dw == 3 && m == 4) return launch_spread3_x2<4, ANOVA_SPREAD_LPP>(a, nb, nrhs, st);
        if (a.packed && dw == 3 && m == 2) return launch_spread3_x2<2, 16>(a, nb, nrhs, st);
    }
    switch (dw) {
        case 1: return dispatch_spread_m<T, 1>(m, a, nb, nrhs, st);
        case 2: return dispatch_spread_m<T, 2>(m, a, nb, nrhs, st);
        case 3: return dispatch_spread_m<T, 3>(m, a, nb, nrhs, st);
    }
    return cudaErrorInvalidValue;
}

template <typename T, int DW>
cudaError_t dispatch_interp_m(int m, const InterpArgs &a, int nseg, int nrhs, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        switch (m) {
            case 2: return launch_interp_t<T, DW, 2>(a, nseg, nrhs, st);
            case 3: return launch_interp_t<T, DW, 3>(a, nseg, nrhs, st);
            case 4: return launch_interp_t<T, DW, 4>(a, nseg, nrhs, st);
            case 5: return launch_interp_t<T, DW, 5>(a, nseg, nrhs, st);
            case 6: return launch_interp_t<T, DW, 6>(a, nseg, nrhs, st);
        }
    } else {
        switch (m) {
            case 3: return launch_interp_t<T, DW, 3>(a, nseg, nrhs, st);
            case 4: return launch_interp_t<T, DW, 4>(a, nseg, nrhs, st);
            case 5: return launch_interp_t<T, DW, 5>(a, nseg, nrhs, st);
            case 6: return launch_interp_t<T, DW, 6>(a, nseg, nrhs, st);
        }
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t dispatch_interp(int dw, int m, const InterpArgs &a, int nseg, int nrhs,
                            cudaStream_t st) {
    switch (dw) {
        case 1: return dispatch_interp_m<T, 1>(m, a, nseg, nrhs, st);
        case 2: return dispatch_interp_m<T, 2>(m, a, nseg, nrhs, st);
        case 3: return dispatch_interp_m<T, 3>(m, a, nseg, nrhs, st);
    }
    return cudaErrorInvalidValue;
}

template <typename T, int NOS, int LINES>
cudaError_t dispatch_conv_dw(int dw, const ConvArgs &a, int nt, int nrhs, cudaStream_t st) {
    switch (dw) {
        case 1: return launch_conv_t<T, NOS, 1, LINES>(a, nt, nrhs, st);
        case 2: return launch_conv_t<T, NOS, 2, LINES>(a, nt, nrhs, st);
        case 3: return launch_conv_t<T, NOS, 3, LINES>(a, nt, nrhs, st);
    }
    return cudaErrorInvalidValue;
}

template <typename T, int NOS>
cudaError_t dispatch_conv_lines(int lines, int dw, const ConvArgs &a, int nt, int nrhs, cudaStream_t st) {
    switch (lines) {
        case 8: return dispatch_conv_dw<T, NOS, 8>(dw, a, nt, nrhs, st);
        case 16: return dispatch_conv_dw<T, NOS, 16>(dw, a, nt, nrhs, st);
        case 32: return dispatch_conv_dw<T, NOS, 32>(dw, a, nt, nrhs, st);
    }
    return cudaErrorInvalidValue;
}

// one FFT pass over the tiles [a.tile_begin, a.tile_end) of a tile table cut at `lines` grid
// lines per tile
template <typename T>
cudaError_t dispatch_conv(int n_os, int lines, int dw, const ConvArgs &a, int nt, int nrhs, cudaStream_t st) {
    switch (n_os) {
        case 32: return dispatch_conv_lines<T, 32>(lines, dw, a, nt, nrhs, st);
        case 64: return dispatch_conv_lines<T, 64>(lines, dw, a, nt, nrhs, st);
        case 128: return dispatch_conv_lines<T, 128>(lines, dw, a, nt, nrhs, st);
        case 256: return dispatch_conv_lines<T, 256>(lines, dw, a, nt, nrhs, st);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
WinParams make_winparams(const anova_plan *p) {
    WinParams wp{};
    for (int j = 0; j < 2 * p->m && j < 16; ++j)
        for (int q = 0; q <= kPolyDeg; ++q) wp.c[j][q] = (float)p->poly[(size_t)j * (kPolyDeg + 1) + q];
    for (int j = 0; j < p->m && j < 8; ++j)
        for (int q = 0; q <= kPolyDeg64; ++q) wp.c64[j][q] = p->poly64[(size_t)j * (kPolyDeg64 + 1) + q];
    wp.beta = kb_beta();
    wp.scale = p->m / std::sinh(wp.beta * p->m);
    return wp;
}

template <typename T>
int tile_volume(const anova_plan *p, int dw) {
    const int tw = Prec<T>::B + 2 * p->m - 1;
    int tv = 1;
    for (int k = 0; k < dw; ++k) tv *= tw;
    return tv;
}

// Partial tiles of windows [a0, a1) onto grid0: per-bin sums of multi-item bins, then the
// gather of bin tiles onto every grid point of the windows' boxes.
template <typename T>
anova_status launch_reduce(anova_plan *p, int dw, int a0, int a1, void *grid0, long long grid_stride,
                           int nrhs, int zero_offset, cudaStream_t st) {
    BinReduceArgs ba;
    ba.tiles = p->tiles;
    ba.mbins = p->mbins;
    ba.mb_begin = p->win[a0].mb_begin;
    ba.nmbins = p->win[a1 - 1].mb_end - ba.mb_begin;
    ba.nrhs = nrhs;
    ba.tv_max = tile_volume<T>(p, dw);
    if (ba.nmbins > 0) {
        const int chunks = (ba.tv_max + kBinReduceChunk - 1) / kBinReduceChunk;
        ANOVA_CUDA_TRY(launch_k(k_bin_reduce<T>, dim3(ba.nmbins * chunks, nrhs), dim3(256), 0, st, ba));
        p->launches += 1;
    }
    ReduceArgs ra;
    ra.tiles = p->tiles;
    ra.grid0 = grid0;
    ra.dwin = p->dwin;
    ra.bins = p->bins;
    ra.grid_total = grid_stride;
    ra.w_begin = a0;
    ra.w_end = a1;
    ra.nrhs = nrhs;
    ra.n_os = p->n_os;
    ra.NB = p->NB;
    ra.M = p->m;
    ra.B = Prec<T>::B;
    ra.zero_offset = zero_offset;
    ra.box_cum[0] = 0;
    for (int w = a0; w < a1; ++w) ra.box_cum[w - a0 + 1] = ra.box_cum[w - a0] + p->win[w].box_volume();
    const long long vol = ra.box_cum[a1 - a0];
    if (vol > 0) {
        const int nb = (int)((vol + 255) / 256);
        auto kr = dw == 3 ? k_reduce<T, 3> : dw == 2 ? k_reduce<T, 2> : k_reduce<T, 1>;
        ANOVA_CUDA_TRY(launch_k(kr, dim3(nb, nrhs), dim3(256), 0, st, ra));
        p->launches += 1;
    }
    return ANOVA_OK;
}

// Stage 4 of one group's windows [a0, a1): interpolation from the convolved grids `grid` (the
// layout of the plan's grid workspace) into the per-window results `part`.
template <typename T>
anova_status interp_stage(anova_plan *p, const Group &gr, int a0, int a1, int w0, const T *grid,
                          long long grid_stride, int nrhs, T *part, const WinParams &wp, cudaStream_t st,
                          int *counters, T *pair_scratch = nullptr) {
    const int wi0 = p->win[a0].wi_begin, wi1 = p->win[a1 - 1].wi_end;
    const int s0 = p->win[a0].seg_begin, s1 = p->win[a1 - 1].seg_end;
    const bool packed = packed_path((int)sizeof(T), gr.dw, p->m);
    const bool whole_group = a0 == gr.w_begin && a1 == gr.w_end;
    const int *order = whole_group && ANOVA_GROUP_ORDER ? p->wi_gorder : p->wi_order;
    if (packed && wi1 > wi0) {
        InterpWiArgs xa;
        xa.wis = p->wis;
        xa.segs = p->segs;
        xa.frac = reinterpret_cast<const float *>(p->frac);
        xa.perm = p->perm;
        xa.cellloc = p->cellloc;
        xa.grid = reinterpret_cast<const float *>(grid);
        xa.dwin = p->dwin;
        xa.part = reinterpret_cast<float *>(part);
        xa.n = p->n;
        xa.total = p->n * p->P;
        xa.grid_stride_rhs = grid_stride;
        xa.nrhs = nrhs;
        xa.wi_begin = wi0;
        xa.wi_end = wi1;
        xa.n_os = p->n_os;
        xa.part_w0 = w0;
        xa.wp = wp;
        xa.status = p->dev_status;
        xa.wait_polls = p->wait_polls;
        xa.counters = counters;
        xa.order = order;
        xa.chunks = p->chunks;
        xa.wi_chunk = p->wi_chunk;
        cudaError_t e;
        // the tensor-core form pays a fixed cost per work item and per chunk of up to 128
        // points; it is used when work items are well filled (large n), else the SIMT form
        const bool tc_fill = (p->interp_flags & ANOVA_INTERP_TENSOR) ||
                             (!(p->interp_flags & ANOVA_INTERP_SIMT) &&
                              (double)p->n * (a1 - a0) >= (double)kTcMinPointsPerItem * (wi1 - wi0));
        if (p->m == 4)
            e = ANOVA_INTERP_VARIANT == 2 && tc_fill ? launch_interp3_tc<4>(xa, wi1 - wi0, nrhs, p->sm_count, st)
                                                     : launch_interp3_x2<4>(xa, wi1 - wi0, nrhs, st);
        else
            e = launch_interp3_x2<2>(xa, wi1 - wi0, nrhs, st);
        if (e != cudaSuccess) return cuda_fail(e, "interp launch");
        p->launches += 1;
    } else if (sizeof(T) == 8 && s1 > s0) {
        InterpDirectArgs<T> da;
        da.frac = reinterpret_cast<const T *>(p->frac);
        da.perm = p->perm;
        da.segs = p->segs;
        da.grid = grid;
        da.dwin = p->dwin;
        da.part = part;
        da.n = p->n;
        da.total = p->n * p->P;
        da.grid_stride_rhs = grid_stride;
        da.nrhs = nrhs;
        da.seg_begin = s0;
        da.seg_end = s1;
        da.n_os = p->n_os;
        da.part_w0 = w0;
        da.q_begin = (long long)a0 * p->n;
        da.q_end = (long long)a1 * p->n;
        da.wp = wp;
        cudaError_t e = cudaSuccess;
        bool pair_done = false;
        if constexpr (sizeof(T) == 8) {
          if (ANOVA_F64_PAIR && gr.dw == 3 && pair_scratch && p->m >= 3 && p->m <= 6) {
            pair_done = true;
            // FP32-pair form: the windows' boxes as pairs in the scratch buffer, then the sums
            GridPairArgs ga;
            ga.grid = reinterpret_cast<const double *>(grid);
            ga.pairs = reinterpret_cast<fpair *>(pair_scratch);
            ga.dwin = p->dwin;
            ga.grid_stride = grid_stride;
            ga.w_begin = a0;
            ga.w_end = a1;
            ga.n_os = p->n_os;
            ga.box_cum[0] = 0;
            for (int w = a0; w < a1; ++w) ga.box_cum[w - a0 + 1] = ga.box_cum[w - a0] + p->win[w].box_volume();
            const long long vol = ga.box_cum[a1 - a0];
            e = launch_k(k_grid_pairs<3>, dim3((unsigned)((vol + 255) / 256), nrhs), dim3(256), 0, st, ga);
            if (e == cudaSuccess) {
                p->launches += 1;
                const fpair *pg = reinterpret_cast<const fpair *>(pair_scratch);
                const dim3 grd((unsigned)((da.q_end - da.q_begin + 127) / 128), nrhs);
                switch (p->m) {
                    case 3: e = launch_k(k_interp_pair<3>, grd, dim3(128), 0, st, da, pg); break;
                    case 4: e = launch_k(k_interp_pair<4>, grd, dim3(128), 0, st, da, pg); break;
                    case 5: e = launch_k(k_interp_pair<5>, grd, dim3(128), 0, st, da, pg); break;
                    default: e = launch_k(k_interp_pair<6>, grd, dim3(128), 0, st, da, pg); break;
                }
            }
          }
        }
        if (!pair_done) e = dispatch_interp_direct<T>(gr.dw, p->m, da, nrhs, st);
        if (e != cudaSuccess) return cuda_fail(e, "interp launch");
        p->launches += 1;
    } else if (wi1 > wi0) {
        InterpBinArgs<T> ba;
        ba.wis = p->wis;
        ba.segs = p->segs;
        ba.frac = reinterpret_cast<const T *>(p->frac);
        ba.perm = p->perm;
        ba.cellloc = p->cellloc;
        ba.grid = grid;
        ba.dwin = p->dwin;
        ba.part = part;
        ba.n = p->n;
        ba.total = p->n * p->P;
        ba.grid_stride_rhs = grid_stride;
        ba.nrhs = nrhs;
        ba.wi_begin = wi0;
        ba.wi_end = wi1;
        ba.n_os = p->n_os;
        ba.part_w0 = w0;
        ba.wp = wp;
        cudaError_t e = dispatch_interp_bin<T>(gr.dw, p->m, ba, wi1 - wi0, nrhs, st);
        if (e != cudaSuccess) return cuda_fail(e, "interp launch");
        p->launches += 1;
    }
    return ANOVA_OK;
}

// One matvec over the window range [w0, w1) (all groups intersecting it). `part` receives
// per-window results in original point order; grids g[0..3] are the workspace buffers.
template <typename T>
anova_status matvec_windows(anova_plan *p, const T *v, int nrhs, int w0, int w1, T *part,
                            T *const g[4], long long grid_stride, cudaStream_t st, int *counters) {
    const WinParams wp = make_winparams<T>(p);
    for (const Group &gr : p->groups) {
        const int a0 = std::max(gr.w_begin, w0), a1 = std::min(gr.w_end, w1);
        if (a0 >= a1) continue;
        const int wi0 = p->win[a0].wi_begin, wi1 = p->win[a1 - 1].wi_end;
        const int s0 = p->win[a0].seg_begin, s1 = p->win[a1 - 1].seg_end;
        const bool packed = packed_path((int)sizeof(T), gr.dw, p->m);
        cudaEvent_t e0 = stage_event(p);
        // 1. spread into partial tiles
        SpreadArgs sa;
        sa.packed = packed ? 1 : 0;
        sa.wis = p->wis;
        sa.segs = p->segs;
        sa.frac = p->frac;
        sa.perm = p->perm;
        sa.v = v;
        sa.tiles = p->tiles;
        sa.n = p->n;
        sa.total = p->n * p->P;
        sa.nrhs = nrhs;
        sa.wi_begin = wi0;
        sa.wi_end = wi1;
        sa.wp = wp;
        // largest work items first: over the whole group when the launch covers it
        const bool whole_group = a0 == gr.w_begin && a1 == gr.w_end;
        const int *order = whole_group && ANOVA_GROUP_ORDER ? p->wi_gorder : p->wi_order;
        sa.order = ANOVA_SPREAD_ORDER ? order : nullptr;
        sa.wsplit = p->wsplit;
        sa.wsplit_n = kSpreadSplit;
        if (wi1 > wi0) {
            cudaError_t e = dispatch_spread<T>(gr.dw, p->m, sa, wi1 - wi0, nrhs, st);
            if (e != cudaSuccess) return cuda_fail(e, "spread launch");
            p->launches += 1;
        }
        cudaEvent_t e1 = stage_event(p);
        stage_record(p, STAGE_SPREAD, e0, e1);
        // 2. reduce partial tiles onto the grid boxes
        {
            anova_status rs = launch_reduce<T>(p, gr.dw, a0, a1, g[0], grid_stride, nrhs, 0, st);
            if (rs != ANOVA_OK) return rs;
        }
        cudaEvent_t e2 = stage_event(p);
        stage_record(p, STAGE_REDUCE, e1, e2);
        // 3. axis passes: g0 -> g1 -> g2 -> g3 (the last pass always writes g3)
        for (int pass = 0; pass < gr.dw; ++pass) {
            ConvArgs ca;
            ca.tiles = p->ftiles;
            ca.in = pass == 0 ? g[0] : g[pass];
            ca.out = pass == gr.dw - 1 ? g[3] : g[pass + 1];
            ca.D1br = p->D1br;
            ca.tw = p->tw;
            ca.dwin = p->dwin;
            ca.grid_stride_rhs = grid_stride;
            ca.tile_begin = p->win[a0].tile_begin[pass];
            ca.tile_end = p->win[a1 - 1].tile_end[pass];
            ca.zero_offset = 0;
            const int nt = ca.tile_end - ca.tile_begin;
            if (nt > 0) {
                cudaError_t e = dispatch_conv<T>(p->n_os, p->conv_lines, gr.dw, ca, nt, nrhs, st);
                if (e != cudaSuccess) return cuda_fail(e, "conv launch");
                p->launches += 1;
            }
        }
        cudaEvent_t e3 = stage_event(p);
        stage_record(p, STAGE_FFT, e2, e3);
        // 4. interpolation
        {
            // g[0] is free once the first pass has read it (3-D windows: g0 -> g1 -> g2 -> g3)
            anova_status is = interp_stage<T>(p, gr, a0, a1, w0, g[3], grid_stride, nrhs, part, wp, st, counters,
                                              gr.dw == 3 ? g[0] : nullptr);
            if (is != ANOVA_OK) return is;
        }
        cudaEvent_t e4 = stage_event(p);
        stage_record(p, STAGE_INTERP, e3, e4);
    }
    return ANOVA_OK;
}

template <typename T>
anova_status matvec_impl(anova_plan *p, const T *v, T *Kv, int nrhs, int only_window) {
    const int chunk = std::min(nrhs, std::max(1, std::min(16, p->rhs_chunk)));
    anova_status st = ensure_workspace(p, chunk);
    if (st != ANOVA_OK) return st;
    T *grids = reinterpret_cast<T *>(p->grids);
    const long long gs = p->grid_total;
    T *g[4];
    for (int k = 0; k < 4; ++k) g[k] = grids + (size_t)k * p->ws_rhs * gs;
    T *part = reinterpret_cast<T *>(p->part);
    // FP64 plans run their windows concurrently on the plan's auxiliary streams (forked from the
    // plan stream and joined back): their stages are long, latency-bound launches per window
    // (measured: 1.94 -> 1.82 ms at n = 7814, three windows). FP32 stages are single launches over
    // all windows that already fill the GPU, and forking them measured slower. Stage timing needs
    // one stream.
    const bool fork = sizeof(T) == 8 && p->fork_windows && p->aux[0] && !p->timing && only_window < 0 && p->P >= 2;
    for (int r0 = 0; r0 < nrhs; r0 += chunk) {
        const int nr = std::min(chunk, nrhs - r0);
        const T *vr = v + (size_t)r0 * p->n;
        T *kr = Kv + (size_t)r0 * p->n;
        if (only_window >= 0) {
            // the single window's result goes straight to Kv (part_w0 = only_window)
            st = matvec_windows<T>(p, vr, nr, only_window, only_window + 1, kr, g, gs, p->stream,
                                   p->dev_status + 1);
            if (st != ANOVA_OK) return st;
            continue;
        }
        if (fork) {
            // groups (window dimensions) one after another: partial tiles of different
            // dimensions share workspace under different strides; windows of one group are
            // independent and run concurrently
            for (const Group &gr : p->groups) {
                const int nw = gr.w_end - gr.w_begin;
                if (nw <= 0) continue;
                const int na = std::min(nw, kAuxStreams);
                ANOVA_CUDA_TRY(cudaEventRecord(p->fork_evt, p->stream));
                for (int k = 0; k < na; ++k) ANOVA_CUDA_TRY(cudaStreamWaitEvent(p->aux[k], p->fork_evt, 0));
                for (int w = gr.w_begin; w < gr.w_end; ++w) {
                    const int k = (w - gr.w_begin) % kAuxStreams;
                    st = matvec_windows<T>(p, vr, nr, w, w + 1, part + (size_t)w * nr * p->n, g, gs, p->aux[k],
                                           p->dev_status + 1 + kStatusCounters * k);
                    if (st != ANOVA_OK) return st;
                }
                for (int k = 0; k < na; ++k) {
                    ANOVA_CUDA_TRY(cudaEventRecord(p->join_evt[k], p->aux[k]));
                    ANOVA_CUDA_TRY(cudaStreamWaitEvent(p->stream, p->join_evt[k], 0));
                }
            }
        } else {
            st = matvec_windows<T>(p, vr, nr, 0, p->P, part, g, gs, p->stream, p->dev_status + 1);
            if (st != ANOVA_OK) return st;
        }
        cudaEvent_t e0 = stage_event(p);
        ANOVA_CUDA_TRY(launch_window_sum<T>(part, kr, p->n, nr, p->P, p->stream));
        p->launches += 1;
        stage_record(p, STAGE_SUM, e0, stage_event(p));
    }
    return ANOVA_OK;
}

}  // namespace anova

namespace anova {

// Split matvec, first half: the spread (and tile reduction) of v onto every window's grid, for all
// nrhs columns, into grids[r][grid_total] (cleared first: the reduction writes only the box of
// this plan's footprints).
template <typename T>
anova_status grids_impl(anova_plan *p, const T *v, T *grids, int nrhs) {
    const int chunk = std::min(nrhs, std::max(1, std::min(16, p->rhs_chunk)));
    anova_status st = ensure_workspace(p, chunk);
    if (st != ANOVA_OK) return st;
    const long long gs = p->grid_total;
    ANOVA_CUDA_TRY(cudaMemsetAsync(grids, 0, sizeof(T) * (size_t)gs * nrhs, p->stream));
    const WinParams wp = make_winparams<T>(p);
    for (int r0 = 0; r0 < nrhs; r0 += chunk) {
        const int nr = std::min(chunk, nrhs - r0);
        for (const Group &gr : p->groups) {
            const int wi0 = p->win[gr.w_begin].wi_begin, wi1 = p->win[gr.w_end - 1].wi_end;
            SpreadArgs sa;
            sa.packed = packed_path((int)sizeof(T), gr.dw, p->m) ? 1 : 0;
            sa.wis = p->wis;
            sa.segs = p->segs;
            sa.frac = p->frac;
            sa.perm = p->perm;
            sa.v = v + (size_t)r0 * p->n;
            sa.tiles = p->tiles;
            sa.n = p->n;
            sa.total = p->n * p->P;
            sa.nrhs = nr;
            sa.wi_begin = wi0;
            sa.wi_end = wi1;
            sa.wp = wp;
            sa.order = ANOVA_SPREAD_ORDER ? p->wi_order : nullptr;
            sa.wsplit = p->wsplit;
            sa.wsplit_n = kSpreadSplit;
            if (wi1 > wi0) {
                cudaError_t e = dispatch_spread<T>(gr.dw, p->m, sa, wi1 - wi0, nr, p->stream);
                if (e != cudaSuccess) return cuda_fail(e, "spread launch");
                p->launches += 1;
            }
            st = launch_reduce<T>(p, gr.dw, gr.w_begin, gr.w_end, grids + (size_t)r0 * gs, gs, nr, 0, p->stream);
            if (st != ANOVA_OK) return st;
        }
    }
    return ANOVA_OK;
}

// Split matvec, second half: every window's grid of `grids` convolved over the whole grid (FFT,
// scaling, inverse FFT: the summed grid is not confined to this plan's box), interpolated at the
// plan's points and summed over windows into Kv.
template <typename T>
anova_status from_grids_impl(anova_plan *p, const T *grids, T *Kv, int nrhs) {
    const int chunk = std::min(nrhs, std::max(1, std::min(16, p->rhs_chunk)));
    anova_status st = ensure_workspace(p, chunk);
    if (st != ANOVA_OK) return st;
    const long long gs = p->grid_total;
    T *ws = reinterpret_cast<T *>(p->grids);
    T *g[4];
    for (int k = 0; k < 4; ++k) g[k] = ws + (size_t)k * p->ws_rhs * gs;
    T *part = reinterpret_cast<T *>(p->part);
    const WinParams wp = make_winparams<T>(p);
    for (int r0 = 0; r0 < nrhs; r0 += chunk) {
        const int nr = std::min(chunk, nrhs - r0);
        for (const Group &gr : p->groups) {
            for (int pass = 0; pass < gr.dw; ++pass) {
                ConvArgs ca;
                ca.tiles = p->ftiles_full;
                ca.in = pass == 0 ? (const void *)(grids + (size_t)r0 * gs) : (const void *)g[pass];
                ca.out = pass == gr.dw - 1 ? g[3] : g[pass + 1];
                ca.D1br = p->D1br;
                ca.tw = p->tw;
                ca.dwin = p->dwin;
                ca.grid_stride_rhs = gs;
                ca.tile_begin = p->win[gr.w_begin].full_begin[pass];
                ca.tile_end = p->win[gr.w_end - 1].full_end[pass];
                ca.zero_offset = 0;
                const int nt = ca.tile_end - ca.tile_begin;
                if (nt > 0) {
                    cudaError_t e = dispatch_conv<T>(p->n_os, p->conv_lines, gr.dw, ca, nt, nr, p->stream);
                    if (e != cudaSuccess) return cuda_fail(e, "conv launch");
                    p->launches += 1;
                }
            }
            st = interp_stage<T>(p, gr, gr.w_begin, gr.w_end, 0, g[3], gs, nr, part, wp, p->stream,
                                 p->dev_status + 1, g[0]);
            if (st != ANOVA_OK) return st;
        }
        ANOVA_CUDA_TRY(launch_window_sum<T>(part, Kv + (size_t)r0 * p->n, p->n, nr, p->P, p->stream));
        p->launches += 1;
    }
    return ANOVA_OK;
}

}  // namespace anova
