// Fused "FFT -> diagonal scaling -> inverse FFT" along one grid axis (arXiv 2312.00538, Sec. 3:
// the Fourier coefficients b_J scale the adjoint-NFFT output before the NFFT).
//
// The scaling D_J = prod_k b_{J_k} / Psi(J_k)^2 is a tensor product and the d-dimensional DFT is
// a tensor product of 1-D DFTs, so F^H diag(D) F = (x)_k F_1^H diag(D_1) F_1 applied axis by
// axis. One launch handles one axis for all windows of a group: a CTA stages 32 grid lines of
// n_os points in shared memory (coalesced), each warp transforms two real lines packed as one
// complex line held in registers (n_os / 32 values per lane), with a radix-2 decimation-in-
// frequency FFT whose short spans run through warp shuffles; the output is left in bit-reversed
// order, scaled by D_1 stored in the same order, and brought back by the mirror-image
// decimation-in-time inverse with conjugate twiddles. Because D_1 is real and even, the packed
// real and imaginary parts stay separate. The inverse is unnormalised, as the fast summation
// needs.
#pragma once

#include "kernels_common.cuh"
#include "pair_arith.cuh"

namespace anova {

struct ConvArgs {
    const int4 *tiles;       // {window, p, q0, axis}
    const void *in;
    void *out;
    const void *D1br;        // T[P][3][n_os]: per window and axis, bit-reversed (eta in axis 0)
    const void *tw;          // T[n_os]: (cos, sin)(-2 pi k / n_os), k < n_os / 2
    const DevWindow *dwin;
    long long grid_stride_rhs;
    int tile_begin, tile_end;
    int zero_offset;         // 1: in/out are one window's grids (ignore the grid offset)
};

__device__ __forceinline__ float flip_sign(float x) { return __int_as_float(__float_as_int(x) ^ 0x80000000); }
__device__ __forceinline__ double flip_sign(double x) {
    return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
}

template <typename T, int NOS>
__device__ __forceinline__ void conv_line(T (&re)[NOS / 32], T (&im)[NOS / 32], const T *twr,
                                          const T *twi, const T *d1, int lane) {
    constexpr int VPL = NOS / 32;
    // forward DIF
#pragma unroll
    for (int h = NOS / 2; h >= 1; h >>= 1) {
        if (h >= 32) {
            const int hv = h / 32;
#pragma unroll
            for (int v = 0; v < VPL; ++v) {
                if ((v % (2 * hv)) < hv) {
                    const int vb = v + hv;
                    const int k = ((32 * v + lane) % (2 * h)) * (NOS / (2 * h));
                    const T wr = twr[k], wi = twi[k];
                    const T ar = re[v], ai = im[v], br = re[vb], bi = im[vb];
                    re[v] = ar + br;
                    im[v] = ai + bi;
                    const T dr = ar - br, di = ai - bi;
                    re[vb] = dr * wr - di * wi;
                    im[vb] = dr * wi + di * wr;
                }
            }
        } else {
            // both halves in one instruction stream: t = partner + s * own (s = +1 above, -1
            // below: a + b and a - b), then t * w with w = 1 above; at span 1 every twiddle is 1
            const bool top = (lane & h) == 0;
            const T sg = top ? T(1) : T(-1);
            const int k = ((lane & ~h) & (2 * h - 1)) * (NOS / (2 * h));
            const T wr = top ? T(1) : twr[k], wi = top ? T(0) : twi[k];
#pragma unroll
            for (int v = 0; v < VPL; ++v) {
                const T yr = __shfl_xor_sync(0xffffffffu, re[v], h);
                const T yi = __shfl_xor_sync(0xffffffffu, im[v], h);
                const T tr = fma(sg, re[v], yr), ti = fma(sg, im[v], yi);
                if (h == 1) {
                    re[v] = tr;
                    im[v] = ti;
                } else if (h == 2) {
                    // w is 1 or -i: t * (-i) = ti - i tr, by selection and a sign flip
                    const bool rot = !top && (lane & 1);
                    re[v] = rot ? ti : tr;
                    im[v] = rot ? flip_sign(tr) : ti;
                } else {
                    re[v] = tr * wr - ti * wi;
                    im[v] = tr * wi + ti * wr;
                }
            }
        }
    }
    // diagonal scaling (frequency bitrev(e) sits at position e)
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        const T dd = d1[32 * v + lane];
        re[v] *= dd;
        im[v] *= dd;
    }
    // inverse DIT with conjugate twiddles (unnormalised)
#pragma unroll
    for (int h = 1; h <= NOS / 2; h <<= 1) {
        if (h < 32) {
            // b * conj(w) below (w = 1 above, and everywhere at span 1), then partner + s * own
            const bool top = (lane & h) == 0;
            const T sg = top ? T(1) : T(-1);
            const int k = ((lane & ~h) & (2 * h - 1)) * (NOS / (2 * h));
            const T wr = top ? T(1) : twr[k], wi = top ? T(0) : twi[k];
#pragma unroll
            for (int v = 0; v < VPL; ++v) {
                if (h == 2) {
                    // conj(w) is 1 or +i: b * i = -bi + i br
                    const bool rot = !top && (lane & 1);
                    const T br = re[v], bi = im[v];
                    re[v] = rot ? flip_sign(bi) : br;
                    im[v] = rot ? br : bi;
                } else if (h != 1) {
                    const T br = re[v], bi = im[v];
                    re[v] = br * wr + bi * wi;
                    im[v] = bi * wr - br * wi;
                }
                const T yr = __shfl_xor_sync(0xffffffffu, re[v], h);
                const T yi = __shfl_xor_sync(0xffffffffu, im[v], h);
                re[v] = fma(sg, re[v], yr);
                im[v] = fma(sg, im[v], yi);
            }
        } else {
            const int hv = h / 32;
#pragma unroll
            for (int v = 0; v < VPL; ++v) {
                if ((v % (2 * hv)) < hv) {
                    const int vb = v + hv;
                    const int k = ((32 * v + lane) % (2 * h)) * (NOS / (2 * h));
                    const T wr = twr[k], wi = twi[k];
                    const T br = re[vb] * wr + im[vb] * wi;
                    const T bi = im[vb] * wr - re[vb] * wi;
                    const T ar = re[v], ai = im[v];
                    re[v] = ar + br;
                    im[v] = ai + bi;
                    re[vb] = ar - br;
                    im[vb] = ai - bi;
                }
            }
        }
    }
}

template <typename T, int NOS, int LINES>
struct ConvCfg {
    static constexpr int LT = LINES;       // grid lines per CTA (at most)
    static constexpr int LS = NOS + 1;     // padded line stride in shared memory
    static constexpr size_t smem = sizeof(T) * ((size_t)LT * LS + NOS + NOS);
};

// Strides of window grids: element (u_0, .., u_{d-1}) at sum_k u_k n_os^{d-1-k}. T is the grids'
// element type, A the arithmetic type of the transforms (T, or pf pairs for FP64 grids; the
// shared-memory layout is the same since sizeof(pf) == sizeof(double)).
template <typename T, int NOS, int DW, int LINES, typename A = T>
__global__ void __launch_bounds__(256) k_conv(ConvArgs a) {
    pdl_wait();
    pdl_trigger();
    static_assert(sizeof(A) == sizeof(T), "the arithmetic type takes the storage type's slots");
    using C = ConvCfg<T, NOS, LINES>;
    constexpr int VPL = NOS / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int LT = C::LT;
    A *buf = reinterpret_cast<A *>(smem_raw);
    A *twr = buf + LT * C::LS;
    A *twi = twr + NOS / 2;
    A *d1 = twi + NOS / 2;

    const int ti = a.tile_begin + blockIdx.x;
    if (ti >= a.tile_end) return;
    const int r = blockIdx.y;
    const int4 tl = a.tiles[ti];
    // tl.w: axis in the low byte; above it the tile's line count (0: up to LT lines)
    const int w = tl.x, p = tl.y, q0 = tl.z, ax = tl.w & 255, tile_lines = tl.w >> 8;
    const DevWindow dw = a.dwin[w];

    for (int i = threadIdx.x; i < NOS / 2; i += blockDim.x) {
        twr[i] = to_arith<A>(reinterpret_cast<const T *>(a.tw)[2 * i]);
        twi[i] = to_arith<A>(reinterpret_cast<const T *>(a.tw)[2 * i + 1]);
    }
    for (int i = threadIdx.x; i < NOS; i += blockDim.x)
        d1[i] = to_arith<A>(reinterpret_cast<const T *>(a.D1br)[((size_t)w * 3 + ax) * NOS + i]);

    // axis stride, line stride (q) and outer stride (p)
    long long S[3] = {0, 0, 0};
    {
        long long s = 1;
        for (int k = DW - 1; k >= 0; --k) { S[k] = s; s *= NOS; }
    }
    int qd = -1, pd = -1;
    if (DW == 3) {
        // the two non-axis dims: q = the faster one (larger index), p = the other
        int o0 = -1, o1 = -1;
        for (int k = 0; k < 3; ++k) if (k != ax) { if (o0 < 0) o0 = k; else o1 = k; }
        pd = o0;
        qd = o1;
    } else if (DW == 2) {
        qd = 1 - ax;
    }
    const long long s_ax = S[ax];
    const long long s_q = qd >= 0 ? S[qd] : 0;
    const long long s_p = pd >= 0 ? S[pd] : 0;
    const long long goff = (a.zero_offset ? 0 : dw.grid_off) + p * s_p;
    const T *in = reinterpret_cast<const T *>(a.in) + (size_t)r * a.grid_stride_rhs + goff;
    T *out = reinterpret_cast<T *>(a.out) + (size_t)r * a.grid_stride_rhs + goff;
    const int nlines = DW == 1 ? 1 : min(tile_lines > 0 ? tile_lines : LT, NOS - q0);

    for (int i = threadIdx.x; i < LT * NOS; i += blockDim.x) {
        int j, u;
        if (s_ax == 1) { u = i % NOS; j = i / NOS; } else { j = i % LT; u = i / LT; }
        T val = T(0);
        if (j < nlines) val = in[(long long)u * s_ax + (long long)(q0 + j) * s_q];
        buf[j * C::LS + u] = to_arith<A>(val);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int pr = warp; pr < LT / 2; pr += blockDim.x / 32) {
        if (2 * pr >= nlines) break;
        A re[VPL], im[VPL];
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            re[v] = buf[(2 * pr) * C::LS + 32 * v + lane];
            im[v] = buf[(2 * pr + 1) * C::LS + 32 * v + lane];
        }
        conv_line<A, NOS>(re, im, twr, twi, d1, lane);
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            buf[(2 * pr) * C::LS + 32 * v + lane] = re[v];
            buf[(2 * pr + 1) * C::LS + 32 * v + lane] = im[v];
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < LT * NOS; i += blockDim.x) {
        int j, u;
        if (s_ax == 1) { u = i % NOS; j = i / NOS; } else { j = i % LT; u = i / LT; }
        if (j < nlines) out[(long long)u * s_ax + (long long)(q0 + j) * s_q] = to_storage<T>(buf[j * C::LS + u]);
    }
}

}  // namespace anova
