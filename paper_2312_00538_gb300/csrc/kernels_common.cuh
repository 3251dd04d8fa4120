// Device building blocks shared by the spread / interpolation / FFT kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "anova_internal.h"

#ifndef ANOVA_PDL
#define ANOVA_PDL 1
#endif

namespace anova {

// ---------------------------------------------------------------- programmatic dependent launch
// The kernels of one matvec are launched with programmatic stream serialisation: a kernel's CTAs
// may be scheduled while its predecessor in the stream is still finishing, and each kernel waits
// (griddepcontrol.wait: the predecessor has completed and its writes are visible) before it
// reads anything, then lets its own successor be scheduled. Launch latency and the ramp of the
// next grid overlap the tail of the previous one. A kernel launched without the attribute
// passes the wait at once.
__device__ __forceinline__ void pdl_wait() {
#if ANOVA_PDL
    asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}
__device__ __forceinline__ void pdl_trigger() {
#if ANOVA_PDL
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}

// Launches kern<<<grid, block, smem, st>>>(args...), with programmatic stream serialisation when
// it is compiled in (every kernel launched here calls pdl_wait() before its first dependent read).
template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                     Args &&...args) {
#if ANOVA_PDL
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
#else
    kern<<<grid, block, smem, st>>>(static_cast<KArgs>(args)...);
    return cudaGetLastError();
#endif
}

// Window polynomial coefficients (FP32 kernels) and Kaiser-Bessel constants (FP64 kernels),
// passed by value so that they live in the kernel-parameter constant bank.
struct WinParams {
    float c[16][kPolyDeg + 1];    // c[j][p]: psi(f + m - 1 - j) ~ sum_p c z^p, z = 2f - 1 (FP32)
    double c64[8][kPolyDeg64 + 1];// the same for j < m in FP64 (degree 13, error ~1e-14)
    double beta;                  // Kaiser-Bessel shape pi (2 - 1/oversampling)
    double scale;                 // m / sinh(beta m): normalises psi(0) to 1
};

// The 2M window weights of one coordinate with fractional cell offset f in [0, 1):
// w[j] = psi(f + M - 1 - j), the weight of grid point c - M + 1 + j for a point in cell c.
template <typename T, int M>
struct Weights;

// The window is even, so the weight of offset 2M-1-j at z equals the weight of offset j at -z.
// With p_j(z) = E_j(z^2) + z O_j(z^2), both come from one evaluation of E_j and O_j at z^2.
template <int M>
struct Weights<float, M> {
    static __device__ __forceinline__ void eval(float f, const WinParams &wp, float *w) {
        static_assert(kPolyDeg % 2 == 1, "even/odd split assumes an odd degree");
        const float z = fmaf(2.0f, f, -1.0f);
        const float z2 = z * z;
#pragma unroll
        for (int j = 0; j < M; ++j) {
            float e = wp.c[j][kPolyDeg - 1], o = wp.c[j][kPolyDeg];
#pragma unroll
            for (int p = kPolyDeg - 3; p >= 0; p -= 2) {
                e = fmaf(e, z2, wp.c[j][p]);
                o = fmaf(o, z2, wp.c[j][p + 1]);
            }
            w[j] = fmaf(z, o, e);
            w[2 * M - 1 - j] = fmaf(-z, o, e);
        }
    }
};

template <int M>
struct Weights<double, M> {
    static __device__ __forceinline__ void eval(double f, const WinParams &wp, double *w) {
        static_assert(kPolyDeg64 % 2 == 1, "even/odd split assumes an odd degree");
        const double z = fma(2.0, f, -1.0);
        const double z2 = z * z;
#pragma unroll
        for (int j = 0; j < M; ++j) {
            double e = wp.c64[j][kPolyDeg64 - 1], o = wp.c64[j][kPolyDeg64];
#pragma unroll
            for (int p = kPolyDeg64 - 3; p >= 0; p -= 2) {
                e = fma(e, z2, wp.c64[j][p]);
                o = fma(o, z2, wp.c64[j][p + 1]);
            }
            w[j] = fma(z, o, e);
            w[2 * M - 1 - j] = fma(-z, o, e);
        }
    }
};

// One pair of window weights, lo = psi(f + M - 1 - j) and hi = psi(f - M + j), from the
// even/odd coefficients cj[0..D] of pair j (D = kPolyDeg or kPolyDeg64); the same operations in
// the same order as Weights<T, M>::eval, so both give identical values.
template <typename T, int D>
__device__ __forceinline__ void window_pair(T f, const T *cj, T &lo, T &hi) {
    const T z = fma(T(2), f, T(-1));
    const T z2 = z * z;
    T e = cj[D - 1], o = cj[D];
#pragma unroll
    for (int p = D - 3; p >= 0; p -= 2) {
        e = fma(e, z2, cj[p]);
        o = fma(o, z2, cj[p + 1]);
    }
    lo = fma(z, o, e);
    hi = fma(-z, o, e);
}

template <typename T>
struct PolyDegOf {
    static constexpr int D = kPolyDeg;
};
template <>
struct PolyDegOf<double> {
    static constexpr int D = kPolyDeg64;
};

// Coefficient j, p of the window polynomials of type T.
template <typename T>
__device__ __forceinline__ T window_coef(const WinParams &wp, int j, int p);
template <>
__device__ __forceinline__ float window_coef<float>(const WinParams &wp, int j, int p) { return wp.c[j][p]; }
template <>
__device__ __forceinline__ double window_coef<double>(const WinParams &wp, int j, int p) { return wp.c64[j][p]; }

__device__ __forceinline__ int cell_coord(int packed, int k) { return (packed >> (10 * k)) & 1023; }

// ---------------------------------------------------------------- packed FP32 pairs (f32x2)
// Blackwell executes fma/mul/add on two FP32 lanes per instruction; the FMA pipe rate in FLOP/s
// is unchanged, but every instruction does two operations, which frees issue slots for the loads
// that feed the spread and interpolation loops.
typedef float2 f32x2;

__device__ __forceinline__ f32x2 pack2(float lo, float hi) { return make_float2(lo, hi); }
__device__ __forceinline__ void unpack2(f32x2 v, float &lo, float &hi) {
    lo = v.x;
    hi = v.y;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f32x2 zero2() { return make_float2(0.0f, 0.0f); }
// two pairs from one 16-byte aligned shared-memory load
__device__ __forceinline__ void lds_pairs(const float *p, f32x2 &a, f32x2 &b) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    a = make_float2(t.x, t.y);
    b = make_float2(t.z, t.w);
}

// Load n contiguous T from 16-byte aligned shared memory.
template <typename T, int CNT>
__device__ __forceinline__ void lds_vec(const T *p, T *out) {
    if constexpr (sizeof(T) == 4 && CNT % 4 == 0) {
#pragma unroll
        for (int i = 0; i < CNT / 4; ++i) {
            const float4 q = reinterpret_cast<const float4 *>(p)[i];
            out[4 * i + 0] = q.x;
            out[4 * i + 1] = q.y;
            out[4 * i + 2] = q.z;
            out[4 * i + 3] = q.w;
        }
    } else if constexpr (sizeof(T) == 8 && CNT % 2 == 0) {
#pragma unroll
        for (int i = 0; i < CNT / 2; ++i) {
            const double2 q = reinterpret_cast<const double2 *>(p)[i];
            out[2 * i + 0] = q.x;
            out[2 * i + 1] = q.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < CNT; ++i) out[i] = p[i];
    }
}

template <int DW, int M>
struct Geo {
    static constexpr int W2 = 2 * M;                                   // footprint edge
    static constexpr int ROWS = DW == 3 ? W2 * W2 : (DW == 2 ? W2 : 1); // rows of the last dim
    static constexpr int RPL = (ROWS + 31) / 32;                       // rows per lane
    static constexpr int WS = (W2 + 3) / 4 * 4;                        // padded weights per dim
    static constexpr int PSTRIDE = DW * WS;                            // staged weights per point
    static constexpr int VOL = DW == 3 ? W2 * W2 * W2 : (DW == 2 ? W2 * W2 : W2);
};

constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

}  // namespace anova
