// A number as an unevaluated sum hi + lo of two FP32 values (|lo| <= half an ulp of hi after
// every operation), with the arithmetic the FFT passes need, for FP64 plans on a GPU whose FP64
// pipe runs at 1/64 of its FP32 rate. Sums use the exact two-sum of hi parts; products keep the
// exact error of hi * hi (fma) and the cross terms; results are renormalised. All operations are
// explicitly rounded so that no contraction into fused multiply-adds changes them. Relative error
// per operation ~2^-46.
#pragma once

namespace anova {

// the pair overloads below must not hide the standard ones inside this namespace
using ::fma;
using ::__shfl_xor_sync;

struct pf {
    float hi, lo;
    pf() = default;
    __host__ __device__ constexpr pf(int v) : hi((float)v), lo(0.0f) {}
    __host__ __device__ constexpr pf(float h, float l) : hi(h), lo(l) {}
};

__device__ __forceinline__ pf pf_fast_norm(float s, float e) {
    const float h = __fadd_rn(s, e);
    return pf(h, __fsub_rn(e, __fsub_rn(h, s)));
}
__device__ __forceinline__ pf operator+(pf a, pf b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return pf_fast_norm(s, e);
}
__device__ __forceinline__ pf operator-(pf a) { return pf(-a.hi, -a.lo); }
__device__ __forceinline__ pf operator-(pf a, pf b) { return a + (-b); }
__device__ __forceinline__ pf operator*(pf a, pf b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return pf_fast_norm(p, e);
}
__device__ __forceinline__ pf &operator*=(pf &a, pf b) {
    a = a * b;
    return a;
}
__device__ __forceinline__ pf fma(pf a, pf b, pf c) { return a * b + c; }
__device__ __forceinline__ pf flip_sign(pf x) { return -x; }
__device__ __forceinline__ pf __shfl_xor_sync(unsigned mask, pf v, int lane_mask) {
    return pf(::__shfl_xor_sync(mask, v.hi, lane_mask), ::__shfl_xor_sync(mask, v.lo, lane_mask));
}

// storage <-> arithmetic type (identity unless the arithmetic runs in pairs)
template <typename A, typename S>
__device__ __forceinline__ A to_arith(S x) { return (A)x; }
template <>
__device__ __forceinline__ pf to_arith<pf, double>(double x) {
    const float h = __double2float_rn(x);
    return pf(h, __double2float_rn(x - (double)h));
}
template <typename S, typename A>
__device__ __forceinline__ S to_storage(A x) { return (S)x; }
template <>
__device__ __forceinline__ double to_storage<double, pf>(pf x) { return (double)x.hi + (double)x.lo; }

}  // namespace anova
