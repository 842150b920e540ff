// vp_sum.cuh -- compensated summation for the FEL bunching sums.
//
// The bunching <exp(-i theta)> is small (1e-4 at the start of the FEL run) and
// comes out of sums over columns that cancel almost completely, so the column
// sums must be far more accurate than one FP32 rounding. DSum keeps an
// unevaluated sum hi + lo updated with error-free transformations: Knuth's
// TwoSum for additions and the FMA form of the exact product (a*b = p + e with
// e = fma(a, b, -p)). Intrinsics with explicit rounding keep the compiler from
// contracting the steps.
#pragma once

namespace vp {

__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }

template <typename T>
struct DSum {
    T hi, lo;
    __device__ __forceinline__ DSum() : hi(T(0)), lo(T(0)) {}
    __device__ __forceinline__ void add(T x)
    {
        const T t = rn_add(hi, x);
        const T bb = rn_sub(t, hi);
        const T err = rn_add(rn_sub(hi, rn_sub(t, bb)), rn_sub(x, bb));
        hi = t;
        lo = rn_add(lo, err);
    }
    __device__ __forceinline__ void add_prod(T a, T b)
    {
        const T p = rn_mul(a, b);
        const T e = fma(a, b, -p);
        add(p);
        lo = rn_add(lo, e);
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

}  // namespace vp
