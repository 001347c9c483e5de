// Double-float accumulation of FP32 products, for the FP64-accurate
// convolutions of the refinement on the FP32 pipe.
//
// A value is carried as a float pair (s, c) with value s + c.  An FP64
// input x is split into hi = float(x) and lo = float(x - hi).  A product
// with an FP32 tap t is formed exactly as t hi = p + e (p = t hi rounded,
// e = fma(t, hi, -p): the FMA error-free product), p is added to s with
// Knuth's error-free TwoSum (s + p = s' + er exactly), and er + e + t lo go
// into c.  The result carries ~2^-44 of relative error per term instead of
// FP32's 2^-24.
#pragma once

#include <cuda_runtime.h>

namespace mirage {

// The error-free steps must not be fused into FMAs (a fused s + t xh breaks
// TwoSum's exactness): on the device they use the round-to-nearest
// intrinsics, which the compiler never contracts; host builds (tests) are
// compiled without contraction.
#if defined(__CUDA_ARCH__)
__device__ __forceinline__ float df_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float df_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float df_sub(float a, float b) { return __fsub_rn(a, b); }
#else
inline float df_mul(float a, float b) { return a * b; }
inline float df_add(float a, float b) { return a + b; }
inline float df_sub(float a, float b) { return a - b; }
#endif

__host__ __device__ __forceinline__ void df_split(double x, float& hi, float& lo) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

// (s, c) += t * (xh + xl)
__host__ __device__ __forceinline__ void df_madd(float& s, float& c, float t, float xh, float xl) {
    const float pr = df_mul(t, xh);
    const float e = fmaf(t, xh, -pr);  // t xh - pr, exactly
    const float sn = df_add(s, pr);    // TwoSum(s, pr) = sn + er
    const float bv = df_sub(sn, s);
    const float er = df_add(df_sub(s, df_sub(sn, bv)), df_sub(pr, bv));
    s = sn;
    c = fmaf(t, xl, df_add(c, df_add(er, e)));
}

}  // namespace mirage
