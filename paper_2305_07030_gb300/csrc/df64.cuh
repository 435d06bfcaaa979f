// Double-float arithmetic: a value is an unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi)/2, about 48 significant bits.
//
// GB300 runs FP64 at roughly 1/70 of its FP32 rate, so the high-precision
// parts of the mixed solver (the lead phase and the reference refreshes) run
// on the FP32 pipes in this representation instead. Built from the classical
// error-free transformations: Knuth's TwoSum, Dekker's Fast2Sum and the
// FMA-based TwoProduct; intrinsics keep the compiler from contracting or
// reassociating any step.
#pragma once
#include <cuda_runtime.h>

namespace fe2 {

struct df {
    float hi, lo;
};

__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }

// s + e = a + b exactly (TwoSum, no precondition).
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = fadd(a, b);
    const float bb = fsub(s, a);
    const float e = fadd(fsub(a, fsub(s, bb)), fsub(b, bb));
    return {s, e};
}
// s + e = a + b exactly when |a| >= |b| (Fast2Sum).
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = fadd(a, b);
    return {s, fsub(b, fsub(s, a))};
}
// p + e = a * b exactly (TwoProduct with a fused multiply-add).
__device__ __forceinline__ df two_prod(float a, float b) {
    const float p = fmul(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df df_from(float a) { return {a, 0.f}; }
__device__ __forceinline__ df df_from_double(double d) {
    const float h = __double2float_rn(d);
    return {h, __double2float_rn(d - (double)h)};
}
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

// Accurate addition (both parts' errors carried).
__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    const df t = two_sum(a.lo, b.lo);
    s.lo = fadd(s.lo, t.hi);
    s = fast_two_sum(s.hi, s.lo);
    s.lo = fadd(s.lo, t.lo);
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// Addition of a plain float.
__device__ __forceinline__ df df_add_f(df a, float b) {
    df s = two_sum(a.hi, b);
    s.lo = fadd(s.lo, a.lo);
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_mul(df a, df b) {
    df p = two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ df df_mul_f(df a, float b) {
    df p = two_prod(a.hi, b);
    p.lo = __fmaf_rn(a.lo, b, p.lo);
    return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ df df_sqr(df a) {
    df p = two_prod(a.hi, a.hi);
    p.lo = __fmaf_rn(fadd(a.hi, a.hi), a.lo, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

// 1/sqrt(a), a > 0: FP32 estimate y0 plus one Newton step in double-float,
// y = y0 + y0 (1 - a y0^2) / 2, which doubles the estimate's ~22 good bits.
__device__ __forceinline__ df df_rsqrt(df a) {
    const float y0 = rsqrtf(a.hi);
    const df y2 = two_prod(y0, y0);
    // r = 1 - a * y0^2 evaluated in double-float
    const df ay2 = df_mul(a, y2);
    const df r = df_add_f(df_neg(ay2), 1.0f);
    const float corr = fmul(fmul(0.5f, y0), r.hi);
    return fast_two_sum(y0, corr);
}

// 1/a: FP32 estimate plus one Newton step in double-float.
__device__ __forceinline__ df df_rcp(df a) {
    const float y0 = __frcp_rn(a.hi);
    const df r = df_add_f(df_neg(df_mul_f(a, y0)), 1.0f);
    return fast_two_sum(y0, fmul(y0, r.hi));
}

}  // namespace fe2
