// Two-float arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers (|lo| <= ulp(hi)/2, about 48 significant bits), and every operation
// runs on the FP32 pipe with error-free transformations -- TwoProduct from one
// FMA, TwoSum after Knuth (TAOCP vol. 2, 4.2.2) and Dekker (1971).  Intrinsics
// with explicit rounding keep the compiler from contracting them into FMAs.
#pragma once

#include <cuda_runtime.h>

namespace chfsi {
namespace {

struct DF {
    float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

__device__ __forceinline__ DF fast_norm(float s, float e) {
    DF r;
    r.hi = __fadd_rn(s, e);
    r.lo = __fsub_rn(e, __fsub_rn(r.hi, s));
    return r;
}

// a * b for two-floats (the lo*lo term is below the format's precision).
__device__ __forceinline__ DF df_mul(DF a, DF b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_norm(p, e);
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return fast_norm(s, e);
}

__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }

// (sh, sl) += h * y : TwoProduct of the hi parts, cross terms into the error,
// TwoSum of the product into the running hi; errors accumulate in sl.
__device__ __forceinline__ void df_madd(float hh, float hl, float yh, float yl, float& sh, float& sl) {
    const float p = __fmul_rn(hh, yh);
    float e = fmaf(hh, yh, -p);
    e = fmaf(hh, yl, e);
    e = fmaf(hl, yh, e);
    float t, err;
    two_sum(sh, p, t, err);
    sh = t;
    sl = __fadd_rn(sl, __fadd_rn(err, e));
}

__device__ __forceinline__ DF df_from_double(double x) {
    DF r;
    r.hi = (float)x;
    r.lo = (float)(x - (double)r.hi);
    return r;
}


}  // namespace
}  // namespace chfsi
