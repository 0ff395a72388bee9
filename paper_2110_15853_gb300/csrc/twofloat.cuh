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


// Packed form: two independent two-float lanes in one pair of FP32 registers,
// driven by the sm_100-family packed instructions (add/sub/mul/fma .rn.f32x2),
// which do the work of two FP32 instructions per issue slot.  Every lane is
// rounded exactly like the scalar intrinsics above, so the packed routines give
// bit-identical results to their scalar counterparts.
typedef unsigned long long F2;

__device__ __forceinline__ F2 pk2(float a, float b) {
    F2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(F2 v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ F2 add2(F2 a, F2 b) {
    F2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ F2 sub2(F2 a, F2 b) {
    F2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ F2 mul2(F2 a, F2 b) {
    F2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) {
    F2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// Packed df_madd: (sh, sl) += h * y in both lanes, h shared by the lanes and given
// as hh2 = (hh, hh), nhh2 = (-hh, -hh), hl2 = (hl, hl).  The negated product
// np = -fl(hh*yh) stands in for p (rounding is sign-symmetric), so TwoProduct,
// TwoSum and the error update are the scalar steps with p replaced by -np.
__device__ __forceinline__ void df_madd2(F2 hh2, F2 nhh2, F2 hl2, F2 yh2, F2 yl2, F2& sh2, F2& sl2) {
    const F2 np = mul2(nhh2, yh2);
    F2 e = fma2(hh2, yh2, np);
    e = fma2(hh2, yl2, e);
    e = fma2(hl2, yh2, e);
    const F2 s = sub2(sh2, np);
    const F2 z = sub2(s, sh2);
    const F2 t2 = sub2(sh2, sub2(s, z));
    const F2 err = sub2(t2, add2(np, z));
    sh2 = s;
    sl2 = add2(sl2, add2(err, e));
}

// Packed fast_norm of both lanes.
__device__ __forceinline__ void fast_norm2(F2& s, F2& e) {
    const F2 hi = add2(s, e);
    e = sub2(e, sub2(hi, s));
    s = hi;
}


}  // namespace
}  // namespace chfsi
