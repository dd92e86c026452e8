// Double-float arithmetic: a value carried as an unevaluated FP32 pair hi + lo (about
// 47 significant bits) with the error-free transformations of Knuth (two-sum) and of
// the fused multiply-add (the exact rounding error of a product), for FP64-class
// accuracy at FP32 throughput.  Used by the double-float stencil of the FP64
// residual and by the z-sweeps of the ill-conditioned lateral modes.
#pragma once

#include "iobm_internal.cuh"

namespace iobm {

// x = hi + lo: hi the leading 24 significant bits of x (truncated), lo the next
// 24 of the remaining 29 (truncated).  |x| < 2^-100 gives 0, and the lo part is
// dropped below 2^-74; |x| must stay below 2^127.
__device__ __forceinline__ void df_split(double x, float& hi, float& lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7ffull) - 1023;
    if (e < -100) {
        hi = 0.f;
        lo = 0.f;
        return;
    }
    hi = __uint_as_float(sgn | ((unsigned)(e + 127) << 23) | (unsigned)((b >> 29) & 0x7fffffull));
    const unsigned rem = (unsigned)(b & 0x1fffffffull);
    lo = 0.f;
    if (rem != 0u && e >= -74) {
        const int p = 31 - __clz(rem);   // leading one of the remainder, 0 .. 28
        const unsigned mant = (p >= 23) ? (rem >> (p - 23)) : (rem << (23 - p));
        lo = __uint_as_float(sgn | ((unsigned)(e - 52 + p + 127) << 23) | (mant & 0x7fffffu));
    }
}

// exact float -> double widening by bit operations (zero and subnormals -> 0)
__device__ __forceinline__ double df_widen(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned ef = (u >> 23) & 0xffu;
    if (ef == 0u) return 0.0;
    const unsigned long long sgn = (unsigned long long)(u & 0x80000000u) << 32;
    const unsigned long long e64 = (ef == 0xffu) ? 0x7ffull : (unsigned long long)(ef - 127u + 1023u);
    return __longlong_as_double((long long)(sgn | (e64 << 52) | ((unsigned long long)(u & 0x7fffffu) << 29)));
}

struct Dfc {        // complex double-float, lanes (re, im)
    float2 hi, lo;
};

__device__ __forceinline__ Dfc df_load(double2 v) {
    Dfc r;
    df_split(v.x, r.hi.x, r.lo.x);
    df_split(v.y, r.hi.y, r.lo.y);
    return r;
}

// The error-free transformations below use the _rn intrinsics, which the
// compiler never contracts into fused multiply-adds: a product fused into a
// later sum would turn the two-sum's correction into the product's rounding
// error and count it twice.

// s + e = a + b exactly (Knuth's two-sum)
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

// one lane of a + b, unnormalised (the rounding error of hi + hi goes into lo)
__device__ __forceinline__ void df_add1(float ah, float al, float bh, float bl, float& sh, float& sl) {
    float e;
    sh = two_sum(ah, bh, e);
    sl = __fadd_rn(e, __fadd_rn(al, bl));
}

__device__ __forceinline__ Dfc df_add(const Dfc& a, const Dfc& b) {
    Dfc r;
    df_add1(a.hi.x, a.lo.x, b.hi.x, b.lo.x, r.hi.x, r.lo.x);
    df_add1(a.hi.y, a.lo.y, b.hi.y, b.lo.y, r.hi.y, r.lo.y);
    return r;
}

// one lane of acc + c s, c = ch + cl
__device__ __forceinline__ void df_acc1(float& ah, float& al, float ch, float cl, float sh, float sl) {
    const float p = __fmul_rn(ch, sh);
    float e1 = __fmaf_rn(ch, sh, -p);   // the product's rounding error, exactly
    e1 = __fmaf_rn(ch, sl, e1);
    e1 = __fmaf_rn(cl, sh, e1);
    float e2;
    ah = two_sum(ah, p, e2);
    al = __fadd_rn(al, __fadd_rn(e1, e2));
}

// acc + c s for a real double-float weight c = (ch, cl)
__device__ __forceinline__ void df_acc(Dfc& acc, float2 c, const Dfc& s) {
    df_acc1(acc.hi.x, acc.lo.x, c.x, c.y, s.hi.x, s.lo.x);
    df_acc1(acc.hi.y, acc.lo.y, c.x, c.y, s.hi.y, s.lo.y);
}

// acc = d x for a real double-float d = (dh, dl)
__device__ __forceinline__ Dfc df_scale(float dh, float dl, const Dfc& x) {
    Dfc r;
    r.hi.x = __fmul_rn(dh, x.hi.x);
    r.hi.y = __fmul_rn(dh, x.hi.y);
    r.lo.x = __fmaf_rn(dl, x.hi.x, __fmaf_rn(dh, x.lo.x, __fmaf_rn(dh, x.hi.x, -r.hi.x)));
    r.lo.y = __fmaf_rn(dl, x.hi.y, __fmaf_rn(dh, x.lo.y, __fmaf_rn(dh, x.hi.y, -r.hi.y)));
    return r;
}

// complex double-float c s accumulated into acc (c, s complex double-float)
__device__ __forceinline__ void df_cacc(Dfc& acc, const Dfc& c, const Dfc& s) {
    // re += c.re s.re - c.im s.im,  im += c.re s.im + c.im s.re
    df_acc1(acc.hi.x, acc.lo.x, c.hi.x, c.lo.x, s.hi.x, s.lo.x);
    df_acc1(acc.hi.x, acc.lo.x, -c.hi.y, -c.lo.y, s.hi.y, s.lo.y);
    df_acc1(acc.hi.y, acc.lo.y, c.hi.x, c.lo.x, s.hi.y, s.lo.y);
    df_acc1(acc.hi.y, acc.lo.y, c.hi.y, c.lo.y, s.hi.x, s.lo.x);
}

// (hi, lo) renormalised so that hi is the FP32 rounding of hi + lo (|hi| >= |lo|
// assumed, Dekker's fast two-sum)
__device__ __forceinline__ void df_norm1(float& hi, float& lo) {
    const float s = __fadd_rn(hi, lo);
    lo = __fsub_rn(lo, __fsub_rn(s, hi));
    hi = s;
}
__device__ __forceinline__ void df_norm(Dfc& a) {
    df_norm1(a.hi.x, a.lo.x);
    df_norm1(a.hi.y, a.lo.y);
}

__device__ __forceinline__ Dfc df_from(float2 v) {
    Dfc r;
    r.hi = v;
    r.lo = make_float2(0.f, 0.f);
    return r;
}

// the FP32 value nearest to hi + lo
__device__ __forceinline__ float2 df_round(const Dfc& a) {
    return make_float2(__fadd_rn(a.hi.x, a.lo.x), __fadd_rn(a.hi.y, a.lo.y));
}

}  // namespace iobm
