// Double-float arithmetic: a value carried as an unevaluated sum hi + lo of
// two floats (about 48 significant bits), built from the error-free
// transformations of Dekker (1971) and Knuth (TAOCP vol. 2): the rounding
// error of a float sum is recovered exactly by the two-sum sequence, that of
// a float product by one FMA.  Used for the per-span phase reference of the
// channel generator, which needs ~1e-12 relative accuracy; GB300's FP64 pipe
// runs at a small fraction of the FP32 rate, so the reference is kept on the
// FP32 pipe.  Only additions appear where contraction into an FMA would
// break an identity.
#pragma once

#include <math.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace xl {

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// |a| >= |b| required
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}

__device__ __forceinline__ ff ff_two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    float e = fmaf(a, b, -p);
    return {p, e};
}

__device__ __forceinline__ ff ff_from_double(double d) {
    float h = (float)d;
    return {h, (float)(d - (double)h)};
}

// exact split of an integer of magnitude < 2^48 into hi + lo floats
__device__ __forceinline__ ff ff_from_int64(long long v) {
    float h = (float)v;
    long long r = v - (long long)h;
    return {h, (float)r};
}

__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = ff_two_sum(a.hi, b.hi);
    ff t = ff_two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = ff_fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return ff_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    ff p = ff_two_prod(a.hi, b.hi);
    p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
    return ff_fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
    ff p = ff_two_prod(a.hi, b);
    p.lo = fmaf(a.lo, b, p.lo);
    return ff_fast_two_sum(p.hi, p.lo);
}

// a / b: float quotient, then one correction from the exact remainder
__device__ __forceinline__ ff ff_div(ff a, ff b) {
    float q1 = __fdiv_rn(a.hi, b.hi);
    ff r = ff_sub(a, ff_mul_f(b, q1));
    float q2 = __fdiv_rn(r.hi, b.hi);
    return ff_fast_two_sum(q1, q2);
}

// sqrt(a), a > 0: float square root, then one Newton step on the exact residual
__device__ __forceinline__ ff ff_sqrt(ff a) {
    float y = __fsqrt_rn(a.hi);
    ff y2 = ff_two_prod(y, y);
    float d = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, y2.hi), y2.lo), a.lo);
    return ff_fast_two_sum(y, __fdiv_rn(d, __fmul_rn(2.0f, y)));
}

// ---- FP64 values on the FP32 pipe, and packed (FP32x2) double-float
// products with double-float sums (the receivers and the Appendix A Cholesky)

// Split of an FP64 value into two floats, hi + lo = d to ~2^-48 relative,
// with integer and FP32 instructions only (FP64 <-> FP32 conversions occupy
// the FP64 pipe): hi is d truncated to 24 significant bits (sign, rebiased
// exponent, top 23 stored mantissa bits); the remaining 29 mantissa bits m
// give lo = RN(m) 2^(e - 1075), RN(m) formed exactly from m's low 23 and high
// 6 bits (2^23 + a is exact in FP32) by one FMA.  Values whose hi or lo would
// leave the normal FP32 range (|d| < 2^-74 but not zero, |d| >= 2^128, inf,
// NaN) take the FP64 conversion; a zero (the imaginary part of every Gram
// diagonal) is split by integer operations too, since an FP64 instruction
// costs a full warp's issue even when one lane takes it.
__device__ __forceinline__ void split_f64(double d, float& hi, float& lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const uint32_t bh = (uint32_t)(b >> 32), bl = (uint32_t)b;
    const uint32_t e = (bh >> 20) & 0x7FFu;  // biased exponent
    if (((bh & 0x7FFFFFFFu) | bl) == 0u) {
        hi = lo = __uint_as_float(bh);  // +0 or -0
    } else if (e - 949u <= 1150u - 949u) {
        const uint32_t sg = bh & 0x80000000u;
        hi = __uint_as_float(sg | ((e - 896u) << 23) | ((bh & 0xFFFFFu) << 3) | (bl >> 29));
        const uint32_t m = bl & 0x1FFFFFFFu;
        const float fa = __fsub_rn(__uint_as_float(0x4B000000u | (m & 0x7FFFFFu)), 8388608.0f);
        const float fb = __fsub_rn(__uint_as_float(0x4B000000u | (m >> 23)), 8388608.0f);
        const float l = __fmul_rn(__fmaf_rn(fb, 8388608.0f, fa), __uint_as_float((e - 948u) << 23));
        lo = __uint_as_float(__float_as_uint(l) | sg);
    } else {
        hi = (float)d;
        lo = (float)(d - (double)hi);
    }
}

// (s, c) += x * y, lane-wise on two lanes: x, y double-float (hi, lo).
__device__ __forceinline__ void ff2_mac(float2& s, float2& c, float2 xh, float2 xl, float2 yh, float2 yl) {
    const float2 p = __fmul2_rn(xh, yh);
    float2 e = __ffma2_rn(xh, yh, make_float2(-p.x, -p.y));  // exact: xh yh = p + e
    e = __ffma2_rn(xh, yl, e);
    e = __ffma2_rn(xl, yh, e);
    const float2 t = __fadd2_rn(s, p);  // two-sum: s + p = t + err exactly
    const float2 bb = __fadd2_rn(t, make_float2(-s.x, -s.y));
    const float2 ea = __fadd2_rn(s, make_float2(-(t.x - bb.x), -(t.y - bb.y)));
    const float2 eb = __fadd2_rn(p, make_float2(-bb.x, -bb.y));
    s = t;
    c = __fadd2_rn(c, __fadd2_rn(__fadd2_rn(ea, eb), e));
}

// (s, c) += (s2, c2) lane-wise for double-float values (two-sum on the high
// parts, low parts summed alongside).
__device__ __forceinline__ void ff2_add(float2& s, float2& c, float2 s2, float2 c2) {
    const float2 t = __fadd2_rn(s, s2);
    const float2 bb = __fadd2_rn(t, make_float2(-s.x, -s.y));
    const float2 ea = __fadd2_rn(s, make_float2(-(t.x - bb.x), -(t.y - bb.y)));
    const float2 eb = __fadd2_rn(s2, make_float2(-bb.x, -bb.y));
    s = t;
    c = __fadd2_rn(__fadd2_rn(c, c2), __fadd2_rn(ea, eb));
}

// Pivot of the Cholesky factorisation: y = 1/sqrt(d) in FP64 with five FP64
// instructions.  The FP32 seed comes from d's high mantissa bits and goes back
// to FP64 exactly, both by integer operations; one third-order step
//   y = y0 (1 + r/2 + 3 r^2/8),  r = 1 - d y0^2  (y0^2 exact in FP64)
// leaves a truncation error (5/16) r^3 ~ 2^-64, below FP64 rounding (the FP64
// pipe issues one warp instruction per ~64 cycles per scheduler whatever the
// active lanes, so the single-lane pivot chain is kept short).  Returns false
// unless d is a positive finite number.
__device__ __forceinline__ bool rsqrt_pivot(double d, double& y) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const uint32_t bh = (uint32_t)(b >> 32), bl = (uint32_t)b;
    const uint32_t e = bh >> 20;  // sign and biased exponent: negative d lands above 2047
    if (e - 923u <= 1122u - 923u) {  // 2^-100 <= d < 2^100
        const float sf = __uint_as_float(((e - 896u) << 23) | ((bh & 0xFFFFFu) << 3) | (bl >> 29));
        const uint32_t yb = __float_as_uint(rsqrtf(sf));
        const double y0 = __hiloint2double((int)((((yb >> 23) + 896u) << 20) | ((yb & 0x7FFFFFu) >> 3)),
                                           (int)((yb & 7u) << 29));
        const double r = fma(-d, y0 * y0, 1.0);
        y = fma(y0 * r, fma(r, 0.375, 0.5), y0);
        return true;
    }
    if (!(d > 0.0) || !isfinite(d)) return false;
    y = 1.0 / sqrt(d);
    return true;
}

}  // namespace xl
