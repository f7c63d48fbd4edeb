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

#include <cuda_runtime.h>

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

}  // namespace xl
