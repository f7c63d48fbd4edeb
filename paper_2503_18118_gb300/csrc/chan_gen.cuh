// On-the-fly channel generation (Sec. II-B) shared by the FP32 SIMT and the
// tensor-core Gram kernels.  Channel entries are produced in registers and
// go straight into shared-memory tiles; they are never written to HBM.
//
// FP32 phase with an accurate per-span reference.  The phase 2 pi r_k(n)/lambda
// reaches ~10^5 rad, far beyond FP32 resolution, so for every user and every
// span of REF_SPAN elements a reference element n_c at the span centre is
// evaluated to ~48 bits in double-float arithmetic (ff.cuh):
//   frac0 = r(n_c)/lambda - rint(r(n_c)/lambda)          (cycles, |.| <= 1/2)
//   A     = (spacing/lambda) (y_{n_c} - y_k) / r(n_c)     (dr/dn at n_c, cycles per element)
// For element n = n_c + m, with u = m spacing/lambda and lengths in
// wavelengths, the distance splits exactly into
//   r(n) - r(n_c) = m A + R,   R = 2 u^2 x^2 / (r_c ((r_c + r - u)(r_c + r + u)))
// (subtract the tangent line from r - r_c = (2 e_c u + u^2)/(r + r_c) and
// simplify; no term cancels because r_c + r > |u| for x > 0).  m A is formed
// exactly against A held as two floats (an FP32 product plus FMA residual, or
// in the packed path a 16-bit high part whose product with m is exact), and
// every partial sum is reduced modulo one cycle before it is added.  An FP32
// emulation puts the worst phase error at ~4e-6 rad for the scalar generator
// and ~8e-6 rad for the packed one of the tensor-core kernels (users 3-30 m
// from 16384- and 131072-element 100 GHz arrays, 5-50 m from a 65536-element
// 28 GHz array), below the BF16 hi/lo split's 2^-16.  The planar-wave model
// is the linear term alone (R = 0).
#pragma once

#include "common.cuh"
#include "ff.cuh"

namespace xl {

constexpr int REF_SPAN = 128;  // elements per phase reference

// Per launch, prepared on the host from the FP64 geometry.
struct GenParams {
    ff delta;       // element spacing [m]
    ff inv_lambda;  // 1/lambda [1/m]
    ff dprime;      // spacing / lambda
    float dprime_f;
    int model;
    long long nm1;  // N - 1
};

// Per user, built once per CTA from the FP64 position.
struct UserGeo {
    ff x, y, x2;   // metres, metres^2
    ff r0u, su;    // planar model: |user| and sin(theta)
    float xl2;     // (x/lambda)^2
    float x2x2;    // 2 (x/lambda)^2
    float ampc;    // amplitude constant (model dependent)
    int ok;        // valid position
};

// Per user, per reference span.
struct UserRef {
    float frac0, a_hi, a_lo, e0, r0, kx;  // kx = 2 (x/lambda)^2 / r0
};

inline GenParams make_gen_params(const Geom& g) {
    auto split = [](double d) {
        float h = (float)d;
        return ff{h, (float)(d - (double)h)};
    };
    GenParams p;
    p.delta = split(g.spacing);
    p.inv_lambda = split(g.inv_lambda);
    p.dprime = split(g.spacing * g.inv_lambda);
    p.dprime_f = (float)(g.spacing * g.inv_lambda);
    p.model = g.model;
    p.nm1 = (long long)(g.N - 1);
    return p;
}

// Amplitude constant of the model (FP64): FSPL lambda/(4 pi r) = c / r' with
// c = 1/(4 pi) and r' in wavelengths; PNUSW sqrt(beta0 x) r^{-3/2} = c r'^{-3/2}
// with c = sqrt(beta0) sqrt(x/lambda) / lambda; UPW sqrt(beta0) / |user|.
__device__ __forceinline__ double amp_const(const Geom& g, double x, double y) {
    if (g.model == XLMIMO_FSPL_USW) return 1.0 / (4.0 * 3.14159265358979323846);
    if (g.model == XLMIMO_PNUSW) return sqrt(g.beta0) * sqrt(x * g.inv_lambda) * g.inv_lambda;
    return sqrt(g.beta0) / sqrt(x * x + y * y);
}

__device__ __forceinline__ UserGeo make_user_geo(const Geom& g, double x, double y) {
    UserGeo u;
    u.ok = user_ok(x, y);
    if (!u.ok) { x = 1.0; y = 0.0; }
    u.x = ff_from_double(x);
    u.y = ff_from_double(y);
    u.x2 = ff_from_double(x * x);
    u.x2.lo += (float)fma(x, x, -(double)u.x2.hi - (double)u.x2.lo);  // x^2 to ~2^-48
    double r0 = sqrt(x * x + y * y);
    u.r0u = ff_from_double(r0);
    u.su = ff_from_double(y / r0);
    double xl = x * g.inv_lambda;
    u.xl2 = (float)(xl * xl);
    u.x2x2 = (float)(2.0 * xl * xl);
    u.ampc = (float)amp_const(g, x, y);
    return u;
}

// Reference quantities of user u at element nc, in double-float.
__device__ __forceinline__ UserRef make_user_ref(const GenParams& p, const UserGeo& u, long long nc) {
    // y_{n_c} = (n_c - (N-1)/2) spacing = (2 n_c - (N-1)) * spacing / 2, exact integer split
    ff half_idx = ff_from_int64(2 * nc - p.nm1);
    half_idx.hi *= 0.5f;
    half_idx.lo *= 0.5f;
    ff ync = ff_mul(half_idx, p.delta);
    UserRef R;
    ff q0, A;
    if (p.model == XLMIMO_UPW) {
        q0 = ff_mul(ff_sub(u.r0u, ff_mul(ync, u.su)), p.inv_lambda);
        A = ff_neg(ff_mul(p.dprime, u.su));
        R.e0 = 0.f;
        R.r0 = 1.f;
        R.kx = 0.f;
    } else {
        ff e0 = ff_sub(ync, u.y);
        ff r0 = ff_sqrt(ff_add(u.x2, ff_mul(e0, e0)));
        q0 = ff_mul(r0, p.inv_lambda);
        A = ff_div(ff_mul(p.dprime, e0), r0);
        R.e0 = e0.hi * p.inv_lambda.hi;
        R.r0 = q0.hi;
        R.kx = __fdiv_rn(u.x2x2, q0.hi);
    }
    R.frac0 = __fadd_rn(__fsub_rn(q0.hi, rintf(q0.hi)), q0.lo);
    R.frac0 -= rintf(R.frac0);
    R.a_hi = A.hi;
    R.a_lo = A.lo;
    return R;
}

// x - rint(x) for |x| < 2^22 by adding and removing 1.5 * 2^23 (exact in
// round-to-nearest), which keeps the reduction on the FMA pipe.
__device__ __forceinline__ float frac_rn(float x) {
    const float magic = 12582912.0f;
    float t = __fsub_rn(__fadd_rn(x, magic), magic);
    return __fsub_rn(x, t);
}

// Channel entry h_k(n_c + m) as FP32 complex (re, im) = amp (cos phi, -sin phi);
// mf = (float)m, an exact small integer.
__device__ __forceinline__ float2 gen_entry_f32(int model, float dprime, float xl2, float x2x2, float ampc,
                                                const UserRef& R, float mf) {
    // linear term m*A: exact product plus residual, reduced modulo one cycle
    float p = __fmul_rn(mf, R.a_hi);
    float pe = fmaf(mf, R.a_hi, -p);
    float g = R.frac0 + frac_rn(p) + fmaf(mf, R.a_lo, pe);
    float amp;
    if (model == XLMIMO_UPW) {
        amp = ampc;
    } else {
        float u = mf * dprime;
        float en = R.e0 + u;
        float r2 = fmaf(en, en, xl2);
        float rs = rsqrtf(r2);
        float rp = r2 * rs;
        float sum = R.r0 + rp;
        float u2 = u * u;
        float den = R.r0 * fmaf(sum, sum, -u2);  // r_c ((r_c + r)^2 - u^2), no cancellation
        g += frac_rn(__fdividef(x2x2 * u2, den));
        amp = (model == XLMIMO_FSPL_USW) ? ampc * rs : ampc * rs * rsqrtf(rp);
    }
    g = frac_rn(g);
    float s, co;
    __sincosf(6.283185307179586f * g, &s, &co);
    return make_float2(amp * co, -amp * s);
}

// ---- paired generation on the packed FP32x2 pipe ----------------------------
// Two consecutive elements of one user per call; every FP32 operation is a
// packed two-lane instruction (the transcendental ones stay scalar).  The
// algebra is that of gen_entry_f32 with some terms carried negated so that
// each step is a single packed multiply, add or FMA.

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

__device__ __forceinline__ float rcp_approx(float x) {  // relative error ~2^-23
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float2 frac2(float2 x) {  // x - rint(x), |x| < 2^22
    const float2 m = f2(12582912.0f), nm = f2(-12582912.0f);
    float2 t = __fadd2_rn(__fadd2_rn(x, m), nm);
    return __ffma2_rn(t, f2(-1.0f), x);
}

// Packed per-span constants of one user.  The linear phase term m A is
// formed per 8-element slice: with the slice centre mc (a half-integer,
// |mc| <= 2^8) and A = ah + al, ah keeping 15 significant bits, mc ah is
// exact in FP32 and reduced modulo one cycle once per slice; an element at
// offset t from the centre (|t| <= 7/2) then adds t A in one FMA, small
// enough to need no reduction.
struct PairConst {
    float frac0, ah, al;                          // slice base
    float2 af, e0, r0, xl2, kx, dp, ampc;         // kx = 2 x^2 / r_c
};

__device__ __forceinline__ PairConst make_pair_const(const UserRef& R, float dprime, float xl2, float x2x2,
                                                     float ampc) {
    PairConst c;
    const float ah = __uint_as_float(__float_as_uint(R.a_hi) & 0xFFFFFE00u);
    c.frac0 = R.frac0;
    c.ah = ah;
    c.al = __fadd_rn(__fsub_rn(R.a_hi, ah), R.a_lo);
    c.af = f2(__fadd_rn(R.a_hi, R.a_lo));
    c.e0 = f2(R.e0);
    c.r0 = f2(R.r0);
    c.xl2 = f2(xl2);
    c.kx = f2(R.kx);
    c.dp = f2(dprime);
    c.ampc = f2(ampc);
    return c;
}

// Phase (cycles, |.| <= 1) at the slice centre mc, from the span reference.
__device__ __forceinline__ float slice_base(const PairConst& c, float mc) {
    return __fadd_rn(__fmaf_rn(mc, c.al, c.frac0), frac_rn(__fmul_rn(mc, c.ah)));
}

// Entries at offsets m.x, m.y from the span centre (|m| <= 256; u = m
// spacing/lambda), which are t.x, t.y from the centre of their slice (phase
// base, from slice_base):
// re = amp cos(phi), im = -amp sin(phi) for each of the two.  UNIT leaves the
// model's amplitude constant out (the caller applies it to the Gram in FP64).
template <int MODEL, bool UNIT = false>
__device__ __forceinline__ void gen_pair(const PairConst& c, float2 u, float2 t, float base, float2& re,
                                         float2& im) {
    const float2 m1 = f2(-1.0f);
    float2 g = __ffma2_rn(t, c.af, f2(base));   // |g| <= 1 + 7/4
    float2 amp = f2(1.0f);
    if (MODEL == XLMIMO_UPW) {
        if (!UNIT) amp = c.ampc;
    } else {
        float2 nu2 = __fmul2_rn(u, make_float2(-u.x, -u.y));  // -u^2
        float2 en = __fadd2_rn(c.e0, u);
        float2 r2 = __ffma2_rn(en, en, c.xl2);
        float2 rs = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
        float2 sum = __ffma2_rn(r2, rs, c.r0);      // r_c + r
        float2 den = __ffma2_rn(sum, sum, nu2);     // (r_c + r)^2 - u^2
        float2 inv = make_float2(rcp_approx(den.x), rcp_approx(den.y));
        float2 nR = __fmul2_rn(__fmul2_rn(c.kx, nu2), inv);  // -R
        g = __ffma2_rn(frac2(nR), m1, g);
        amp = UNIT ? rs : __fmul2_rn(c.ampc, rs);
        if (MODEL == XLMIMO_PNUSW) {
            float2 rp = __fmul2_rn(r2, rs);
            amp = __fmul2_rn(amp, make_float2(rsqrtf(rp.x), rsqrtf(rp.y)));
        }
    }
    // the angle is -phi (its sine is the entry's -sin(phi)); |g| <= 13/4, so
    // |angle| <= 13 pi / 2, within the range where sin.approx / cos.approx
    // keep their stated absolute error
    g = __fmul2_rn(g, f2(-6.283185307179586f));
    float s0, c0, s1, c1;
    __sincosf(g.x, &s0, &c0);
    __sincosf(g.y, &s1, &c1);
    if (UNIT && MODEL == XLMIMO_UPW) {
        re = make_float2(c0, c1);
        im = make_float2(s0, s1);
    } else {
        re = __fmul2_rn(amp, make_float2(c0, c1));
        im = __fmul2_rn(amp, make_float2(s0, s1));
    }
}

}  // namespace xl
