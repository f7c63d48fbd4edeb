// Finite-aperture correction of the closed-form correlation (not the
// paper's; derived for this library): the stationary-phase value of Eq. (6)
// and its free-space analogue assume the stationary point of the pair phase
// phi(y) = 2 pi (r_i(y) - r_j(y)) / lambda lies inside an unbounded aperture.
// The point is where the line through the two users meets the array axis,
// y* = y_i - x_i (y_j - y_i) / (x_j - x_i); with phi'' = (2 pi / lambda)
// (x_i^2 / r_i^3 - x_j^2 / r_j^3) at y*, s = sign(phi''), and the aperture
// [-H, H], H = N spacing / 2, the quadratic phase integrates to the unbounded
// value times
//   F = [(C(u_hi) - C(u_lo)) + j s (S(u_hi) - S(u_lo))] / (1 + j s),
//   u = (edge - y*) sqrt(|phi''| / pi),
// C + j S the Fresnel integrals.  An edge more than U_CUT = 2 Fresnel lengths
// away counts at its limit C = S = sign(u)/2 (the quadratic model's tail has
// the wrong phase there).  MASK is the step F = [|y*| <= H].
#pragma once

#include "common.cuh"
#include "ff.cuh"

namespace xl {

enum { APERTURE_NONE = 0, APERTURE_MASK = 1, APERTURE_FRESNEL = 2 };
constexpr float APERTURE_U_CUT = 2.0f;

// Fresnel integrals C(u), S(u) for |u| <= 2 by their power series
//   C = sum_n (-1)^n a^{2n} / ((2n)! (4n+1)) u,  S = sum_n (-1)^n a^{2n+1} / ((2n+1)! (4n+3)) u,
// a = pi u^2 / 2, summed through the common term a^k / k!; beyond the cut the limits.
__device__ __forceinline__ void fresnel_cs_cut(float u, float& c, float& s) {
    if (!(fabsf(u) <= APERTURE_U_CUT)) {
        c = s = copysignf(0.5f, u);
        return;
    }
    const float a = 1.5707963267948966f * u * u;
    float t = 1.0f, sc = 0.0f, ss = 0.0f;
    // fully unrolled: the reciprocals 1/k and 1/(2k + 1) are constants, so
    // each term costs multiplications and one addition, no division
#pragma unroll
    for (int k = 0; k < 34; ++k) {
        if (k > 0) t *= a * (1.0f / (float)k);
        const float term = ((k >> 1) & 1 ? -t : t) * (1.0f / (float)(2 * k + 1));
        if (k & 1) ss += term;
        else sc += term;
    }
    c = u * sc;
    s = u * ss;
}

// F of the pair (i, j) (complex): mode APERTURE_*, positions in metres,
// H = N spacing / 2.  The stationary point and the mask decision are taken in
// double-float on the FP32 pipe (~2^-44 relative: the FP64 values split by
// integer operations, as GB300's FP64 pipe issues one warp instruction per
// ~64 cycles per scheduler), the Fresnel factor in FP32 (~1e-5).
__device__ __forceinline__ float2 aperture_factor(int mode, double xi, double yi, double xj, double yj, double H,
                                                  double inv_lambda) {
    if (mode == APERTURE_NONE) return make_float2(1.0f, 0.0f);
    if (xj == xi) return make_float2(0.0f, 0.0f);
    auto split = [](double d) {
        ff v;
        split_f64(d, v.hi, v.lo);
        return v;
    };
    const ff Xi = split(xi), Yi = split(yi), Xj = split(xj), Yj = split(yj), Hf = split(H);
    // y* = y_i - x_i (y_j - y_i) / (x_j - x_i)
    const ff q = ff_div(ff_mul(Xi, ff_sub(Yj, Yi)), ff_sub(Xj, Xi));
    const ff ys = ff_sub(Yi, q);
    const ff hp = ff_sub(Hf, ys), hm = ff_add(Hf, ys);  // H - y*, H + y*
    if (mode == APERTURE_MASK) {
        // |y*| <= H: both H - y* and H + y* non-negative
        const bool in = (hp.hi > 0.0f || (hp.hi == 0.0f && hp.lo >= 0.0f)) &&
                        (hm.hi > 0.0f || (hm.hi == 0.0f && hm.lo >= 0.0f));
        return make_float2(in ? 1.0f : 0.0f, 0.0f);
    }
    const float fxi = Xi.hi, fxj = Xj.hi, dyi = -q.hi, dyj = ff_sub(ys, Yj).hi;
    const float ri2 = fxi * fxi + dyi * dyi, rj2 = fxj * fxj + dyj * dyj;
    const float ci = fxi * fxi * rsqrtf(ri2) / ri2, cj = fxj * fxj * rsqrtf(rj2) / rj2;  // x^2 / r^3
    float il_h, il_l;
    split_f64(inv_lambda, il_h, il_l);
    const float p2 = 6.283185307179586f * il_h * (ci - cj);
    if (!(p2 != 0.0f)) return make_float2(0.0f, 0.0f);
    const float sc = sqrtf(fabsf(p2) * 0.3183098861837907f);
    float ch, sh, cl, sl;
    fresnel_cs_cut(hp.hi * sc, ch, sh);
    fresnel_cs_cut(-hm.hi * sc, cl, sl);
    const float a = ch - cl, b = sh - sl, sg = p2 > 0.0f ? 1.0f : -1.0f;
    return make_float2(0.5f * (a + b), 0.5f * sg * (b - a));
}

}  // namespace xl
