// On-the-fly channel generation (Sec. II-B) shared by the FP32 SIMT and the
// tensor-core Gram kernels.  Channel entries are produced in registers and
// go straight into shared memory tiles; they are never written to HBM.
//
// FP32 phase with an FP64 reference.  The phase 2 pi r_k(n) / lambda reaches
// ~10^5 rad, far beyond FP32 resolution, so every kernel keeps, per user and
// per span of REF_SPAN elements, a reference element n_c at the span centre
// whose quantities are computed in FP64:
//   frac0 = r(n_c)/lambda - rint(r(n_c)/lambda)          (cycles, |.| <= 1/2)
//   A     = (spacing/lambda) (y_{n_c} - y_k) / r(n_c)     (d r / d n at n_c, cycles per element)
// For element n = n_c + m, with u = m spacing/lambda and all lengths in
// wavelengths, the distance splits exactly into
//   r(n) - r(n_c) = m A + R,   R = 2 u^2 x^2 / (r_c ((r_c + r - u)(r_c + r + u)))
// (subtract the tangent line from r - r_c = (2 e_c u + u^2)/(r + r_c) and
// simplify; no term cancels because r_c + r > |u| for x > 0).  m A is
// formed as an exact FP32 product plus FMA residual against the FP64 slope
// split in two floats, and every partial sum is reduced modulo one cycle
// before it is added, so the phase error stays near 1e-6 rad for spans of
// 128 elements at 3 m from a 16384-element 100 GHz array.
// The planar-wave model is the linear term alone (R = 0).
#pragma once

#include "common.cuh"

namespace xl {

constexpr int REF_SPAN = 128;  // elements per FP64 phase reference

struct UserConst {  // per user, per kernel
    float xl2;   // (x/lambda)^2
    float x2x2;  // 2 (x/lambda)^2
    float ampc;  // amplitude constant (model dependent, see make_user_const)
    float pad;
};

struct UserRef {  // per user, per reference span
    float frac0;
    float a_hi, a_lo;
    float e0;  // (y_{n_c} - y_k) / lambda
    float r0;  // r(n_c) / lambda
    float pad[3];
};

__device__ __forceinline__ UserConst make_user_const(const Geom& g, double x, double y) {
    UserConst c;
    double xl = x * g.inv_lambda;
    c.xl2 = (float)(xl * xl);
    c.x2x2 = (float)(2.0 * xl * xl);
    if (g.model == XLMIMO_FSPL_USW) {
        c.ampc = (float)(1.0 / (4.0 * 3.14159265358979323846));  // lambda/(4 pi r) = 1/(4 pi r')
    } else if (g.model == XLMIMO_PNUSW) {
        c.ampc = (float)(sqrt(g.beta0) * sqrt(xl) * g.inv_lambda);  // times r'^{-3/2}
    } else {
        c.ampc = (float)(sqrt(g.beta0) / sqrt(x * x + y * y));  // constant over the array
    }
    c.pad = 0.f;
    return c;
}

// FP64 reference quantities of user (x, y) at element n_c.
__device__ __forceinline__ UserRef make_user_ref(const Geom& g, double x, double y, int64_t nc) {
    UserRef R;
    double ync = element_y(nc, g.N, g.spacing);
    double q0, A;
    if (g.model == XLMIMO_UPW) {
        double r0 = sqrt(x * x + y * y);
        double s = y / r0;
        q0 = (r0 - ync * s) * g.inv_lambda;
        A = -g.spacing * s * g.inv_lambda;
        R.e0 = 0.f;
        R.r0 = 1.f;
    } else {
        double e0 = ync - y;
        double r0 = sqrt(fma(e0, e0, x * x));
        q0 = r0 * g.inv_lambda;
        A = g.spacing * g.inv_lambda * (e0 / r0);
        R.e0 = (float)(e0 * g.inv_lambda);
        R.r0 = (float)q0;
    }
    R.frac0 = (float)(q0 - rint(q0));
    R.a_hi = (float)A;
    R.a_lo = (float)(A - (double)R.a_hi);
    R.pad[0] = R.pad[1] = R.pad[2] = 0.f;
    return R;
}

// Channel entry h_k(n_c + m) as FP32 complex (re, im) = amp (cos phi, -sin phi).
__device__ __forceinline__ float2 gen_entry_f32(int model, float dprime, const UserConst& c, const UserRef& R,
                                                int m) {
    float mf = (float)m;
    // linear term m*A, exact product plus residual, reduced modulo one cycle
    float p = mf * R.a_hi;
    float pe = fmaf(mf, R.a_hi, -p);
    float pf = p - rintf(p);
    float g = R.frac0 + pf + fmaf(mf, R.a_lo, pe);
    g -= rintf(g);
    float amp;
    if (model == XLMIMO_UPW) {
        amp = c.ampc;
    } else {
        float u = mf * dprime;
        float en = R.e0 + u;
        float r2 = fmaf(en, en, c.xl2);
        float rs = rsqrtf(r2);
        float rp = r2 * rs;
        float sum = R.r0 + rp;
        float den = R.r0 * ((sum - u) * (sum + u));
        float rem = __fdividef(c.x2x2 * u * u, den);
        rem -= rintf(rem);
        g += rem;
        g -= rintf(g);
        amp = (model == XLMIMO_FSPL_USW) ? c.ampc * rs : c.ampc * rs * rsqrtf(rp);
    }
    float s, co;
    __sincosf(6.283185307179586f * g, &s, &co);
    return make_float2(amp * co, -amp * s);
}

}  // namespace xl
