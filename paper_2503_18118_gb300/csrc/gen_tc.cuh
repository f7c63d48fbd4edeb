// Channel generation for the tensor-core Gram kernels by a local expansion
// per 8-element slice (Sec. II-B's spherical-wave entries, evaluated without
// a square root or a division per entry).
//
// Lengths are in wavelengths, phases in cycles.  For a user at (x, y) and an
// element n = n_c + m of a reference span with centre n_c (e0 = y_{n_c} - y,
// r_c = |(x, e0)|, double-float reference phase frac0 and slope A), the
// distance of the element at u = m d (d = spacing / lambda) is
//   r(u) = r_c + u e0 / r_c + R(u),  R = 2 u^2 x^2 / (r_c ((r_c + r)^2 - u^2))
// (exact; see chan_gen.cuh).  Once per slice, at its centre m_s (a half
// integer) and u_s = m_s d, the kernel evaluates in FP32
//   phi_s = frac(frac0 + m_s A + R(u_s))          phase at the centre
//   c1 = d e_s / r_s,  c2 = d^2 x^2 / (2 r_s^3),  c3 = -c1 c2 / r_s
//                                                  d^k r / dt^k / k!, t in elements
//   b0 = 1 / r_s, b1 = -c1 / r_s^2, b2 = (c1^2 - d^2 x^2 / (2 r_s^2)) / r_s^3
//                                                  the same for the amplitude 1/r
// (e_s = e0 + u_s, r_s = r(u_s): one reciprocal square root refined by one
// Newton step, one reciprocal), and each of the slice's entries at t = -7/2
// .. 7/2 is the cubic phi_s + c1 t + c2 t^2 + c3 t^3 and the quadratic
// amplitude b0 + b1 t + b2 t^2: five FMAs, then one sine and one cosine.
// The Taylor remainders after these terms are |r''''| (t d)^4 / 24 <~
// 3 (7/4)^4 / (24 r^3) cycles and ~(7/4 / r)^3 relative; an FP32 emulation
// over the workloads' geometries (users 3-30 m from 16384- to 262144-element
// 100 GHz arrays, 5-50 m from 65536- and 262144-element 28 GHz arrays) puts
// the worst phase error at 2.6e-6 rad (100 GHz) and 5.9e-6 rad (28 GHz) and
// the amplitude error at 2.2e-7 relative.  Users closer than NEAR_DIST
// wavelengths per unit of d to the array axis fall back to the exact
// per-entry formula (gen_pair of chan_gen.cuh), chosen per CTA.
//
// PNUSW has amplitude r^(-3/2) (b0 = r_s^(-3/2), b1 = -3/2 c1 b0 / r_s,
// b2 = 3/8 b0 (5 c1^2 - 2 d^2 x^2 / r_s^2) / r_s^2); the planar wave is the
// linear phase alone with a constant amplitude.
//
// Two independent slices are evaluated side by side in the two lanes of the
// packed FP32x2 instructions: the two 64-element sub-tiles of a stage for
// K <= 32, the two user slots (users k and k + 32) for K <= 64.
#pragma once

#include "tc_common.cuh"

namespace xl {

// Minimum distance of every user from the array axis, in wavelengths per unit
// of spacing / lambda, for the slice expansion (200 wavelengths at half-wave
// spacing; the Taylor remainder grows as (t d)^4 / x^3).
constexpr float NEAR_DIST = 400.0f;

// Per user and reference span, in shared memory (two float4).
struct SpanC {
    float frac0, ah, al, e0;  // phase at the span centre, slope A = ah + al (ah: 15 bits), e0
    float r0, kx, xl2, aw;    // r_c, 2 x^2 / r_c, x^2, amplitude weight
};

__device__ __forceinline__ SpanC make_span_c(const UserRef& R, float xl2, float aw) {
    SpanC s;
    const float ah = __uint_as_float(__float_as_uint(R.a_hi) & 0xFFFFFE00u);
    s.frac0 = R.frac0;
    s.ah = ah;
    s.al = __fadd_rn(__fsub_rn(R.a_hi, ah), R.a_lo);
    s.e0 = R.e0;
    s.r0 = R.r0;
    s.kx = R.kx;
    s.xl2 = xl2;
    s.aw = aw;
    return s;
}

// Expansion coefficients of two slices (one per lane); angles in radians of
// -2 pi phi (the entry is amp (cos(-2 pi phi) + j sin(-2 pi phi))).
struct SliceCo {
    float2 ph, c1, c2, c3;  // angle polynomial in t
    float2 b0, b1, b2;      // amplitude polynomial in t (times the amplitude weight)
};

template <int MODEL>
__device__ __forceinline__ SliceCo slice_co(const SpanC& s0, const SpanC& s1, float2 mc, float dp) {
    const float2 m1 = f2(-1.0f), tp = f2(-6.283185307179586f);
    const float2 frac0 = make_float2(s0.frac0, s1.frac0), ah = make_float2(s0.ah, s1.ah), al = make_float2(s0.al, s1.al);
    const float2 aw = make_float2(s0.aw, s1.aw);
    // linear part: frac(m_s ah) is exact (ah has 15 significant bits, m_s 9)
    const float2 lin = __fadd2_rn(frac2(__fmul2_rn(mc, ah)), __ffma2_rn(mc, al, frac0));
    SliceCo c;
    if (MODEL == XLMIMO_UPW) {
        c.ph = __fmul2_rn(frac2(lin), tp);
        c.c1 = __fmul2_rn(__fadd2_rn(ah, al), tp);
        c.c2 = c.c3 = f2(0.f);
        c.b0 = aw;
        c.b1 = c.b2 = f2(0.f);
        return c;
    }
    const float2 e0 = make_float2(s0.e0, s1.e0), r0 = make_float2(s0.r0, s1.r0), kx = make_float2(s0.kx, s1.kx);
    const float2 xl2 = make_float2(s0.xl2, s1.xl2);
    const float2 dp2 = f2(dp);
    const float2 us = __fmul2_rn(mc, dp2);
    const float2 es = __fadd2_rn(e0, us);
    const float2 r2 = __ffma2_rn(es, es, xl2);
    float2 rs = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
    // one Newton step: rs (3/2 - r2 rs^2 / 2)
    const float2 h = __fmul2_rn(__fmul2_rn(r2, rs), rs);
    rs = __fmul2_rn(rs, __ffma2_rn(h, f2(-0.5f), f2(1.5f)));
    const float2 rn = __fmul2_rn(r2, rs);                     // r_s
    const float2 sum = __fadd2_rn(r0, rn);                    // r_c + r_s
    const float2 nu2 = __fmul2_rn(us, __fmul2_rn(us, m1));    // -u_s^2
    const float2 den = __ffma2_rn(sum, sum, nu2);             // (r_c + r_s)^2 - u_s^2
    const float2 inv = make_float2(rcp_approx(den.x), rcp_approx(den.y));
    const float2 nR = __fmul2_rn(__fmul2_rn(kx, nu2), inv);  // -R(u_s)
    const float2 phi = frac2(__ffma2_rn(nR, m1, lin));
    const float2 c1 = __fmul2_rn(__fmul2_rn(es, rs), dp2);
    const float2 rs2 = __fmul2_rn(rs, rs);
    const float2 q2h = __fmul2_rn(__fmul2_rn(xl2, f2(0.5f * dp * dp)), rs2);  // d^2 x^2 / (2 r_s^2)
    c.ph = __fmul2_rn(phi, tp);
    c.c1 = __fmul2_rn(c1, tp);
    c.c2 = __fmul2_rn(__fmul2_rn(q2h, rs), tp);
    c.c3 = __fmul2_rn(__fmul2_rn(c.c2, c1), __fmul2_rn(rs, m1));
    if (MODEL == XLMIMO_PNUSW) {
        const float2 rh = make_float2(rsqrtf(rn.x), rsqrtf(rn.y));  // r_s^(-1/2)
        const float2 b0 = __fmul2_rn(rs, rh);
        c.b0 = __fmul2_rn(b0, aw);
        c.b1 = __fmul2_rn(__fmul2_rn(c1, f2(-1.5f)), __fmul2_rn(rs, c.b0));
        const float2 p = __ffma2_rn(__fmul2_rn(c1, c1), f2(5.0f), __fmul2_rn(q2h, f2(-4.0f)));
        c.b2 = __fmul2_rn(__fmul2_rn(c.b0, rs2), __fmul2_rn(p, f2(0.375f)));
    } else {
        c.b0 = __fmul2_rn(rs, aw);
        c.b1 = __fmul2_rn(__fmul2_rn(c1, rs2), __fmul2_rn(aw, m1));
        c.b2 = __fmul2_rn(__fmul2_rn(c.b0, rs2), __ffma2_rn(c1, c1, __fmul2_rn(q2h, m1)));
    }
    return c;
}

// Added to a packed pair of 16-bit floats, doubles both (an increment of
// each exponent field: bit 7 of a BF16 half, bit 10 of an FP16 half).  The
// remainders it is applied to are normal numbers or exact zeros; a zero
// becomes the smallest normal number (2^-126 in BF16, 2^-14 ~ 6e-5 in FP16,
// against scaled entries near 1 whose remainders are below 2^-11: the FP16
// path clears it instead).
template <int PREC>
__device__ __forceinline__ uint32_t double_halves(uint32_t w) {
    if (PREC == TCP_F16X3) {
        const uint32_t z = ((w & 0x7FFFu) == 0u ? 0x0000FFFFu : 0u) | ((w & 0x7FFF0000u) == 0u ? 0xFFFF0000u : 0u);
        return (w + 0x04000400u) & ~z;
    }
    return w + 0x00800080u;
}

// 16-bit words of two consecutive entries (a, b) of each lane: hi words and
// lo words, low half = the first entry.  TRUNC: hi by truncation, lo the
// exact remainder rounded; LO2: the lo words hold twice the remainder.
template <int PREC, bool TRUNC, bool LO2>
__device__ __forceinline__ void split_lanes(float2 a, float2 b, uint32_t& hi0, uint32_t& hi1, uint32_t& lo0,
                                            uint32_t& lo1) {
    if (PREC == TCP_F16X3) {
        const __half2 h0 = __floats2half2_rn(a.x, b.x), h1 = __floats2half2_rn(a.y, b.y);
        const float2 f0 = __half22float2(h0), f1 = __half22float2(h1);
        const float2 ra = __fadd2_rn(a, make_float2(-f0.x, -f1.x)), rb = __fadd2_rn(b, make_float2(-f0.y, -f1.y));
        const __half2 l0 = __floats2half2_rn(ra.x, rb.x), l1 = __floats2half2_rn(ra.y, rb.y);
        hi0 = *reinterpret_cast<const uint32_t*>(&h0);
        hi1 = *reinterpret_cast<const uint32_t*>(&h1);
        lo0 = *reinterpret_cast<const uint32_t*>(&l0);
        lo1 = *reinterpret_cast<const uint32_t*>(&l1);
        if (LO2) {
            lo0 = double_halves<PREC>(lo0);
            lo1 = double_halves<PREC>(lo1);
        }
        return;
    }
    if (TRUNC) {
        hi0 = __byte_perm(__float_as_uint(a.x), __float_as_uint(b.x), 0x7632);
        hi1 = __byte_perm(__float_as_uint(a.y), __float_as_uint(b.y), 0x7632);
    } else {
        const __nv_bfloat162 h0 = __floats2bfloat162_rn(a.x, b.x), h1 = __floats2bfloat162_rn(a.y, b.y);
        hi0 = *reinterpret_cast<const uint32_t*>(&h0);
        hi1 = *reinterpret_cast<const uint32_t*>(&h1);
    }
    if (PREC == TCP_BF16) {
        lo0 = lo1 = 0u;
        return;
    }
    // the hi parts back as floats: the upper 16 bits of each value
    const float2 ha = make_float2(__uint_as_float(hi0 << 16), __uint_as_float(hi1 << 16));
    const float2 hb = make_float2(__uint_as_float(hi0 & 0xFFFF0000u), __uint_as_float(hi1 & 0xFFFF0000u));
    const float2 ra = __ffma2_rn(ha, f2(-1.0f), a), rb = __ffma2_rn(hb, f2(-1.0f), b);
    const __nv_bfloat162 l0 = __floats2bfloat162_rn(ra.x, rb.x), l1 = __floats2bfloat162_rn(ra.y, rb.y);
    lo0 = *reinterpret_cast<const uint32_t*>(&l0);
    lo1 = *reinterpret_cast<const uint32_t*>(&l1);
    if (LO2) {
        lo0 = double_halves<PREC>(lo0);
        lo1 = double_halves<PREC>(lo1);
    }
}

// Entries 4h .. 4h + 3 of each lane's slice as 16-bit words w[lane][comp][q]
// (comp: Re hi, Im hi, Re lo, Im lo; q: entries 4h + 2q, 4h + 2q + 1); h may
// differ between the threads of a warp.
// PARTIAL: entry i of lane l is zero for i >= rem[l].
template <int MODEL, int PREC, bool TRUNC, bool LO2, bool PARTIAL>
__device__ __forceinline__ void slice_words(const SliceCo& co, int h, int rem0, int rem1, uint32_t (&w)[2][4][2]) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        float2 re[2], im[2];
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            const int i = 4 * h + 2 * q + hh;
            const float2 T = f2((float)(4 * h) + (float)(2 * q + hh) - 3.5f);
            float2 a, m;
            if (MODEL == XLMIMO_UPW) {
                a = __ffma2_rn(T, co.c1, co.ph);
                m = co.b0;
            } else {
                a = __ffma2_rn(__ffma2_rn(__ffma2_rn(T, co.c3, co.c2), T, co.c1), T, co.ph);
                m = __ffma2_rn(__ffma2_rn(T, co.b2, co.b1), T, co.b0);
            }
            float s0, k0, s1, k1;
            __sincosf(a.x, &s0, &k0);
            __sincosf(a.y, &s1, &k1);
            re[hh] = __fmul2_rn(m, make_float2(k0, k1));
            im[hh] = __fmul2_rn(m, make_float2(s0, s1));
            if (PARTIAL) {
                if (i >= rem0) { re[hh].x = 0.f; im[hh].x = 0.f; }
                if (i >= rem1) { re[hh].y = 0.f; im[hh].y = 0.f; }
            }
        }
        split_lanes<PREC, TRUNC, LO2>(re[0], re[1], w[0][0][q], w[1][0][q], w[0][2][q], w[1][2][q]);
        split_lanes<PREC, TRUNC, LO2>(im[0], im[1], w[0][1][q], w[1][1][q], w[0][3][q], w[1][3][q]);
    }
}

// ---- periodic drain of the tensor-memory accumulator ------------------------
// tcgen05 accumulates in FP32 with each accumulation rounded towards zero, so
// a long sum of positive terms (a Gram diagonal) loses up to one unit in the
// last place per step.  The kernels therefore accumulate a period of
// DRAIN_STAGES stages into the working accumulator W and then add it into a
// running total T (also in tensor memory) with round-to-nearest FP32 adds on
// the CUDA cores; the next period starts W afresh.  The bias is then bounded
// by the steps of one period, whatever the number of elements.

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// T += W (first: T = W) over `cols` columns of this warp's 32 lanes, starting
// at column c0 of W and of T (tmem addresses with the lane quarter in bits 16+).
template <int COLS>
__device__ __forceinline__ void drain_cols(uint32_t w_addr, uint32_t t_addr, bool first) {
#pragma unroll
    for (int c = 0; c < COLS; c += 16) {
        uint32_t a[16], b[16];
        tmem_ld16(w_addr + c, a);
        if (!first) tmem_ld16(t_addr + c, b);
        tmem_wait_ld();
        if (!first) {
#pragma unroll
            for (int j = 0; j < 16; j += 2) {
                const float2 s = __fadd2_rn(make_float2(__uint_as_float(a[j]), __uint_as_float(a[j + 1])),
                                            make_float2(__uint_as_float(b[j]), __uint_as_float(b[j + 1])));
                a[j] = __float_as_uint(s.x);
                a[j + 1] = __float_as_uint(s.y);
            }
        }
        tmem_st16(t_addr + c, a);
    }
    tmem_wait_st();
}

}  // namespace xl
