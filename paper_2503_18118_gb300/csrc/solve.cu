// Linear receivers from the Gram matrix (Sec. V): ZF (Eq. 21), MMSE, MRC,
// matched or built from another Gram matrix (modified ZF, Sec. V-B), and the
// capacity log2 det (Eq. 9).  One CTA per trial; the K x K complex matrices
// live in shared memory and every solve is FP64.
//
//   Z = Gf (ZF) or Gf + sigma^2 diag(p)^{-1} (MMSE) is factored Z = L L^H by
//   a right-looking Cholesky.  X = L^{-1} by forward substitution; then
//   [Z^{-1}]_kk = sum_i |X_ik|^2 (matched receivers) or M = Z^{-1} = X^H X
//   (mismatched receivers).  A Z that is not numerically positive definite
//   (possible for a closed-form Gf at small N) is inverted by Gauss-Jordan
//   elimination with partial pivoting instead (trial status 1); a zero pivot
//   marks the trial singular (status 4, SINRs 0).
//   Mismatched SINR, receiver W^H = M H^H on the true channel G:
//     SINR_k = p_k |(MG)_kk|^2 / (sum_{j!=k} p_j |(MG)_kj|^2 + sigma^2 (M G M^H)_kk).
//   Capacity: log2 det(I + sigma^{-2} P^{1/2} G P^{1/2})
//            = sum_k log2(p_k / sigma^2) + 2 sum_k log2 L'_kk,  L' the Cholesky
//   factor of G + sigma^2 diag(p)^{-1} (shared with matched MMSE).
#include <math.h>

#include "common.cuh"

namespace xl {

constexpr int SOLVE_THREADS = 128;

struct cd {
    double x, y;
};
__device__ __forceinline__ cd cmk(double a, double b) { return {a, b}; }
__device__ __forceinline__ cd cadd(cd a, cd b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ cd csub(cd a, cd b) { return {a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ cd cmul(cd a, cd b) { return {fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x)}; }
__device__ __forceinline__ cd cmulc(cd a, cd b) { return {fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y)}; }  // a conj(b)
__device__ __forceinline__ double cabs2(cd a) { return fma(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ cd cdivr(cd a, double r) { return {a.x / r, a.y / r}; }
__device__ __forceinline__ cd cdiv(cd a, cd b) {
    double d = b.x * b.x + b.y * b.y;
    return {(a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d};
}
// acc + a b, acc - a b, acc - a conj(b), acc + conj(a) b: four FP64 FMAs each
__device__ __forceinline__ cd cmac(cd acc, cd a, cd b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
    return acc;
}
__device__ __forceinline__ cd cmsub(cd acc, cd a, cd b) {
    acc.x = fma(-a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(-a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
    return acc;
}
__device__ __forceinline__ cd cmsubc(cd acc, cd a, cd b) {
    acc.x = fma(-a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(-a.y, b.x, acc.y);
    acc.y = fma(a.x, b.y, acc.y);
    return acc;
}
__device__ __forceinline__ cd cmacc(cd acc, cd a, cd b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
    return acc;
}

// Row r and column c of the q-th entry of a lower triangle stored row by
// row (c <= r), without FP64 arithmetic.
__device__ __forceinline__ void tri_index(int q, int* r, int* c) {
    int rr = (int)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);
    while ((rr + 1) * (rr + 2) / 2 <= q) ++rr;
    while (rr * (rr + 1) / 2 > q) --rr;
    *r = rr;
    *c = q - rr * (rr + 1) / 2;
}

// 1/sqrt(d) for d > 0 in FP64: FP32 seed and two Newton steps (the FP64 pipe
// runs one warp instruction per ~64 cycles per scheduler whatever the active
// lanes, so single-lane sqrt/divide sequences are kept short).
__device__ __forceinline__ double rsqrt_f64(double d) {
    if (d < 1e-30 || d > 1e30) return 1.0 / sqrt(d);  // outside the FP32 seed's range
    double y = (double)rsqrtf((float)d);
    y = y * fma(-0.5 * d, y * y, 1.5);
    y = y * fma(-0.5 * d, y * y, 1.5);
    return y;
}

// In-place lower Cholesky of the Hermitian K x K matrix A (row-major, lower
// triangle used).  Returns 1 on success; dinv[k] = 1 / L_kk and piv[k] = L_kk^2
// (for the log-determinant, summed lane-parallel by the caller).  Per column:
// pivot, column scale, trailing update of the lower triangle.
__device__ int chol_lower(cd* A, int K, int* flag, double* dinv, double* pivd) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int k = 0; k < K; ++k) {
        if (tid == 0) {
            double d = A[k * K + k].x;
            if (!(d > 0.0) || !isfinite(d)) {
                *flag = 1;
            } else {
                double y = rsqrt_f64(d);
                A[k * K + k] = cmk(d * y, 0.0);
                dinv[k] = y;
                pivd[k] = d;
            }
        }
        __syncthreads();
        const int failed = *flag;
        if (failed) {
            __syncthreads();  // every thread has read the flag before anyone may reset it
            return 0;
        }
        const double iv = dinv[k];
        for (int i = k + 1 + tid; i < K; i += nt) A[i * K + k] = cmk(A[i * K + k].x * iv, A[i * K + k].y * iv);
        __syncthreads();
        const int m = K - k - 1;
        const int tri = m * (m + 1) / 2;
        for (int q = tid; q < tri; q += nt) {
            int r, c;
            tri_index(q, &r, &c);
            const int i = k + 1 + r, j = k + 1 + c;
            A[i * K + j] = cmsubc(A[i * K + j], A[i * K + k], A[j * K + k]);  // -= L_ik conj(L_jk)
        }
        __syncthreads();
    }
    return 1;
}

// sum_k log2(v[k] * scale) over k < K, evaluated by warp 0 with all lanes
// busy and reduced by shuffles; the result is valid in thread 0.
__device__ double warp0_sum_log2(const double* v, int K, double scale) {
    double acc = 0.0;
    if (threadIdx.x < 32) {
        for (int k = threadIdx.x; k < K; k += 32) acc += log2(v[k] * scale);
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    }
    return acc;
}

// ---- double-float (FP32 pair) arithmetic for the triangular inverse and the
// receiver products.  The Cholesky factorisation stays FP64; what follows it
// -- the inverse X = L^{-1}, and for the mismatched receiver M = X^H X and
// A = M G, which cancel heavily (A = I + a small remainder) -- needs more
// than FP32, and FP64 on this GPU issues a warp instruction every ~64 cycles
// per scheduler.  These run in double-float on the FP32 pipe instead
// (48-bit significand): a value is hi + lo (|lo| <= half
// an ulp of hi), products by Dekker's exact two-product (FMA residual) with
// the cross terms hi*lo + lo*hi, sums by Knuth's two-sum on the hi parts with
// the low-order parts summed alongside (~2^-48 relative over K <= 64 terms).
// Real and imaginary lanes travel together through packed FP32x2 operations.
struct cf {
    float2 hi, lo;  // (re, im) high and low parts; same 16 bytes as a cd
};

__device__ __forceinline__ cf to_cf(cd a) {
    const float rh = (float)a.x, ih = (float)a.y;
    return {make_float2(rh, ih), make_float2((float)(a.x - (double)rh), (float)(a.y - (double)ih))};
}

__device__ __forceinline__ cd from_cf(cf a) {
    return cmk((double)a.hi.x + (double)a.lo.x, (double)a.hi.y + (double)a.lo.y);
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

// acc += a b (conj_a: conj(a) b), complex double-float: the real lanes carry
// (re a re b, re a im b) and the imaginary ones (-+ im a im b, +- im a re b).
__device__ __forceinline__ void cf_mac(float2& s, float2& c, const cf& a, const cf& b, bool conj_a) {
    ff2_mac(s, c, make_float2(a.hi.x, a.hi.x), make_float2(a.lo.x, a.lo.x), b.hi, b.lo);
    const float sg = conj_a ? 1.0f : -1.0f;  // re: -/+ im a im b; im: +/- im a re b
    ff2_mac(s, c, make_float2(sg * a.hi.y, -sg * a.hi.y), make_float2(sg * a.lo.y, -sg * a.lo.y),
            make_float2(b.hi.y, b.hi.x), make_float2(b.lo.y, b.lo.x));
}

__device__ __forceinline__ cd cf_result(float2 s, float2 c) { return cmk((double)s.x + (double)c.x, (double)s.y + (double)c.y); }

// acc - a b for normalized double-float complex values (one two-product per
// real term, then renormalized by a fast two-sum).
__device__ __forceinline__ cf cf_fms(const cf& acc, const cf& a, const cf& b) {
    float2 s = acc.hi, c = acc.lo;
    const cf na = {make_float2(-a.hi.x, -a.hi.y), make_float2(-a.lo.x, -a.lo.y)};
    cf_mac(s, c, na, b, false);
    const float2 t = __fadd2_rn(s, c);
    return {t, __fadd2_rn(__fadd2_rn(s, make_float2(-t.x, -t.y)), c)};
}

// a * v for a double-float complex a and a real FP64 v (as hi + lo).
__device__ __forceinline__ cf cf_scale(const cf& a, double v) {
    const float vh = (float)v, vl = (float)(v - (double)vh);
    float2 s = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
    ff2_mac(s, c, a.hi, a.lo, make_float2(vh, vh), make_float2(vl, vl));
    const float2 t = __fadd2_rn(s, c);
    return {t, __fadd2_rn(__fadd2_rn(s, make_float2(-t.x, -t.y)), c)};
}

// In place: a K x K complex FP64 matrix becomes double-float (same bytes).
__device__ void to_cf_inplace(cd* A, int K) {
    const int tid = threadIdx.x, nt = blockDim.x;
    cf* F = reinterpret_cast<cf*>(A);
    for (int e = tid; e < K * K; e += nt) {
        const cf v = to_cf(A[e]);
        F[e] = v;
    }
    __syncthreads();
}

// M = X^H X for lower-triangular X (double-float): M_rc = sum_{l >= max(r, c)}
// conj(X_lr) X_lc, upper triangle computed and mirrored, written in
// double-float (normalized) into M.
__device__ void gram_of_lower_ff(const cd* X, cd* M, int K) {
    const cf* F = reinterpret_cast<const cf*>(X);
    cf* FM = reinterpret_cast<cf*>(M);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int P = K * (K + 1) / 2;
    for (int q = tid; q < P; q += nt) {
        int r = 0, rl = K, w = q;
        while (w >= rl) { w -= rl; ++r; --rl; }
        const int c = r + w;  // r <= c
        float2 s = make_float2(0.f, 0.f), cc = make_float2(0.f, 0.f);
        for (int l = c; l < K; ++l) cf_mac(s, cc, F[l * K + r], F[l * K + c], true);
        const float2 t = __fadd2_rn(s, cc);
        const float2 lo = __fadd2_rn(__fadd2_rn(s, make_float2(-t.x, -t.y)), cc);
        FM[r * K + c] = {t, lo};
        FM[c * K + r] = {make_float2(t.x, -t.y), make_float2(lo.x, -lo.y)};
    }
    __syncthreads();
}

// X = L^{-1} (lower triangular) in double-float by right-looking elimination
// on the identity: for k = 0..K-1 scale row k by 1/L_kk, then subtract L_ik
// times row k from every row i > k, the (K-k-1) x (k+1) block in parallel.
// The strictly lower triangle of the FP64 factor L is converted in place (the
// only part read), X is left in double-float; dinv[k] = 1 / L_kk (FP64).
__device__ void tri_inverse_ff(cd* L, cd* X, int K, const double* dinv) {
    {
        cf* F = reinterpret_cast<cf*>(L);
        const int P = K * (K - 1) / 2;
        for (int q = threadIdx.x; q < P; q += blockDim.x) {
            int r = 1, w = q;
            while (w >= r) { w -= r; ++r; }
            const int e = r * K + w;  // row r > column w
            const cf v = to_cf(L[e]);
            F[e] = v;
        }
        __syncthreads();
    }
    const cf* FL = reinterpret_cast<const cf*>(L);
    cf* FX = reinterpret_cast<cf*>(X);
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < K * K; e += nt)
        FX[e] = {make_float2((e / K) == (e % K) ? 1.0f : 0.0f, 0.0f), make_float2(0.0f, 0.0f)};
    __syncthreads();
    for (int k = 0; k < K; ++k) {
        const double iv = dinv[k];
        for (int j = tid; j <= k; j += nt) FX[k * K + j] = cf_scale(FX[k * K + j], iv);
        __syncthreads();
        const int rows = K - k - 1, cols = k + 1;
        for (int e = tid; e < rows * cols; e += nt) {
            const int i = k + 1 + e / cols, j = e - (e / cols) * cols;
            FX[i * K + j] = cf_fms(FX[i * K + j], FL[i * K + k], FX[k * K + j]);
        }
        __syncthreads();
    }
}

// Z = M G with M already in double-float (mcf) or FP64 (converted in place),
// G converted in place; Z written as FP64.
__device__ void prod_ff(cd* Mx, bool mcf, cd* G, cd* Z, int K) {
    if (!mcf) to_cf_inplace(Mx, K);
    to_cf_inplace(G, K);
    const cf* FM = reinterpret_cast<const cf*>(Mx);
    const cf* FG = reinterpret_cast<const cf*>(G);
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < K * K; e += nt) {
        const int r = e / K, c = e - r * K;
        float2 s = make_float2(0.f, 0.f), cc = make_float2(0.f, 0.f);
        for (int l = 0; l < K; ++l) cf_mac(s, cc, FM[r * K + l], FG[l * K + c], false);
        Z[e] = cf_result(s, cc);
    }
    __syncthreads();
}

// Gauss-Jordan inverse with partial pivoting: A is destroyed, X = A^{-1}.
__device__ int gj_inverse_dev(cd* A, cd* X, int K, int* flag, int* piv) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < K * K; e += nt) X[e] = cmk((e / K) == (e % K) ? 1.0 : 0.0, 0.0);
    __syncthreads();
    for (int c = 0; c < K; ++c) {
        if (tid == 0) {
            int p = c;
            double best = cabs2(A[c * K + c]);
            for (int r = c + 1; r < K; ++r) {
                double v = cabs2(A[r * K + c]);
                if (v > best) { best = v; p = r; }
            }
            if (!(best > 0.0) || !isfinite(best)) *flag = 1;
            *piv = p;
        }
        __syncthreads();
        const int failed = *flag;
        const int p = *piv;
        __syncthreads();  // flag and pivot read by all before they can change
        if (failed) return 0;
        if (p != c) {
            for (int j = tid; j < K; j += nt) {
                cd t = A[c * K + j]; A[c * K + j] = A[p * K + j]; A[p * K + j] = t;
                t = X[c * K + j]; X[c * K + j] = X[p * K + j]; X[p * K + j] = t;
            }
        }
        __syncthreads();
        cd pv = A[c * K + c];
        __syncthreads();
        for (int j = tid; j < K; j += nt) {
            A[c * K + j] = cdiv(A[c * K + j], pv);
            X[c * K + j] = cdiv(X[c * K + j], pv);
        }
        __syncthreads();
        for (int e = tid; e < K * K; e += nt) {
            int r = e / K, j = e - r * K;
            if (r == c) continue;
            cd f = A[r * K + c];
            if (j == c) continue;  // column c of A handled below
            A[r * K + j] = csub(A[r * K + j], cmul(f, A[c * K + j]));
            X[r * K + j] = csub(X[r * K + j], cmul(f, X[c * K + j]));
        }
        __syncthreads();
        for (int r = tid; r < K; r += nt) {
            if (r == c) continue;
            cd f = A[r * K + c];
            X[r * K + c] = csub(X[r * K + c], cmul(f, X[c * K + c]));
            A[r * K + c] = cmk(0.0, 0.0);
        }
        __syncthreads();
    }
    return 1;
}

// One trial's receiver, executed by the whole CTA.  gf/gt: this trial's Gram
// matrices (gt == gf when matched); pw: its K powers; s2: its noise power;
// sinr_t, status_t, cap_t: its outputs (cap_t may be NULL).  Dynamic shared
// memory: (matched ? 2 : 3) K^2 complex doubles plus 2 XLMIMO_MAX_USERS doubles.
__device__ void beamform_trial(const double2* __restrict__ gf, const double2* __restrict__ gt, int matched,
                               const double* __restrict__ pw, double s2, int K, int scheme, int power_mode,
                               double* __restrict__ sinr_t, int* __restrict__ status_t, double* __restrict__ cap_t) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int KK = K * K;
    cd* Z = reinterpret_cast<cd*>(smem);
    cd* X = Z + KK;
    cd* G = X + KK;  // true Gram (mismatched only)
    double* p = reinterpret_cast<double*>(G + (matched ? 0 : KK));
    double* dg = p + XLMIMO_MAX_USERS;
    __shared__ double dinv[XLMIMO_MAX_USERS], pivd[XLMIMO_MAX_USERS], sp[XLMIMO_MAX_USERS];
    __shared__ int flag, piv, st;
    const int tid = threadIdx.x, nt = blockDim.x;
    bool m_is_cf = false;  // X holds M in double-float (else FP64)
    if (tid == 0) { flag = 0; st = 0; }
    for (int k = tid; k < K; k += nt) {
        double v = pw[k];
        p[k] = (power_mode == XLMIMO_POWER_RXSNR) ? v * s2 / gt[k * K + k].x : v;
        sp[k] = s2 / p[k];  // MMSE diagonal loading sigma^2 / p_k
    }
    if (!matched)
        for (int e = tid; e < KK; e += nt) G[e] = cmk(gt[e].x, gt[e].y);
    __syncthreads();

    // ---- capacity: Cholesky of G + s2 diag(p)^-1 (the MMSE matrix of the true channel)
    const bool mmse_reuse = matched && scheme == XLMIMO_MMSE;
    if (cap_t && !mmse_reuse) {
        for (int e = tid; e < KK; e += nt) {
            int r = e / K, c = e - r * K;
            double2 v = gt[e];
            Z[e] = cmk(v.x + (r == c ? sp[r] : 0.0), r == c ? 0.0 : v.y);
        }
        __syncthreads();
        int ok = chol_lower(Z, K, &flag, dinv, pivd);
        double ld = ok ? warp0_sum_log2(pivd, K, 1.0) : 0.0;
        double lp = warp0_sum_log2(p, K, 1.0 / s2);
        if (tid == 0) {
            *cap_t = ok ? lp + ld : nan("");
            flag = 0;
        }
        __syncthreads();
    }

    // ---- receiver matrix Z
    if (scheme == XLMIMO_MRC) {
        if (tid == 0) st = 0;
        for (int e = tid; e < KK; e += nt) X[e] = cmk((e / K) == (e % K) ? 1.0 : 0.0, 0.0);  // M = I
        __syncthreads();
    } else {
        for (int e = tid; e < KK; e += nt) {
            int r = e / K, c = e - r * K;
            double2 v = gf[e];
            double add = (scheme == XLMIMO_MMSE && r == c) ? sp[r] : 0.0;
            Z[e] = cmk(v.x + add, r == c ? 0.0 : v.y);
        }
        __syncthreads();
        int ok = chol_lower(Z, K, &flag, dinv, pivd);
        if (ok) {
            if (mmse_reuse && cap_t) {
                double ld = warp0_sum_log2(pivd, K, 1.0);
                double lp = warp0_sum_log2(p, K, 1.0 / s2);
                if (tid == 0) *cap_t = lp + ld;
            }
            tri_inverse_ff(Z, X, K, dinv);  // X = L^{-1}, double-float
            if (matched) {
                // dg_k = sum_{i >= k} |X_ik|^2 in double-float, one conversion per k
                const cf* FX = reinterpret_cast<const cf*>(X);
                for (int k = tid; k < K; k += nt) {
                    float2 s2a = make_float2(0.f, 0.f), c2a = make_float2(0.f, 0.f);
                    for (int i = k; i < K; ++i) {
                        const cf x = FX[i * K + k];
                        ff2_mac(s2a, c2a, x.hi, x.lo, x.hi, x.lo);  // (re^2, im^2)
                    }
                    dg[k] = ((double)s2a.x + (double)c2a.x) + ((double)s2a.y + (double)c2a.y);
                }
                __syncthreads();
            } else {
                // M = X^H X (double-float) into Z (the factor is no longer needed), then back into X
                gram_of_lower_ff(X, Z, K);
                for (int e = tid; e < KK; e += nt) X[e] = Z[e];
                __syncthreads();
                m_is_cf = true;
            }
        } else {
            // not positive definite: Gauss-Jordan on a fresh copy
            if (tid == 0) { flag = 0; st = 1; }
            for (int e = tid; e < KK; e += nt) {
                int r = e / K, c = e - r * K;
                double2 v = gf[e];
                double add = (scheme == XLMIMO_MMSE && r == c) ? sp[r] : 0.0;
                Z[e] = cmk(v.x + add, v.y);
            }
            __syncthreads();
            int ok2 = gj_inverse_dev(Z, X, K, &flag, &piv);
            if (!ok2) {
                if (tid == 0) st = XLMIMO_ESINGULAR;
                __syncthreads();
                for (int k = tid; k < K; k += nt) sinr_t[k] = 0.0;
                if (tid == 0) *status_t = st;
                if (cap_t && mmse_reuse && tid == 0) *cap_t = nan("");
                return;
            }
            if (matched) {
                for (int k = tid; k < K; k += nt) dg[k] = X[k * K + k].x;
                __syncthreads();
            }
            if (cap_t && mmse_reuse) {
                // recompute the capacity on its own factorisation
                for (int e = tid; e < KK; e += nt) {
                    int r = e / K, c = e - r * K;
                    double2 v = gt[e];
                    Z[e] = cmk(v.x + (r == c ? sp[r] : 0.0), r == c ? 0.0 : v.y);
                }
                __syncthreads();
                int ok3 = chol_lower(Z, K, &flag, dinv, pivd);
                double ld2 = ok3 ? warp0_sum_log2(pivd, K, 1.0) : 0.0;
                double lp = warp0_sum_log2(p, K, 1.0 / s2);
                if (tid == 0) {
                    *cap_t = ok3 ? lp + ld2 : nan("");
                    flag = 0;
                }
                __syncthreads();
            }
        }
    }

    // ---- SINR
    if (matched) {
        const double2* gm = gt;
        for (int k = tid; k < K; k += nt) {
            double v;
            if (scheme == XLMIMO_MRC) {
                double gkk = gm[k * K + k].x;
                double itf = 0.0;
                for (int j = 0; j < K; ++j)
                    if (j != k) { double2 q = gm[k * K + j]; itf += p[j] * (q.x * q.x + q.y * q.y); }
                v = p[k] * gkk * gkk / (itf + s2 * gkk);
            } else {
                v = p[k] / (s2 * dg[k]);
                if (scheme == XLMIMO_MMSE) v -= 1.0;
            }
            sinr_t[k] = v;
        }
    } else {
        // A = M G (M in X) into Z in double-float; X and G are left in double-float
        prod_ff(X, m_is_cf, G, Z, K);
        const cf* FM = reinterpret_cast<const cf*>(X);
        for (int k = tid; k < K; k += nt) {
            double sig = p[k] * cabs2(Z[k * K + k]);
            double itf = 0.0, nz = 0.0;
            for (int j = 0; j < K; ++j) {
                cd a = Z[k * K + j];
                if (j != k) itf = fma(p[j], cabs2(a), itf);
                nz += cmulc(a, from_cf(FM[k * K + j])).x;  // (A M^H)_kk
            }
            sinr_t[k] = sig / fma(s2, nz, itf);
        }
    }
    if (tid == 0) *status_t = st;
}


__global__ void __launch_bounds__(SOLVE_THREADS) beamform_kernel(const double2* __restrict__ gfil,
                                                                 const double2* __restrict__ gtru, int matched,
                                                                 const double* __restrict__ power,
                                                                 const double* __restrict__ noise, int K,
                                                                 int scheme, int power_mode,
                                                                 double* __restrict__ sinr, int* __restrict__ status,
                                                                 double* __restrict__ cap) {
    const int64_t b = blockIdx.x;
    const int64_t KK = (int64_t)K * K;
    beamform_trial(gfil + b * KK, gtru + b * KK, matched, power + b * K, noise[b], K, scheme, power_mode,
                   sinr + b * K, status + b, cap ? cap + b : nullptr);
}

__global__ void __launch_bounds__(SOLVE_THREADS) beamform_ragged_kernel(const DevInst* __restrict__ insts,
                                                                        const int* __restrict__ list,
                                                                        const double2* __restrict__ gram,
                                                                        const double* __restrict__ power, int power_mode,
                                                                        double* __restrict__ sinr,
                                                                        int* __restrict__ status) {
    const int inst = list[blockIdx.x];
    const DevInst in = insts[inst];
    const double2* gm = gram + in.gram_off;
    beamform_trial(gm, gm, 1, power + in.user_off, in.noise, in.k, in.scheme, power_mode, sinr + in.user_off,
                   status + inst, nullptr);
}

int beamform_ragged_prepare() {
    return cuda_status(cudaFuncSetAttribute(beamform_ragged_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024),
                       "ragged receiver attribute");
}

void beamform_trial_launch_bucket(const DevInst* insts, const int* list, int n, int kmax, const double* gram,
                                  const double* power, int power_mode, double* sinr, int* status, cudaStream_t st) {
    size_t smem = 2 * (size_t)kmax * kmax * sizeof(cd) + 2 * XLMIMO_MAX_USERS * sizeof(double);
    beamform_ragged_kernel<<<n, SOLVE_THREADS, smem, st>>>(insts, list, (const double2*)gram, power, power_mode, sinr,
                                                            status);
}

int launch_beamform(const double* gf, const double* gt, const double* power, const double* noise, int K, int B,
                    int scheme, int power_mode, double* sinr, int* status, double* cap, cudaStream_t st) {
    int matched = (gt == nullptr || gt == gf) ? 1 : 0;
    if (!gt) gt = gf;
    size_t KK = (size_t)K * K;
    size_t smem = (matched ? 2 : 3) * KK * sizeof(cd) + 2 * XLMIMO_MAX_USERS * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(beamform_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return cuda_status(e, "beamform attribute");
    beamform_kernel<<<B, SOLVE_THREADS, smem, st>>>((const double2*)gf, (const double2*)gt, matched, power, noise, K,
                                                    scheme, power_mode, sinr, status, cap);
    return cuda_status(cudaGetLastError(), "beamform launch");
}

}  // namespace xl
