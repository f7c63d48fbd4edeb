// Linear receivers from the Gram matrix (Sec. V): ZF (Eq. 21), MMSE, MRC,
// matched or built from another Gram matrix (modified ZF, Sec. V-B), and the
// capacity log2 det (Eq. 9).  One CTA per trial; the K x K complex matrices
// live in shared memory.
//
//   Z = Gf (ZF) or Gf + sigma^2 diag(p)^{-1} (MMSE) is factored Z = L L^H by
//   a right-looking Cholesky: in FP64 for the matched receivers and the
//   capacity, in double-float on the FP32 pipe for the filter of a
//   mismatched receiver unless a pivot shows it ill-conditioned (closely
//   spaced users), which goes to FP64.  X = L^{-1} by forward substitution; then
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
#include "ff.cuh"

namespace xl {

constexpr int SOLVE_THREADS = 128;
static_assert(SOLVE_THREADS >= XLMIMO_MAX_USERS, "load_lower writes the diagonal with one thread per user");
// downlink scratch of mismatched_sinr: |A_kk|^2, per-warp column sums and trace
// shares for up to SOLVE_THREADS / 32 warps
constexpr size_t BF_DL_EXTRA = (size_t)(XLMIMO_MAX_USERS * (1 + SOLVE_THREADS / 32) + SOLVE_THREADS / 32) * sizeof(double);

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

// Pivot and scale of column k of chol_lower, by warp 0 (every lane forms the
// same pivot; lane 0 publishes it).  Returns false when the pivot is not a
// positive finite number.
__device__ __forceinline__ bool chol_pivot(cd* Lk, int k, int K, int lane, float2* dinvf, double* pivd) {
    const double d = Lk[k].x;
    double y = 0.0;
    const bool ok = rsqrt_pivot(d, y);
    if (ok) {
        for (int i = k + 1 + lane; i < K; i += 32) Lk[i] = cmk(Lk[i].x * y, Lk[i].y * y);
    }
    __syncwarp();  // every lane has read the pivot before lane 0 replaces it
    if (lane == 0 && ok) {
        Lk[k] = cmk(d * y, 0.0);
        float yh, yl;
        split_f64(y, yh, yl);
        dinvf[k] = make_float2(yh, yl);
        pivd[k] = d;
    }
    return ok;
}

// In-place lower Cholesky of a Hermitian K x K matrix whose lower triangle
// is stored column by column: T[j K + i] = A_ij for i >= j, so that the
// column being scaled and the trailing entries that a warp updates together
// are contiguous in shared memory (a row-major walk down a column hits one
// bank group 32 times).  Returns 1 on success; T then holds L the same way,
// dinvf[k] = 1 / L_kk as a float pair (hi, lo) and piv[k] = L_kk^2 (for the
// log-determinant, summed lane-parallel by the caller).
// One CTA barrier per column, by look-ahead: while the other warps apply
// column k to the trailing columns k+2.., warp 0 applies it to column k+1
// alone and goes on to that column's pivot and scaling.  The trailing
// triangle is taken from its last column backwards so that consecutive lanes
// walk down one column.  Needs blockDim.x > 32.
__device__ int chol_lower(cd* T, int K, int* flag, float2* dinvf, double* pivd) {
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid < 32 && !chol_pivot(T, 0, K, tid, dinvf, pivd) && tid == 0) *flag = 1;
    __syncthreads();
    for (int k = 0;; ++k) {
        if (*flag) {
            __syncthreads();  // every thread has read the flag before anyone may reset it
            return 0;
        }
        if (k == K - 1) return 1;
        const cd* Lk = T + k * K;
        if (tid < 32) {
            cd* L1 = T + (k + 1) * K;
            const cd l1 = Lk[k + 1];
            for (int i = k + 1 + tid; i < K; i += 32) L1[i] = cmsubc(L1[i], Lk[i], l1);  // A_i,k+1 -= L_ik conj(L_k+1,k)
            __syncwarp();
            if (!chol_pivot(L1, k + 1, K, tid, dinvf, pivd) && tid == 0) *flag = 1;
        } else {
            const int m = K - k - 2;
            const int tri = m * (m + 1) / 2;
            for (int q = tid - 32; q < tri; q += nt - 32) {
                int cr, s;
                tri_index(q, &cr, &s);  // column m-1-cr of the block, entry s down from its diagonal
                const int j = K - 1 - cr, i = j + s;
                T[j * K + i] = cmsubc(T[j * K + i], Lk[i], Lk[j]);  // A_ij -= L_ik conj(L_jk)
            }
        }
        __syncthreads();
    }
}

// sum_k log2(a[k] b[k] scale) over k < K, evaluated by warp 0 with all lanes
// busy and reduced by shuffles; the result is valid in thread 0.  The
// capacity sum_k log2(p_k / sigma^2) + sum_k log2 L_kk^2 takes one logarithm
// per user this way.
__device__ double warp0_sum_log2(const double* a, const double* b, int K, double scale) {
    double acc = 0.0;
    if (threadIdx.x < 32) {
        for (int k = threadIdx.x; k < K; k += 32) acc += log2(a[k] * b[k] * scale);
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
    cf r;
    split_f64(a.x, r.hi.x, r.lo.x);
    split_f64(a.y, r.hi.y, r.lo.y);
    return r;
}

// acc += a b (conj_a: conj(a) b), complex double-float: the real lanes carry
// (re a re b, re a im b) and the imaginary ones (-+ im a im b, +- im a re b).
__device__ __forceinline__ void cf_mac(float2& s, float2& c, const cf& a, const cf& b, bool conj_a) {
    ff2_mac(s, c, make_float2(a.hi.x, a.hi.x), make_float2(a.lo.x, a.lo.x), b.hi, b.lo);
    const float sg = conj_a ? 1.0f : -1.0f;  // re: -/+ im a im b; im: +/- im a re b
    ff2_mac(s, c, make_float2(sg * a.hi.y, -sg * a.hi.y), make_float2(sg * a.lo.y, -sg * a.lo.y),
            make_float2(b.hi.y, b.hi.x), make_float2(b.lo.y, b.lo.x));
}

// acc - a b for normalized double-float complex values (one two-product per
// real term, then renormalized by a fast two-sum).
__device__ __forceinline__ cf cf_fms(const cf& acc, const cf& a, const cf& b) {
    float2 s = acc.hi, c = acc.lo;
    const cf na = {make_float2(-a.hi.x, -a.hi.y), make_float2(-a.lo.x, -a.lo.y)};
    cf_mac(s, c, na, b, false);
    const float2 t = __fadd2_rn(s, c);
    return {t, __fadd2_rn(__fadd2_rn(s, make_float2(-t.x, -t.y)), c)};
}

// a * v for a double-float complex a and a real double-float v = (hi, lo).
__device__ __forceinline__ cf cf_scale(const cf& a, float2 v) {
    float2 s = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
    ff2_mac(s, c, a.hi, a.lo, make_float2(v.x, v.x), make_float2(v.y, v.y));
    const float2 t = __fadd2_rn(s, c);
    return {t, __fadd2_rn(__fadd2_rn(s, make_float2(-t.x, -t.y)), c)};
}

// acc - a conj(b), double-float complex, normalized: the real lanes carry
// (-re a re b, -im a re b), then (-im a im b, +re a im b).
__device__ __forceinline__ cf cf_fms_conj(const cf& acc, const cf& a, const cf& b) {
    float2 s = acc.hi, c = acc.lo;
    ff2_mac(s, c, make_float2(-a.hi.x, -a.hi.y), make_float2(-a.lo.x, -a.lo.y), make_float2(b.hi.x, b.hi.x),
            make_float2(b.lo.x, b.lo.x));
    ff2_mac(s, c, make_float2(-a.hi.y, a.hi.x), make_float2(-a.lo.y, a.lo.x), make_float2(b.hi.y, b.hi.y),
            make_float2(b.lo.y, b.lo.y));
    const float2 t = __fadd2_rn(s, c);
    return {t, __fadd2_rn(__fadd2_rn(s, make_float2(-t.x, -t.y)), c)};
}

// ---- double-float Cholesky (the mismatched receivers' filter matrix)
// A pivot d_k below CHOL_FF_MIN_RATIO times the matrix's own diagonal entry
// d0_k marks the matrix as ill-conditioned (d_k >= lambda_min while
// d0_k <= lambda_max, so the ratio falls with the condition number: closely
// spaced users); the caller then factors it again in FP64.  Above it the
// factor's double-float rounding (~K 2^-48 backward) stays ~2^-27 relative or
// better in the inverse.
constexpr float CHOL_FF_MIN_RATIO = 1.0f / 65536.0f;

// 1/sqrt(d) for d = dh + dl in double-float, FP32 instructions only: the
// MUFU seed y0, r = 1 - d y0^2 with y0^2 and dh y0^2 exact (FMA residuals;
// 1 - t is exact since t lies within 2^-21 of 1), then one third-order step
// y = y0 + y0 (r/2 + 3 r^2/8); |r| ~ 2^-22 leaves (5/16) r^3 ~ 2^-66 and the
// FP32 rounding of the correction ~2^-46 relative.
__device__ __forceinline__ float2 ff_rsqrt(float dh, float dl) {
    const float y0 = rsqrtf(dh);
    const float q = y0 * y0, qe = fmaf(y0, y0, -q);
    const float t = dh * q, te = fmaf(dh, q, -t);
    const float r = (1.0f - t) - (te + fmaf(dh, qe, dl * q));
    const float corr = y0 * (r * fmaf(r, 0.375f, 0.5f));
    const float yh = y0 + corr;
    return make_float2(yh, corr - (yh - y0));
}

// Pivot and scale of column k by warp 0 (every lane forms the same pivot).
// Returns 0, or 1 if the pivot is not a positive finite number, or 2 if it
// is below CHOL_FF_MIN_RATIO d0 or outside [2^-100, 2^100] (FP32 range margin).
__device__ __forceinline__ int chol_pivot_ff(cf* Lk, int k, int K, int lane, float2* dinvf, float d0) {
    const float dh = Lk[k].hi.x, dl = Lk[k].lo.x;
    if (!(dh > 0.0f) || !(dh <= 3.4e38f)) return 1;
    if (dh < CHOL_FF_MIN_RATIO * d0 || dh < 0x1p-100f || dh > 0x1p100f) return 2;
    const float2 y = ff_rsqrt(dh, dl);
    for (int i = k + 1 + lane; i < K; i += 32) Lk[i] = cf_scale(Lk[i], y);
    if (lane == 0) dinvf[k] = y;
    return 0;
}

// chol_lower in double-float (T and L as cf, same layout and look-ahead):
// returns 1 on success (T's strictly lower triangle holds L, dinvf[k] =
// 1 / L_kk; the diagonal of T is not written), 0 if a pivot is not positive
// (flag 1), -1 if the matrix is ill-conditioned (flag 2).  d0: the diagonal
// entries as loaded (FP32).
__device__ int chol_lower_ff(cf* T, int K, int* flag, float2* dinvf, const float* d0) {
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid < 32) {
        const int r = chol_pivot_ff(T, 0, K, tid, dinvf, d0[0]);
        if (r && tid == 0) *flag = r;
    }
    __syncthreads();
    for (int k = 0;; ++k) {
        const int f = *flag;
        if (f) {
            __syncthreads();  // every thread has read the flag before anyone may reset it
            return f == 1 ? 0 : -1;
        }
        if (k == K - 1) return 1;
        const cf* Lk = T + k * K;
        if (tid < 32) {
            cf* L1 = T + (k + 1) * K;
            const cf l1 = Lk[k + 1];
            for (int i = k + 1 + tid; i < K; i += 32) L1[i] = cf_fms_conj(L1[i], Lk[i], l1);
            __syncwarp();
            const int r = chol_pivot_ff(L1, k + 1, K, tid, dinvf, d0[k + 1]);
            if (r && tid == 0) *flag = r;
        } else {
            const int m = K - k - 2;
            const int tri = m * (m + 1) / 2;
            for (int q = tid - 32; q < tri; q += nt - 32) {
                int cr, s;
                tri_index(q, &cr, &s);
                const int j = K - 1 - cr, i = j + s;
                T[j * K + i] = cf_fms_conj(T[j * K + i], Lk[i], Lk[j]);  // A_ij -= L_ik conj(L_jk)
            }
        }
        __syncthreads();
    }
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

// M = X^H X for lower-triangular X (double-float, row stride xs): M_rc =
// sum_{l >= max(r, c)} conj(X_lr) X_lc, upper triangle computed and mirrored,
// written in double-float (normalized) into M (row stride K).
__device__ void gram_of_lower_ff(const cd* X, int xs, cd* M, int K) {
    const cf* F = reinterpret_cast<const cf*>(X);
    cf* FM = reinterpret_cast<cf*>(M);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int P = K * (K + 1) / 2;
    for (int q = tid; q < P; q += nt) {
        int r = 0, rl = K, w = q;
        while (w >= rl) { w -= rl; ++r; --rl; }
        const int c = r + w;  // r <= c
        // two independent double-float chains (even and odd l) for latency, added at the end
        float2 s = make_float2(0.f, 0.f), cc = make_float2(0.f, 0.f), s1 = s, c1 = s;
        int l = c;
        for (; l + 1 < K; l += 2) {
            cf_mac(s, cc, F[l * xs + r], F[l * xs + c], true);
            cf_mac(s1, c1, F[(l + 1) * xs + r], F[(l + 1) * xs + c], true);
        }
        if (l < K) cf_mac(s, cc, F[l * xs + r], F[l * xs + c], true);
        ff2_add(s, cc, s1, c1);
        const float2 t = __fadd2_rn(s, cc);
        const float2 lo = __fadd2_rn(__fadd2_rn(s, make_float2(-t.x, -t.y)), cc);
        FM[r * K + c] = {t, lo};
        FM[c * K + r] = {make_float2(t.x, -t.y), make_float2(lo.x, -lo.y)};
    }
    __syncthreads();
}

// X = L^{-1} (lower triangular, row-major) in double-float.  With L = U D,
// U = L D^{-1} unit lower triangular and D = diag(L_kk), X = D^{-1} U^{-1}:
// U^{-1} by right-looking elimination on the identity (for k = 0..K-2
// subtract U_ik times row k from every row i > k, the (K-k-1) x (k+1) block in
// parallel; one barrier per column, since the unit diagonal needs no row
// scaling), then every row i scaled by 1/L_ii.  L comes from chol_lower,
// column by column (L_ik at T[k K + i], FP64, or double-float when t_ff); its
// strictly lower triangle becomes U in double-float in place (the only part
// read).  dinvf[k] = 1 / L_kk
// (float pair).  X has row stride K + 1: a warp whose lanes cover several
// short rows then spreads over the shared-memory banks instead of hitting
// one bank group once per row.
// In place (X == T, row stride K): X_ij (j <= i) is kept at T[i K + j], the
// upper triangle and diagonal of the factor's column-major storage, which
// the factor's strictly lower part (L_ik at T[k K + i], i > k) never uses.
__device__ void tri_inverse_ff(cd* T, cd* X, int K, const float2* dinvf, bool t_ff) {
    const bool inplace = X == T;
    const int xs = inplace ? K : K + 1;
    const int tid = threadIdx.x, nt = blockDim.x;
    cf* FT = reinterpret_cast<cf*>(T);
    for (int e = tid; e < K * K; e += nt) {
        const int k = e / K, i = e - k * K;
        if (i > k) {
            const cf v = cf_scale(t_ff ? FT[e] : to_cf(T[e]), dinvf[k]);
            FT[e] = v;
        }
    }
    cf* FX = reinterpret_cast<cf*>(X);
    for (int e = tid; e < K * K; e += nt) {
        const int i = e / K, j = e - i * K;
        if (!inplace || j <= i) FX[i * xs + j] = {make_float2(i == j ? 1.0f : 0.0f, 0.0f), make_float2(0.0f, 0.0f)};
    }
    __syncthreads();
    for (int k = 0; k < K - 1; ++k) {
        const cf* Uk = FT + k * K;
        const int rows = K - k - 1, cols = k + 1;
        for (int e = tid; e < rows * cols; e += nt) {
            const int r = e / cols, i = k + 1 + r, j = e - r * cols;
            FX[i * xs + j] = cf_fms(FX[i * xs + j], Uk[i], FX[k * xs + j]);
        }
        __syncthreads();
    }
    for (int e = tid; e < K * K; e += nt) {
        const int i = e / K, j = e - i * K;
        if (j <= i) FX[i * xs + j] = cf_scale(FX[i * xs + j], dinvf[i]);
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

// Gauss-Jordan inverse with partial pivoting in place: A (row-major) becomes
// A^{-1}.  The row interchanges made during the elimination are undone at the
// end as column interchanges, last first.  perm: K ints, col: K complex of
// shared scratch (the pivot column before each step's update).
__device__ int gj_inverse_inplace(cd* A, int K, int* flag, int* piv, int* perm, cd* col) {
    const int tid = threadIdx.x, nt = blockDim.x;
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
            perm[c] = p;
        }
        __syncthreads();
        const int failed = *flag;
        const int p = *piv;
        __syncthreads();  // flag and pivot read by all before they can change
        if (failed) return 0;
        if (p != c) {
            for (int j = tid; j < K; j += nt) {
                const cd t = A[c * K + j];
                A[c * K + j] = A[p * K + j];
                A[p * K + j] = t;
            }
        }
        __syncthreads();
        // the pivot row divided by the pivot (as gj_inverse_dev does, so that an
        // exactly dependent row leaves an exactly zero pivot here too)
        const cd pv = A[c * K + c];
        const cd inv = cdiv(cmk(1.0, 0.0), pv);
        for (int r = tid; r < K; r += nt) col[r] = A[r * K + c];
        __syncthreads();
        for (int j = tid; j < K; j += nt) A[c * K + j] = j == c ? inv : cdiv(A[c * K + j], pv);
        __syncthreads();
        for (int e = tid; e < K * K; e += nt) {
            const int r = e / K, j = e - r * K;
            if (r == c) continue;
            A[e] = j == c ? cmk(-(col[r].x * inv.x - col[r].y * inv.y), -(col[r].x * inv.y + col[r].y * inv.x))
                          : csub(A[e], cmul(col[r], A[c * K + j]));
        }
        __syncthreads();
    }
    for (int c = K - 1; c >= 0; --c) {
        const int q = perm[c];
        if (q != c) {
            for (int r = tid; r < K; r += nt) {
                const cd t = A[r * K + c];
                A[r * K + c] = A[r * K + q];
                A[r * K + q] = t;
            }
        }
        __syncthreads();
    }
    return 1;
}

// Global loads per thread issued together before their results are used
// (the loads of a trial's Gram are latency-bound: one round trip per batch
// instead of one per entry).
constexpr int LOAD_BATCH = 4;

// The lower triangle of c times a Hermitian Gram matrix g (row-major) into
// shared memory column by column, as chol_lower takes it: column j of the
// lower triangle is row j of the upper one conjugated, T[j K + i] =
// c conj(g[j K + i]) for i > j, read and written contiguously.  add[k] (if
// non-NULL) goes onto the diagonal, which the first K threads write (their
// loads issued ahead of the batches) so that only they execute the FP64
// addition; c = 1 (the usual case) costs no multiplication.  Needs
// blockDim.x >= K.
__device__ void load_lower(cd* T, const double2* __restrict__ g, int K, const double* add, double c) {
    const int tid = threadIdx.x, nt = blockDim.x, KK = K * K;
    const double dg = tid < K ? g[tid * K + tid].x : 0.0;
    for (int e0 = tid; e0 < KK; e0 += LOAD_BATCH * nt) {
        double2 v[LOAD_BATCH];
#pragma unroll
        for (int u = 0; u < LOAD_BATCH; ++u) {
            const int e = e0 + u * nt, j = e / K;
            if (e < KK && e - j * K > j) v[u] = g[e];
        }
#pragma unroll
        for (int u = 0; u < LOAD_BATCH; ++u) {
            const int e = e0 + u * nt, j = e / K;
            if (e < KK && e - j * K > j) T[e] = c == 1.0 ? cmk(v[u].x, -v[u].y) : cmk(v[u].x * c, -(v[u].y * c));
        }
    }
    if (tid < K) {
        const double d = c == 1.0 ? dg : dg * c;
        T[tid * K + tid] = cmk(add ? d + add[tid] : d, 0.0);
    }
}

// load_lower in double-float (T as cf), and the diagonal as FP32 into d0.
__device__ void load_lower_ff(cf* T, const double2* __restrict__ g, int K, const double* add, double c, float* d0) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < K * K; e += nt) {
        const int j = e / K, i = e - j * K;
        if (i > j) {
            const double2 v = g[e];
            T[e] = to_cf(c == 1.0 ? cmk(v.x, -v.y) : cmk(v.x * c, -(v.y * c)));
        }
    }
    for (int k = tid; k < K; k += nt) {
        const double d = c == 1.0 ? g[k * K + k].x : g[k * K + k].x * c;
        const cf v = to_cf(cmk(add ? d + add[k] : d, 0.0));
        T[k * K + k] = v;
        d0[k] = v.hi.x;
    }
}

// c g (complex FP64, row-major, global) into shared memory in double-float.
__device__ void load_cf(cd* F, const double2* __restrict__ g, int K, double c) {
    cf* FF = reinterpret_cast<cf*>(F);
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
        const double2 v = g[e];
        const cf w = to_cf(c == 1.0 ? cmk(v.x, v.y) : cmk(v.x * c, v.y * c));
        FF[e] = w;
    }
}

// Power-of-two scale c that brings the largest Gram diagonal of the trial
// near 1 when it lies outside [2^-60, 2^60] (else c = 1).  Every receiver
// quantity is homogeneous in (G, sigma^2): scaling both Gram matrices and the
// noise power by c leaves SINRs and the capacity unchanged, and keeps the
// double-float stages (FP32 exponent range) away from overflow and underflow.
// Executed by warp 0 (exponents compared as integers); valid in every lane.
__device__ double trial_scale(const double2* __restrict__ gf, const double2* __restrict__ gt, int K) {
    int em = 0;
    for (int k = threadIdx.x; k < K; k += 32) {
        const int ef = (int)(((unsigned)__double2hiint(gf[k * K + k].x) >> 20) & 0x7FFu);
        const int et = (int)(((unsigned)__double2hiint(gt[k * K + k].x) >> 20) & 0x7FFu);
        em = max(em, max(ef, et));
    }
    em = __reduce_max_sync(0xffffffffu, em);
    if (em >= 1023 - 60 && em <= 1023 + 60) return 1.0;
    const int sh = min(1000, max(-1000, 1023 - em));
    return __hiloint2double((sh + 1023) << 20, 0);
}

// Sum of the two lanes of a double-float pair as an unevaluated float pair
// (t, e): the value is (double)t + (double)e; FP32 operations only.
__device__ __forceinline__ float2 ff2_fold(float2 s, float2 c) {
    const float t = __fadd_rn(s.x, s.y);
    const float bb = __fsub_rn(t, s.x);
    const float err = __fadd_rn(__fsub_rn(s.x, __fsub_rn(t, bb)), __fsub_rn(s.y, bb));
    return make_float2(t, __fadd_rn(__fadd_rn(c.x, c.y), err));
}

// Sum of the two lanes of a double-float pair, as FP64.
__device__ __forceinline__ double ff2_total(float2 s, float2 c) {
    const float2 f = ff2_fold(s, c);
    return (double)f.x + (double)f.y;
}

// Mismatched-receiver SINR (Sec. V-B) from M and G in double-float (the
// default; mismatched_sinr below is the FP32-correction form):
//   SINR_k = p_k |A_kk|^2 / (sum_{j != k} p_j |A_kj|^2 + sigma^2 Re (A M^H)_kk),
//   A = M G.
// A is never stored: warp w takes users k = w, w + nwarps, ...; lane l forms
// A_kj for j = l (and l + 32 when K > 32) as a dot product of row k of M
// (broadcast) with column j of G (contiguous across lanes), and adds its terms
// to three double-float sums that the warp then reduces by shuffles, so the
// K^3 products cost no FP64 instruction.  The warps leave each user's three
// sums in shared memory; the conversions to FP64 and the divisions then run
// for all users at once, one lane per user (FP64 instructions cost a full
// warp's issue whatever the number of active lanes).
// rec: shared scratch of 3 XLMIMO_MAX_USERS float pairs (the caller's pivot
// arrays, no longer needed at this point).
__device__ void mismatched_sinr_ff(const cf* FM, const cf* FG, const double* p, double s2, int K, double* sinr_t,
                                double* dlbuf, float2 (*rec)[3]) {
    __shared__ float2 pf[XLMIMO_MAX_USERS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    for (int k = tid; k < K; k += blockDim.x) {
        float h, l;
        split_f64(p[k], h, l);
        pf[k] = make_float2(h, l);
    }
    __syncthreads();
    const bool dl = dlbuf != nullptr;
    const float2 z = make_float2(0.f, 0.f);
    // downlink: lane l's column sums sum_{k != j} |A_kj|^2 (j = l, l + 32) over
    // this warp's rows
    float2 cs[2] = {z, z}, cc[2] = {z, z};
    for (int k = warp; k < K; k += nw) {
        const cf* Mk = FM + k * K;
        float2 ss = z, sc = z, is = z, ic = z, ns = z, nc = z;
        for (int j = lane; j < K; j += 32) {
            // four independent double-float chains over l (latency), added at the end
            float2 as = z, ac = z, as1 = z, ac1 = z, as2 = z, ac2 = z, as3 = z, ac3 = z;
            int l = 0;
            for (; l + 3 < K; l += 4) {
                cf_mac(as, ac, Mk[l], FG[l * K + j], false);
                cf_mac(as1, ac1, Mk[l + 1], FG[(l + 1) * K + j], false);
                cf_mac(as2, ac2, Mk[l + 2], FG[(l + 2) * K + j], false);
                cf_mac(as3, ac3, Mk[l + 3], FG[(l + 3) * K + j], false);
            }
            for (; l < K; ++l) cf_mac(as, ac, Mk[l], FG[l * K + j], false);
            ff2_add(as, ac, as1, ac1);
            ff2_add(as2, ac2, as3, ac3);
            ff2_add(as, ac, as2, ac2);
            const float2 ah = __fadd2_rn(as, ac);  // A_kj normalized
            const float2 al = __fadd2_rn(__fadd2_rn(as, make_float2(-ah.x, -ah.y)), ac);
            const cf m = Mk[j];
            ff2_mac(ns, nc, ah, al, m.hi, m.lo);  // (re a re m, im a im m)
            if (j == k) {
                ff2_mac(ss, sc, ah, al, ah, al);  // (re^2, im^2)
            } else if (dl) {
                ff2_mac(cs[j >> 5], cc[j >> 5], ah, al, ah, al);
            } else {
                float2 ps = z, pc = z;
                const float2 pj = pf[j];
                ff2_mac(ps, pc, make_float2(pj.x, pj.x), make_float2(pj.y, pj.y), ah, al);  // p_j a
                ff2_mac(is, ic, ps, pc, ah, al);
            }
        }
        for (int off = 16; off > 0; off >>= 1) {
            float2 o[6];
            const float2 v[6] = {ss, sc, is, ic, ns, nc};
#pragma unroll
            for (int q = 0; q < 6; ++q)
                o[q] = make_float2(__shfl_xor_sync(0xffffffffu, v[q].x, off), __shfl_xor_sync(0xffffffffu, v[q].y, off));
            ff2_add(ss, sc, o[0], o[1]);
            ff2_add(is, ic, o[2], o[3]);
            ff2_add(ns, nc, o[4], o[5]);
        }
        if (lane == 0) {
            rec[k][0] = ff2_fold(ss, sc);
            rec[k][1] = ff2_fold(is, ic);
            rec[k][2] = ff2_fold(ns, nc);
        }
    }
    if (dl) {
        // per-warp column sums: dlbuf[64 + 64 w + j]
        double* colp = dlbuf + XLMIMO_MAX_USERS;
        for (int h = 0; h < 2; ++h) {
            const int j = lane + 32 * h;
            if (j < K) colp[warp * XLMIMO_MAX_USERS + j] = ff2_total(cs[h], cc[h]);
        }
    }
    __syncthreads();
    if (!dl) {
        for (int k = tid; k < K; k += blockDim.x) {
            const double S = (double)rec[k][0].x + (double)rec[k][0].y, I = (double)rec[k][1].x + (double)rec[k][1].y;
            const double N = (double)rec[k][2].x + (double)rec[k][2].y;
            sinr_t[k] = p[k] * S / fma(s2, N, I);
        }
        return;
    }
    // downlink: beta^2 = P_T / tr(M G M^H), tr = sum_k N_k; |A_kk|^2 = S_k;
    // column sums in fixed warp order
    double* colp = dlbuf + XLMIMO_MAX_USERS;
    for (int k = tid; k < K; k += blockDim.x) dlbuf[k] = (double)rec[k][0].x + (double)rec[k][0].y;
    __syncthreads();
    double pt = 0.0, tr = 0.0;
    for (int k = 0; k < K; ++k) {
        pt += p[k];
        tr += (double)rec[k][2].x + (double)rec[k][2].y;
    }
    const double b2 = pt / tr;
    for (int k = tid; k < K; k += blockDim.x) {
        double col = 0.0;
        for (int w = 0; w < nw; ++w) col += colp[w * XLMIMO_MAX_USERS + k];
        sinr_t[k] = b2 * dlbuf[k] / fma(b2, col, s2);
    }
}

// FP32 value nearest to d (within one FP32 rounding plus 2^-48 relative),
// by integer and FP32 instructions only.
__device__ __forceinline__ float f32_of(double d) {
    float h, l;
    split_f64(d, h, l);
    return __fadd_rn(h, l);
}

// D = c (G - Gf): the true Gram minus the filter's Gram, both c-scaled, in
// FP32 (row-major K x K); D = c G when gf is NULL.  With c = 1 (every Gram diagonal within 2^+-60)
// each part is split into float pairs and subtracted on the FP32 pipe:
// (Gh - Gfh) + (Gl - Gfl), whose roundings are u |D| each (u = 2^-24) plus
// 2^-48 |G|; otherwise the difference is formed and scaled in FP64.
__device__ void load_delta(float2* D, const double2* __restrict__ gf, const double2* __restrict__ gt, int K, double c) {
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
        const double2 a = gt[e], b = gf ? gf[e] : make_double2(0.0, 0.0);
        float2 d;
        if (c == 1.0) {
            float ah, al, bh, bl;
            split_f64(a.x, ah, al);
            split_f64(b.x, bh, bl);
            d.x = __fadd_rn(__fsub_rn(ah, bh), __fsub_rn(al, bl));
            split_f64(a.y, ah, al);
            split_f64(b.y, bh, bl);
            d.y = __fadd_rn(__fsub_rn(ah, bh), __fsub_rn(al, bl));
        } else {
            d = make_float2(f32_of((a.x - b.x) * c), f32_of((a.y - b.y) * c));
        }
        D[e] = d;
    }
}

// Mismatched-receiver SINR (Sec. V-B).  M = Z^{-1} is the inverse of the
// filter's matrix Z = Gf (ZF) or Gf + diag(sp) (MMSE, sp_j = sigma^2 / p_j)
// and the receiver meets the true Gram G:
//   SINR_k = p_k |A_kk|^2 / (sum_{j != k} p_j |A_kj|^2 + sigma^2 (A M^H)_kk),  A = M G.
// Since M Z = I, A = I + B with B = M (G - Z) = M D - M diag(sp): only the
// correction B is formed, and (A M^H)_kk = M_kk + sum_j B_kj conj(M_kj).
// Besides being small where the closed form is accurate, this drops the
// inverse's own residual M Z - I from A (its error is dM D, not dM G).
// M is double-float (FM); B = M_hi D is a K^3 product in FP32 (two
// independent chains), then the loading term M_kj sp_j (FMA-exact product of
// the high parts plus the cross terms) is subtracted.  Per entry
//   |dB_kj| <= ((K + 2) u (|M| |D|)_kj + 3 u |M_kj| sp_j + u |B_kj|,  u = 2^-24;
// the signal, interference and noise sums are FP32 too (positive terms for
// the interference), and M_kk enters the noise term in double-float.  Warp w
// takes users k = w, w + nwarps, ...; lane l forms B_kj for j = l (and
// l + 32 when K > 32) from row k of M (broadcast) and column j of D
// (contiguous across lanes), and adds its terms to the three per-user sums,
// reduced by shuffles.  The SINRs are then finished for all users at once,
// one lane per user, in FP64.
// MRC (M = I, no inverse): plus_i = false, D = c G and A = B = D.
// rec: shared scratch of 3 XLMIMO_MAX_USERS floats.  sp: NULL for ZF.
__device__ void mismatched_sinr(const cf* FM, const float2* D, const double* sp, bool plus_i, const double* p,
                                double s2, int K, double* sinr_t, double* dlbuf, float (*rec)[3]) {
    __shared__ float pf[XLMIMO_MAX_USERS];
    __shared__ float2 spf[XLMIMO_MAX_USERS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    for (int k = tid; k < K; k += blockDim.x) {
        pf[k] = f32_of(p[k]);
        float h = 0.f, l = 0.f;
        if (sp) split_f64(sp[k], h, l);
        spf[k] = make_float2(h, l);
    }
    __syncthreads();
    const bool dl = dlbuf != nullptr;
    // downlink: lane l's column sums sum_{k != j} |A_kj|^2 (j = l, l + 32) over
    // this warp's rows
    float cs0 = 0.f, cs1 = 0.f;
    for (int k = warp; k < K; k += nw) {
        const cf* Mk = FM + k * K;
        float ss = 0.f, is = 0.f, ns = 0.f;
        for (int j = lane; j < K; j += 32) {
            // B_kj = sum_l M_kl D_lj: (re, im) chains for even and odd l
            float2 a0 = make_float2(0.f, 0.f), a1 = a0;
            int l = 0;
            for (; l + 1 < K; l += 2) {
                const float2 m0 = Mk[l].hi, d0 = D[l * K + j];
                const float2 m1 = Mk[l + 1].hi, d1 = D[(l + 1) * K + j];
                a0.x = fmaf(m0.x, d0.x, a0.x);
                a0.y = fmaf(m0.x, d0.y, a0.y);
                a1.x = fmaf(m1.x, d1.x, a1.x);
                a1.y = fmaf(m1.x, d1.y, a1.y);
                a0.x = fmaf(-m0.y, d0.y, a0.x);
                a0.y = fmaf(m0.y, d0.x, a0.y);
                a1.x = fmaf(-m1.y, d1.y, a1.x);
                a1.y = fmaf(m1.y, d1.x, a1.y);
            }
            if (l < K) {
                const float2 m0 = Mk[l].hi, d0 = D[l * K + j];
                a0.x = fmaf(m0.x, d0.x, a0.x);
                a0.y = fmaf(m0.x, d0.y, a0.y);
                a0.x = fmaf(-m0.y, d0.y, a0.x);
                a0.y = fmaf(m0.y, d0.x, a0.y);
            }
            float2 b = make_float2(a0.x + a1.x, a0.y + a1.y);
            const cf m = Mk[j];
            if (sp) {
                // b -= M_kj sp_j: p = M_hi sp_hi exactly as p + e
                const float2 sj = spf[j];
                const float2 pr = make_float2(m.hi.x * sj.x, m.hi.y * sj.x);
                const float2 er = make_float2(fmaf(m.lo.x, sj.x, fmaf(m.hi.x, sj.y, fmaf(m.hi.x, sj.x, -pr.x))),
                                              fmaf(m.lo.y, sj.x, fmaf(m.hi.y, sj.y, fmaf(m.hi.y, sj.x, -pr.y))));
                b = make_float2((b.x - pr.x) - er.x, (b.y - pr.y) - er.y);
            }
            ns = fmaf(b.x, m.hi.x, fmaf(b.y, m.hi.y, ns));  // Re(B_kj conj(M_kj))
            const float b2 = fmaf(b.x, b.x, b.y * b.y);
            if (j == k) {
                ss = plus_i ? fmaf(2.f, b.x, b2) : b2;  // |A_kk|^2 - 1, or |A_kk|^2 for MRC
            } else if (dl) {
                if (j < 32) cs0 += b2;
                else cs1 += b2;
            } else {
                is = fmaf(pf[j], b2, is);
            }
        }
        for (int off = 16; off > 0; off >>= 1) {
            ss += __shfl_xor_sync(0xffffffffu, ss, off);
            is += __shfl_xor_sync(0xffffffffu, is, off);
            ns += __shfl_xor_sync(0xffffffffu, ns, off);
        }
        if (lane == 0) {
            rec[k][0] = ss;
            rec[k][1] = is;
            rec[k][2] = ns;
        }
    }
    if (dl) {
        // per-warp column sums: dlbuf[64 + 64 w + j]
        double* colp = dlbuf + XLMIMO_MAX_USERS;
        if (lane < K) colp[warp * XLMIMO_MAX_USERS + lane] = (double)cs0;
        if (lane + 32 < K) colp[warp * XLMIMO_MAX_USERS + lane + 32] = (double)cs1;
    }
    __syncthreads();
    // S_k = |A_kk|^2, N_k = (A M^H)_kk
    const double one = plus_i ? 1.0 : 0.0;
    auto nk = [&](int k) {
        const cf m = FM[k * K + k];
        return one * ((double)m.hi.x + (double)m.lo.x) + (double)rec[k][2];
    };
    if (!dl) {
        for (int k = tid; k < K; k += blockDim.x) {
            const double S = one + (double)rec[k][0];
            sinr_t[k] = p[k] * S / fma(s2, nk(k), (double)rec[k][1]);
        }
        return;
    }
    // downlink: beta^2 = P_T / tr(M G M^H), tr = sum_k N_k; |A_kk|^2 = S_k;
    // column sums in fixed warp order
    double* colp = dlbuf + XLMIMO_MAX_USERS;
    for (int k = tid; k < K; k += blockDim.x) dlbuf[k] = one + (double)rec[k][0];
    __syncthreads();
    double pt = 0.0, tr = 0.0;
    for (int k = 0; k < K; ++k) {
        pt += p[k];
        tr += nk(k);
    }
    const double b2 = pt / tr;
    for (int k = tid; k < K; k += blockDim.x) {
        double col = 0.0;
        for (int w = 0; w < nw; ++w) col += colp[w * XLMIMO_MAX_USERS + k];
        sinr_t[k] = b2 * dlbuf[k] / fma(b2, col, s2);
    }
}


// One trial's receiver, executed by the whole CTA.  gf/gt: this trial's Gram
// matrices (gt == gf when matched); scheme may carry XLMIMO_MISMATCH_FP32
// (the mismatched SINR from the FP32 correction); pw: its K powers; s2: its
// noise power;
// sinr_t, status_t, cap_t: its outputs (cap_t may be NULL).  Dynamic shared
// memory: (2 K^2 + K) complex doubles plus 2 XLMIMO_MAX_USERS doubles, and
// BF_DL_EXTRA bytes more for the downlink scheme from another Gram matrix.
// ONEBUF (matched receivers only: gt == gf, matched = 1): the triangular
// inverse lives in the upper triangle of the factor's buffer and the
// Gauss-Jordan fallback works in place, so K^2 complex doubles plus the
// 2 XLMIMO_MAX_USERS doubles suffice.
template <bool ONEBUF = false>
__device__ void beamform_trial(const double2* __restrict__ gf, const double2* __restrict__ gt, int matched,
                               const double* __restrict__ pw, double s2, int K, int scheme, int power_mode,
                               double* __restrict__ sinr_t, int* __restrict__ status_t, double* __restrict__ cap_t) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int KK = K * K;
    cd* Z = reinterpret_cast<cd*>(smem);
    // K rows of K + 1 (the triangular inverse's padded stride); ONEBUF: the
    // inverse shares Z (matched receivers only)
    cd* X = ONEBUF ? Z : Z + KK;
    double* p = reinterpret_cast<double*>(ONEBUF ? Z + KK : X + KK + K);
    double* dg = p + XLMIMO_MAX_USERS;
    // pivots, MMSE loading and pivot inverses; the mismatched SINR reuses the
    // same bytes for its per-user sums once they are no longer needed
    __shared__ double sbuf[3 * XLMIMO_MAX_USERS];
    double* pivd = sbuf;
    double* sp = sbuf + XLMIMO_MAX_USERS;
    float2* dinvf = reinterpret_cast<float2*>(sbuf + 2 * XLMIMO_MAX_USERS);
    __shared__ int flag, piv, st;
    __shared__ double cs;
    const int tid = threadIdx.x, nt = blockDim.x;
    const bool fp32_corr = (scheme & XLMIMO_MISMATCH_FP32) != 0;
    // a matched receiver factored in double-float (FP64 for an ill-conditioned
    // system), unless the capacity needs the FP64 pivots
    const bool ff_factor = (scheme & XLMIMO_FACTOR_FF) != 0 && cap_t == nullptr;
    scheme &= ~(XLMIMO_MISMATCH_FP32 | XLMIMO_FACTOR_FF);
    bool m_in_z = false;  // M in Z in double-float (else in X in FP64, from Gauss-Jordan)
    if (tid < 32) {
        const double c = trial_scale(gf, gt, K);
        if (tid == 0) { flag = 0; st = 0; cs = c; }
    }
    __syncthreads();
    // the matrices below are c G and the noise power c sigma^2 (s2c); the
    // powers p and the MRC branch, which reads the Gram directly, use sigma^2
    const double c = cs, s2c = c * s2;
    for (int k = tid; k < K; k += nt) {
        double v = pw[k];
        p[k] = (power_mode == XLMIMO_POWER_RXSNR) ? v * s2 / gt[k * K + k].x : v;
        sp[k] = s2c / p[k];  // MMSE diagonal loading sigma^2 / p_k
    }
    __syncthreads();

    // ---- capacity: Cholesky of G + s2 diag(p)^-1 (the MMSE matrix of the true channel)
    const bool mmse_reuse = matched && scheme == XLMIMO_MMSE;
    if (cap_t && !mmse_reuse) {
        load_lower(Z, gt, K, sp, c);
        __syncthreads();
        int ok = chol_lower(Z, K, &flag, dinvf, pivd);
        const double cp = ok ? warp0_sum_log2(pivd, p, K, 1.0 / s2c) : 0.0;
        if (tid == 0) {
            *cap_t = ok ? cp : nan("");
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
        int ok;
        bool z_ff = false;  // the factor in Z is double-float
        if (!matched || ff_factor) {
            // the filter of a mismatched receiver (and a matched one with
            // XLMIMO_FACTOR_FF): double-float factorisation, FP64 when a pivot
            // shows it ill-conditioned (dg is free here)
            float* d0 = reinterpret_cast<float*>(dg);
            load_lower_ff(reinterpret_cast<cf*>(Z), gf, K, scheme == XLMIMO_MMSE ? sp : nullptr, c, d0);
            __syncthreads();
            ok = chol_lower_ff(reinterpret_cast<cf*>(Z), K, &flag, dinvf, d0);
            if (ok < 0) {
                if (tid == 0) flag = 0;
                load_lower(Z, gf, K, scheme == XLMIMO_MMSE ? sp : nullptr, c);
                __syncthreads();
                ok = chol_lower(Z, K, &flag, dinvf, pivd);
            } else {
                z_ff = true;
            }
        } else {
            load_lower(Z, gf, K, scheme == XLMIMO_MMSE ? sp : nullptr, c);
            __syncthreads();
            ok = chol_lower(Z, K, &flag, dinvf, pivd);
        }
        if (ok) {
            if (mmse_reuse && cap_t) {
                const double cp = warp0_sum_log2(pivd, p, K, 1.0 / s2c);
                if (tid == 0) *cap_t = cp;
            }
            tri_inverse_ff(Z, X, K, dinvf, z_ff);  // X = L^{-1}, double-float
            if (matched) {
                // dg_k = sum_{i >= k} |X_ik|^2 in double-float, one conversion per k
                const cf* FX = reinterpret_cast<const cf*>(X);
                for (int k = tid; k < K; k += nt) {
                    float2 s2a = make_float2(0.f, 0.f), c2a = make_float2(0.f, 0.f);
                    for (int i = k; i < K; ++i) {
                        const cf x = FX[i * (ONEBUF ? K : K + 1) + k];
                        ff2_mac(s2a, c2a, x.hi, x.lo, x.hi, x.lo);  // (re^2, im^2)
                    }
                    dg[k] = ((double)s2a.x + (double)c2a.x) + ((double)s2a.y + (double)c2a.y);
                }
                __syncthreads();
            } else {
                // M = X^H X (double-float) into Z (the factor is no longer needed)
                gram_of_lower_ff(X, K + 1, Z, K);
                m_in_z = true;
            }
        } else {
            // not positive definite: Gauss-Jordan on a fresh copy
            if (tid == 0) { flag = 0; st = 1; }
            for (int e = tid; e < KK; e += nt) {
                int r = e / K, col = e - r * K;
                double2 v = gf[e];
                double add = (scheme == XLMIMO_MMSE && r == col) ? sp[r] : 0.0;
                Z[e] = cmk(fma(v.x, c, add), v.y * c);
            }
            __syncthreads();
            __shared__ int gjperm[ONEBUF ? XLMIMO_MAX_USERS : 1];
            __shared__ cd gjcol[ONEBUF ? XLMIMO_MAX_USERS : 1];
            int ok2 = ONEBUF ? gj_inverse_inplace(Z, K, &flag, &piv, gjperm, gjcol) : gj_inverse_dev(Z, X, K, &flag, &piv);
            if (!ok2) {
                if (tid == 0) st = XLMIMO_ESINGULAR;
                __syncthreads();
                for (int k = tid; k < K; k += nt) sinr_t[k] = 0.0;
                if (tid == 0) *status_t = st;
                if (cap_t && mmse_reuse && tid == 0) *cap_t = nan("");
                return;
            }
            if (matched) {
                for (int k = tid; k < K; k += nt) dg[k] = (ONEBUF ? Z : X)[k * K + k].x;
                __syncthreads();
            }
            if (cap_t && mmse_reuse) {
                // recompute the capacity on its own factorisation
                load_lower(Z, gt, K, sp, c);
                __syncthreads();
                int ok3 = chol_lower(Z, K, &flag, dinvf, pivd);
                const double cp = ok3 ? warp0_sum_log2(pivd, p, K, 1.0 / s2c) : 0.0;
                if (tid == 0) {
                    *cap_t = ok3 ? cp : nan("");
                    flag = 0;
                }
                __syncthreads();
            }
        }
    }

    // ---- SINR
    if (matched) {
        const double2* gm = gt;
        double dl_v = 0.0;  // downlink ZF: P_T / (sigma^2 tr(G^-1)) for every user
        if (scheme == XLMIMO_ZF_DL) {
            double pt = 0.0, tr = 0.0;
            for (int k = 0; k < K; ++k) {
                pt += p[k];
                tr += dg[k];
            }
            dl_v = pt / (s2c * tr);
        }
        for (int k = tid; k < K; k += nt) {
            double v;
            if (scheme == XLMIMO_ZF_DL) {
                v = dl_v;
            } else if (scheme == XLMIMO_MRC) {
                double gkk = gm[k * K + k].x;
                double itf = 0.0;
                for (int j = 0; j < K; ++j)
                    if (j != k) { double2 q = gm[k * K + j]; itf += p[j] * (q.x * q.x + q.y * q.y); }
                v = p[k] * gkk * gkk / (itf + s2 * gkk);
            } else {
                v = p[k] / (s2c * dg[k]);
                if (scheme == XLMIMO_MMSE) v -= 1.0;
            }
            sinr_t[k] = v;
        }
    } else {
        // M in double-float, the true Gram into the other buffer (double-float)
        // M in double-float; the true Gram (double-float) or D = c (G - Gf)
        // (FP32, fp32_corr) into the other buffer
        cd* Mb = m_in_z ? Z : X;
        cd* Gb = m_in_z ? X : Z;
        if (!m_in_z) to_cf_inplace(Mb, K);
        double* dlb = scheme == XLMIMO_ZF_DL ? dg + XLMIMO_MAX_USERS : nullptr;
        if (fp32_corr) {
            const bool mrc = scheme == XLMIMO_MRC;
            float2* Db = reinterpret_cast<float2*>(Gb);
            load_delta(Db, mrc ? nullptr : gf, gt, K, c);
            __syncthreads();
            mismatched_sinr(reinterpret_cast<const cf*>(Mb), Db, scheme == XLMIMO_MMSE ? sp : nullptr, !mrc, p, s2c, K,
                            sinr_t, dlb, reinterpret_cast<float(*)[3]>(sbuf));
        } else {
            load_cf(Gb, gt, K, c);
            __syncthreads();
            mismatched_sinr_ff(reinterpret_cast<const cf*>(Mb), reinterpret_cast<const cf*>(Gb), p, s2c, K, sinr_t, dlb,
                               reinterpret_cast<float2(*)[3]>(sbuf));
        }
    }
    if (tid == 0) *status_t = st;
}


// rate_t = sum_k log2(1 + SINR_k) of the trial just computed (Sec. V-C), by
// warp 0 in the same order as sumrate_kernel (lane-strided sums, then a fixed
// shuffle tree).
__device__ void trial_rate(const double* sinr_t, int K, double* rate_t) {
    __syncthreads();  // every thread's SINR writes are visible to the CTA
    if (threadIdx.x < 32) {
        double r = 0.0;
        for (int k = threadIdx.x; k < K; k += 32) r += log2(1.0 + sinr_t[k]);
        for (int off = 16; off > 0; off >>= 1) r += __shfl_xor_sync(0xffffffffu, r, off);
        if (threadIdx.x == 0) *rate_t = r;
    }
}

__global__ void __launch_bounds__(SOLVE_THREADS, 6) beamform_kernel(const double2* __restrict__ gfil,
                                                                 const double2* __restrict__ gtru, int matched,
                                                                 const double* __restrict__ power,
                                                                 const double* __restrict__ noise, int K,
                                                                 int scheme, int power_mode,
                                                                 double* __restrict__ sinr, int* __restrict__ status,
                                                                 double* __restrict__ cap, double* __restrict__ rate) {
    const int64_t b = blockIdx.x;
    const int64_t KK = (int64_t)K * K;
    beamform_trial(gfil + b * KK, gtru + b * KK, matched, power + b * K, noise[b], K, scheme, power_mode,
                   sinr + b * K, status + b, cap ? cap + b : nullptr);
    if (rate) trial_rate(sinr + b * K, K, rate + b);
}

// Matched receivers (gt == gf) with the triangular inverse in the factor's
// buffer: K^2 complex doubles of shared memory instead of 2K^2 + K, so more
// trials per SM (ten at K = 32, registers capped at 48 without spills); the
// same arithmetic as beamform_kernel, result for result.
__global__ void __launch_bounds__(SOLVE_THREADS, 10) beamform_matched_kernel(const double2* __restrict__ g,
                                                                      const double* __restrict__ power,
                                                                      const double* __restrict__ noise, int K,
                                                                      int scheme, int power_mode,
                                                                      double* __restrict__ sinr,
                                                                      int* __restrict__ status,
                                                                      double* __restrict__ cap,
                                                                      double* __restrict__ rate) {
    const int64_t b = blockIdx.x;
    const int64_t KK = (int64_t)K * K;
    beamform_trial<true>(g + b * KK, g + b * KK, 1, power + b * K, noise[b], K, scheme, power_mode, sinr + b * K,
                         status + b, cap ? cap + b : nullptr);
    if (rate) trial_rate(sinr + b * K, K, rate + b);
}

__global__ void __launch_bounds__(SOLVE_THREADS, 10) beamform_ragged_kernel(const DevInst* __restrict__ insts,
                                                                        const int* __restrict__ list,
                                                                        const double2* __restrict__ gram,
                                                                        const double* __restrict__ power, int power_mode,
                                                                        double* __restrict__ sinr,
                                                                        int* __restrict__ status) {
    const int inst = list[blockIdx.x];
    const DevInst in = insts[inst];
    const double2* gm = gram + in.gram_off;
    beamform_trial<true>(gm, gm, 1, power + in.user_off, in.noise, in.k, in.scheme, power_mode, sinr + in.user_off,
                   status + inst, nullptr);
}

int beamform_ragged_prepare() {
    return cuda_status(cudaFuncSetAttribute(beamform_ragged_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024),
                       "ragged receiver attribute");
}

void beamform_trial_launch_bucket(const DevInst* insts, const int* list, int n, int kmax, const double* gram,
                                  const double* power, int power_mode, double* sinr, int* status, cudaStream_t st) {
    // matched receivers with the inverse in the factor's buffer (ONEBUF)
    size_t smem = (size_t)kmax * kmax * sizeof(cd) + 2 * XLMIMO_MAX_USERS * sizeof(double);
    beamform_ragged_kernel<<<n, SOLVE_THREADS, smem, st>>>(insts, list, (const double2*)gram, power, power_mode, sinr,
                                                            status);
}

int launch_beamform(const double* gf, const double* gt, const double* power, const double* noise, int K, int B,
                    int scheme, int power_mode, double* sinr, int* status, double* cap, cudaStream_t st,
                    double* rate) {
    int matched = (gt == nullptr || gt == gf) ? 1 : 0;
    if (!gt) gt = gf;
    size_t KK = (size_t)K * K;
    if (matched) {
        const size_t sm1 = KK * sizeof(cd) + 2 * XLMIMO_MAX_USERS * sizeof(double);
        cudaError_t e = cudaFuncSetAttribute(beamform_matched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             200 * 1024);
        if (e != cudaSuccess) return cuda_status(e, "beamform attribute");
        beamform_matched_kernel<<<B, SOLVE_THREADS, sm1, st>>>((const double2*)gf, power, noise, K,
                                                               scheme & ~XLMIMO_MISMATCH_FP32, power_mode, sinr,
                                                               status, cap, rate);
        return cuda_status(cudaGetLastError(), "beamform launch");
    }
    size_t smem = (2 * KK + K) * sizeof(cd) + 2 * XLMIMO_MAX_USERS * sizeof(double);
    if ((scheme & ~(XLMIMO_MISMATCH_FP32 | XLMIMO_FACTOR_FF)) == XLMIMO_ZF_DL) smem += BF_DL_EXTRA;
    cudaError_t e = cudaFuncSetAttribute(beamform_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return cuda_status(e, "beamform attribute");
    beamform_kernel<<<B, SOLVE_THREADS, smem, st>>>((const double2*)gf, (const double2*)gt, matched, power, noise, K,
                                                    scheme, power_mode, sinr, status, cap, rate);
    return cuda_status(cudaGetLastError(), "beamform launch");
}

}  // namespace xl
