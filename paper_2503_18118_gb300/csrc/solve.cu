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
__device__ __forceinline__ cd cmul(cd a, cd b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ cd cmulc(cd a, cd b) { return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y}; }  // a conj(b)
__device__ __forceinline__ cd cconjmul(cd a, cd b) { return {a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x}; }  // conj(a) b
__device__ __forceinline__ double cabs2(cd a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ cd cdivr(cd a, double r) { return {a.x / r, a.y / r}; }
__device__ __forceinline__ cd cdiv(cd a, cd b) {
    double d = b.x * b.x + b.y * b.y;
    return {(a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d};
}

// In-place lower Cholesky of the Hermitian K x K matrix A (row-major, lower
// triangle used).  Returns 1 on success and sum_k log2 L_kk in *log2det;
// dinv[k] = 1 / L_kk.  Column k is scaled during the pivot phase of column
// k+1 (the trailing update of column k uses the unscaled column and 1/d_k),
// so each column costs two barriers.
__device__ int chol_lower(cd* A, int K, double* log2det, int* flag, double* dinv) {
    const int tid = threadIdx.x, nt = blockDim.x;
    double ld = 0.0;
    for (int k = 0; k < K; ++k) {
        // pivot of column k; scale column k-1 by 1/L_{k-1,k-1}
        if (tid == 0) {
            double d = A[k * K + k].x;
            if (!(d > 0.0) || !isfinite(d)) {
                *flag = 1;
            } else {
                double l = sqrt(d);
                A[k * K + k] = cmk(l, 0.0);
                dinv[k] = 1.0 / l;
            }
        }
        if (k > 0) {
            const double iv = dinv[k - 1];
            for (int i = k + tid; i < K; i += nt) A[i * K + k - 1] = cmk(A[i * K + k - 1].x * iv, A[i * K + k - 1].y * iv);
        }
        __syncthreads();
        const int failed = *flag;
        __syncthreads();  // every thread has read the flag before anyone may reset it
        if (failed) return 0;
        const double lkk = A[k * K + k].x;
        ld += log2(lkk);
        // trailing update with the unscaled column: A_ij -= A_ik conj(A_jk) / d_k
        const double id2 = dinv[k] * dinv[k];
        const int m = K - k - 1;
        for (int e = tid; e < m * m; e += nt) {
            const int r = e / m, c = e - r * m;
            if (c > r) continue;
            const int i = k + 1 + r, j = k + 1 + c;
            cd t = cmulc(A[i * K + k], A[j * K + k]);
            A[i * K + j] = cmk(A[i * K + j].x - t.x * id2, A[i * K + j].y - t.y * id2);
        }
        __syncthreads();
    }
    *log2det = 2.0 * ld;
    return 1;
}

// X = L^{-1} (lower), by forward substitution on the columns of I in parallel.
__device__ void tri_inverse(const cd* L, cd* X, int K, const double* dinv) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < K * K; e += nt) X[e] = cmk(0.0, 0.0);
    __syncthreads();
    for (int i = 0; i < K; ++i) {
        const double iv = dinv[i];
        for (int j = tid; j <= i; j += nt) {
            cd acc = cmk(i == j ? 1.0 : 0.0, 0.0);
            for (int k = j; k < i; ++k) acc = csub(acc, cmul(L[i * K + k], X[k * K + j]));
            X[i * K + j] = cmk(acc.x * iv, acc.y * iv);
        }
        __syncthreads();
    }
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

__global__ void __launch_bounds__(SOLVE_THREADS) beamform_kernel(const double2* __restrict__ gfil,
                                                                 const double2* __restrict__ gtru, int matched,
                                                                 const double* __restrict__ power,
                                                                 const double* __restrict__ noise, int K,
                                                                 int scheme, int power_mode,
                                                                 double* __restrict__ sinr, int* __restrict__ status,
                                                                 double* __restrict__ cap) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int KK = K * K;
    cd* Z = reinterpret_cast<cd*>(smem);
    cd* X = Z + KK;
    cd* G = X + KK;  // true Gram (mismatched only)
    double* p = reinterpret_cast<double*>(G + (matched ? 0 : KK));
    double* dg = p + XLMIMO_MAX_USERS;
    __shared__ double dinv[XLMIMO_MAX_USERS];
    __shared__ int flag, piv, st;
    __shared__ double ld_cap;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int b = blockIdx.x;
    const double2* gf = gfil + (int64_t)b * KK;
    const double2* gt = gtru + (int64_t)b * KK;
    const double s2 = noise[b];
    if (tid == 0) { flag = 0; st = 0; ld_cap = 0.0; }
    for (int k = tid; k < K; k += nt) {
        double v = power[(int64_t)b * K + k];
        p[k] = (power_mode == XLMIMO_POWER_RXSNR) ? v * s2 / gt[k * K + k].x : v;
    }
    if (!matched)
        for (int e = tid; e < KK; e += nt) G[e] = cmk(gt[e].x, gt[e].y);
    __syncthreads();

    // ---- capacity: Cholesky of G + s2 diag(p)^-1 (the MMSE matrix of the true channel)
    const bool mmse_reuse = matched && scheme == XLMIMO_MMSE;
    if (cap && !mmse_reuse) {
        for (int e = tid; e < KK; e += nt) {
            int r = e / K, c = e - r * K;
            double2 v = gt[e];
            Z[e] = cmk(v.x + (r == c ? s2 / p[r] : 0.0), r == c ? 0.0 : v.y);
        }
        __syncthreads();
        double ld = 0.0;
        int ok = chol_lower(Z, K, &ld, &flag, dinv);
        if (tid == 0) {
            double s = 0.0;
            for (int k = 0; k < K; ++k) s += log2(p[k] / s2);
            cap[b] = ok ? s + ld : nan("");
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
            double add = (scheme == XLMIMO_MMSE && r == c) ? s2 / p[r] : 0.0;
            Z[e] = cmk(v.x + add, r == c ? 0.0 : v.y);
        }
        __syncthreads();
        double ld = 0.0;
        int ok = chol_lower(Z, K, &ld, &flag, dinv);
        if (ok) {
            if (mmse_reuse && cap && tid == 0) {
                double s = 0.0;
                for (int k = 0; k < K; ++k) s += log2(p[k] / s2);
                cap[b] = s + ld;
            }
            tri_inverse(Z, X, K, dinv);  // X = L^{-1}
            if (matched) {
                for (int k = tid; k < K; k += nt) {
                    double acc = 0.0;
                    for (int i = k; i < K; ++i) acc += cabs2(X[i * K + k]);
                    dg[k] = acc;
                }
                __syncthreads();
            } else {
                // M = X^H X into Z (Z no longer needed)
                for (int e = tid; e < KK; e += nt) {
                    int r = e / K, c = e - r * K;
                    int l0 = r > c ? r : c;
                    cd acc = cmk(0.0, 0.0);
                    for (int l = l0; l < K; ++l) acc = cadd(acc, cconjmul(X[l * K + r], X[l * K + c]));
                    Z[e] = acc;
                }
                __syncthreads();
                for (int e = tid; e < KK; e += nt) X[e] = Z[e];
                __syncthreads();
            }
        } else {
            // not positive definite: Gauss-Jordan on a fresh copy
            if (tid == 0) { flag = 0; st = 1; }
            for (int e = tid; e < KK; e += nt) {
                int r = e / K, c = e - r * K;
                double2 v = gf[e];
                double add = (scheme == XLMIMO_MMSE && r == c) ? s2 / p[r] : 0.0;
                Z[e] = cmk(v.x + add, v.y);
            }
            __syncthreads();
            int ok2 = gj_inverse_dev(Z, X, K, &flag, &piv);
            if (!ok2) {
                if (tid == 0) st = XLMIMO_ESINGULAR;
                __syncthreads();
                for (int k = tid; k < K; k += nt) sinr[(int64_t)b * K + k] = 0.0;
                if (tid == 0) status[b] = st;
                if (cap && mmse_reuse && tid == 0) cap[b] = nan("");
                return;
            }
            if (matched) {
                for (int k = tid; k < K; k += nt) dg[k] = X[k * K + k].x;
                __syncthreads();
            }
            if (cap && mmse_reuse) {
                // recompute the capacity on its own factorisation
                for (int e = tid; e < KK; e += nt) {
                    int r = e / K, c = e - r * K;
                    double2 v = gt[e];
                    Z[e] = cmk(v.x + (r == c ? s2 / p[r] : 0.0), r == c ? 0.0 : v.y);
                }
                __syncthreads();
                double ld2 = 0.0;
                int ok3 = chol_lower(Z, K, &ld2, &flag, dinv);
                if (tid == 0) {
                    double s = 0.0;
                    for (int k = 0; k < K; ++k) s += log2(p[k] / s2);
                    cap[b] = ok3 ? s + ld2 : nan("");
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
            sinr[(int64_t)b * K + k] = v;
        }
    } else {
        // row k of A = M G (M in X) formed on the fly
        for (int k = tid; k < K; k += nt) {
            double sig = 0.0, itf = 0.0, nz = 0.0;
            for (int j = 0; j < K; ++j) {
                cd a = cmk(0.0, 0.0);
                for (int l = 0; l < K; ++l) a = cadd(a, cmul(X[k * K + l], G[l * K + j]));
                if (j == k) sig = p[k] * cabs2(a);
                else itf += p[j] * cabs2(a);
                nz += cmulc(a, X[k * K + j]).x;  // (A M^H)_kk term
            }
            sinr[(int64_t)b * K + k] = sig / (itf + s2 * nz);
        }
    }
    if (tid == 0) status[b] = st;
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
