// Closed-form Gram matrices of "modified ZF" (Sec. V-B), replacing the
// O(N K^2) inner products by O(K^2) formulas (FP64, except the spherical-model
// off-diagonals: distance and phase in double-float, sine, cosine and
// magnitude in FP32; see the kernel).
//
// PNUSW.  Diagonal: the received power of Eq. (4) over P,
//   G~_ii = beta0 / (spacing x_i) * B_i,
//   B_i = (D/2 - y_i)/sqrt(x_i^2 + (D/2 - y_i)^2) + (D/2 + y_i)/sqrt(x_i^2 + (D/2 + y_i)^2),
// D = N spacing (with spacing = lambda/2 this is the bracket of Eq. 4).
// Off-diagonal: rho_ij sqrt(G~_ii G~_jj) with rho_ij of Eq. (6).  The B_i
// factors of Eq. (6) cancel against those of the diagonal, leaving the
// N-independent value
//   G~_ij = beta0 / spacing * sqrt(lambda) |dx| / (d^{3/2} sqrt(x_i x_j)) * e^{j phi_ij},
//   phi_ij = sgn(|x_i| - |x_j|) (2 pi d / lambda - pi/4),  sgn of Eq. (7),
// d the distance between the users, dx = |x_i| - |x_j|.
// Free-space spherical wave (same two steps for the amplitude lambda/(4 pi r)):
//   G~_ii = c2 / (spacing x_i) (atan((D/2 - y_i)/x_i) + atan((D/2 + y_i)/x_i)),
//   G~_ij = c2 / spacing * sqrt(lambda / (d x_i x_j)) e^{j phi_ij},  c2 = (lambda / 4 pi)^2.
// Planar wave: exact, G_ij = beta0 / (r_i r_j) e^{j 2 pi (r_i - r_j)/lambda} D_N(v),
//   D_N(v) = sin(pi N v) / sin(pi v),  v = spacing (sin theta_j - sin theta_i) / lambda.
// Only i <= j is evaluated; the lower triangle is the conjugate mirror, so
// the output is Hermitian by construction.
#include <math.h>

#include "aperture.cuh"
#include "common.cuh"

namespace xl {

__device__ __forceinline__ double2 cis_cycles(double q) {  // e^{j 2 pi q}
    double f = q - rint(q);
    double s, c;
    sincospi(2.0 * f, &s, &c);
    return make_double2(c, s);
}

// Off-diagonal entries (i < j) come first in the index space, then the K
// diagonal entries of every trial, so that each warp runs one kind.  The
// spherical-model off-diagonals form the distance d and reduce the phase
// sgn (2 pi d / lambda - pi/4) in double-float on the FP32 pipe (~2^-44
// relative, from FP64 positions split by integer operations: GB300's FP64
// pipe issues one warp instruction per ~64 cycles per scheduler) and
// evaluate its sine, cosine and the magnitude in FP32: entries carry ~1e-7
// relative error, far below the 1e-4-level stationary-phase error of the
// formula itself.  At most 48 registers: the Monte-Carlo step runs it in
// 64-thread blocks beside three Gram CTAs, which leave 3,328 registers per SM.
__global__ void __maxnreg__(48) closed_form_kernel(Geom g, const double* __restrict__ users, int K, int B,
                                   double2* __restrict__ gram) {
    const int64_t P = (int64_t)K * (K - 1) / 2;
    const int64_t n_off = (int64_t)B * P;
    const int64_t total = n_off + (int64_t)B * K;
    const float c2f = (float)(g.lambda * g.lambda / (16.0 * 3.14159265358979323846 * 3.14159265358979323846));
    auto split = [](double d) {
        ff v;
        split_f64(d, v.hi, v.lo);
        return v;
    };
    const ff inv_l = split(g.inv_lambda);
    // 32-bit index arithmetic whenever the index space fits (a 64-bit division
    // per entry costs more than the entry's arithmetic)
    const bool narrow = total <= 0x7FFFFFFF;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t b;
        int i, j;
        if (e < n_off) {
            int p;
            if (narrow) {
                const int bb = (int)e / (int)P;
                b = bb;
                p = (int)e - bb * (int)P;
            } else {
                b = e / P;
                p = (int)(e - b * P);
            }
            // strict upper-triangle index p -> (i, j), row by row: counted from
            // the end it is the lower-triangle index of (K-2-i, K-1-j)
            int ri, cj;
            tri_index((int)P - 1 - p, &ri, &cj);
            i = K - 2 - ri;
            j = K - 1 - cj;
        } else {
            if (narrow) {
                const int d = (int)(e - n_off), bb = d / K;
                b = bb;
                i = j = d - bb * K;
            } else {
                const int64_t d = e - n_off;
                b = d / K;
                i = j = (int)(d - b * K);
            }
        }
        const double* u = users + b * K * 2;
        double xi = u[2 * i], yi = u[2 * i + 1], xj = u[2 * j], yj = u[2 * j + 1];
        double2 v;
        if (!user_ok(xi, yi) || !user_ok(xj, yj)) {
            v = make_double2(nan(""), nan(""));
        } else if (g.model == XLMIMO_UPW) {
            double ri = sqrt(xi * xi + yi * yi), rj = sqrt(xj * xj + yj * yj);
            double vv = g.spacing * (yj / rj - yi / ri) * g.inv_lambda;
            double sv = sinpi(vv);
            double dir = fabs(sv) < 1e-300 ? (double)g.N : sinpi((double)g.N * vv) / sv;
            double2 ph = cis_cycles((ri - rj) * g.inv_lambda);
            double m = g.beta0 / (ri * rj) * dir;
            v = make_double2(m * ph.x, m * ph.y);
        } else if (i == j) {
            double h = 0.5 * (double)g.N * g.spacing;
            double val;
            if (g.model == XLMIMO_PNUSW) {
                double a = h - yi, c = h + yi;
                val = g.beta0 / (g.spacing * xi) * (a / sqrt(xi * xi + a * a) + c / sqrt(xi * xi + c * c));
            } else {
                double c2 = g.lambda * g.lambda / (16.0 * 3.14159265358979323846 * 3.14159265358979323846);
                val = c2 / (g.spacing * xi) * (atan((h - yi) / xi) + atan((h + yi) / xi));
            }
            v = make_double2(val, 0.0);
        } else {
            // x > 0 for valid users
            const ff Xi = split(xi), Xj = split(xj), dx = ff_sub(Xi, Xj), dy = ff_sub(split(yi), split(yj));
            const ff d = ff_sqrt(ff_add(ff_mul(dx, dx), ff_mul(dy, dy)));
            ff q = ff_add(ff_mul(d, inv_l), ff{-0.125f, 0.0f});  // phase in cycles
            if (!(dx.hi > 0.0f || (dx.hi == 0.0f && dx.lo > 0.0f))) q = ff_neg(q);
            const float fr = __fadd_rn(__fsub_rn(q.hi, rintf(q.hi)), q.lo);
            float sn, cs;
            __sincosf(6.283185307179586f * fr, &sn, &cs);
            const float df = d.hi, xif = Xi.hi, xjf = Xj.hi;
            float m;
            if (g.model == XLMIMO_PNUSW)
                m = (float)(g.beta0 / g.spacing * sqrt(g.lambda)) * fabsf(dx.hi) / (df * sqrtf(df) * sqrtf(xif * xjf));
            else
                m = c2f / (float)g.spacing * sqrtf((float)g.lambda / (df * xif * xjf));
            v = make_double2((double)(m * cs), (double)(m * sn));
        }
        double2* G = gram + b * K * K;
        if (i == j) {
            G[i * K + i] = make_double2(v.x, 0.0);
        } else {
            G[i * K + j] = v;
            G[j * K + i] = make_double2(v.x, -v.y);
        }
    }
}

// Off-diagonal entries (i < j) of every trial times the finite-aperture
// factor (aperture.cuh); the conjugate mirrored, the diagonal untouched.
// lower_only: write conj(G~_ij F_ij) below the diagonal only, keeping G~_ij
// above it (the surrogate's base; see xlmimo_surrogate_gram).
__global__ void aperture_apply_kernel(int mode, double H, double inv_lambda, const double2* __restrict__ users, int K,
                                      int64_t pairs, bool lower_only, double2* __restrict__ gram) {
    const int P = K * (K - 1) / 2;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < pairs; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = r / P;
        int q = (int)(r - b * P), i = 0, rl = K - 1;
        while (q >= rl) { q -= rl; ++i; --rl; }
        const int j = i + 1 + q;
        const double2 ui = users[b * K + i], uj = users[b * K + j];
        const float2 f = aperture_factor(mode, ui.x, ui.y, uj.x, uj.y, H, inv_lambda);
        double2* G = gram + b * K * K;
        const double2 v = G[i * K + j];
        const double re = v.x * f.x - v.y * f.y, im = v.x * f.y + v.y * f.x;
        if (!lower_only) G[i * K + j] = make_double2(re, im);
        G[j * K + i] = make_double2(re, -im);
    }
}

static int aperture_launch(const Geom& g, int mode, const double* users, int K, int B, bool lower_only, double* gram,
                           cudaStream_t st) {
    if (mode == APERTURE_NONE || K < 2) return XLMIMO_OK;
    const int64_t pairs = (int64_t)B * (K * (K - 1) / 2);
    int64_t blocks = (pairs + 255) / 256;
    if (blocks > 16LL * num_sms()) blocks = 16LL * num_sms();
    aperture_apply_kernel<<<(unsigned)blocks, 256, 0, st>>>(mode, 0.5 * (double)g.N * g.spacing, g.inv_lambda,
                                                            (const double2*)users, K, pairs, lower_only,
                                                            (double2*)gram);
    return cuda_status(cudaGetLastError(), "aperture launch");
}

int launch_aperture_apply(const Geom& g, int mode, const double* users, int K, int B, double* gram, cudaStream_t st) {
    return aperture_launch(g, mode, users, K, B, false, gram, st);
}

int launch_aperture_base(const Geom& g, int mode, const double* users, int K, int B, double* gram, cudaStream_t st) {
    return aperture_launch(g, mode, users, K, B, true, gram, st);
}

int launch_closed_form(const Geom& g, const double* users, int K, int B, double* gram, cudaStream_t st, int threads) {
    int64_t total = (int64_t)B * K * (K + 1) / 2;  // off-diagonal pairs plus diagonals
    int64_t blocks = (total + threads - 1) / threads;
    int64_t cap = 16LL * num_sms();
    if (blocks > cap) blocks = cap;
    closed_form_kernel<<<(unsigned)blocks, threads, 0, st>>>(g, users, K, B, (double2*)gram);
    return cuda_status(cudaGetLastError(), "closed_form launch");
}

}  // namespace xl
