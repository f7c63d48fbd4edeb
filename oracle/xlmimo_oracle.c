/*
 * Plain FP64 CPU oracle for near-field XL-MIMO multiuser beamforming
 * (Cui, Park, Alouini, "Channel Capacity Saturation Point and Beamforming
 * Acceleration for Near-Field XL-MIMO Multiuser Communications").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA library; the two agree only through
 * the mathematics written out below.
 *
 * Everything here is the plain definition: channel vectors are built
 * explicitly, the Gram matrix is the explicit inner product of those vectors,
 * matrix inverses are textbook Gauss-Jordan elimination with partial
 * pivoting, determinants are products of elimination pivots.  No blocking,
 * no fusion, no reordering beyond the definitions.  OpenMP only splits the
 * independent Monte-Carlo trials across host cores.
 *
 * Conventions shared with the public C interface (stated, not included):
 *   users  : [B][K][2] doubles, (x_k, y_k) in metres, x_k > 0, the ULA lies
 *            on the y axis centred at the origin (Sec. II-A).
 *   element n = 0..N-1 sits at y_n = (n - (N-1)/2) * spacing.
 *   gram   : [B][K][K][2] doubles (re, im), row-major,
 *            G[i][j] = h_i^H h_j (conjugate on the row user, Sec. III).
 *   model  : 0 = PNUSW (Eq. 3), 1 = free-space USW  (lambda/(4 pi r)) e^{-j2pi r/lambda},
 *            2 = UPW (planar-wave far-field model used as comparison in Sec. V-A).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORC_PNUSW 0
#define ORC_FSPL 1
#define ORC_UPW 2

#define ORC_ZF 0
#define ORC_MMSE 1
#define ORC_MRC 2
#define ORC_ZF_DL 3

#define ORC_POWER_ABS 0
#define ORC_POWER_RXSNR 1

static const double ORC_PI = 3.14159265358979323846;

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Element position on the y axis (Sec. II-A: ULA centred at the origin). */
static double element_y(int64_t n, int64_t N, double spacing) {
    return ((double)n - 0.5 * (double)(N - 1)) * spacing;
}

/* One channel entry h_k(n) between user (x, y) and element at (0, yn). */
static cplx channel_entry(int model, double lambda, double beta0, double x, double y, double yn) {
    if (model == ORC_UPW) {
        /* Planar wave: amplitude and phase referred to the array centre,
         * path difference y_n sin(theta) across the aperture. */
        double r0 = sqrt(x * x + y * y);
        double s = y / r0;
        double path = r0 - yn * s;
        return sqrt(beta0) / r0 * cexp(-I * 2.0 * ORC_PI * path / lambda);
    }
    double r = sqrt(x * x + (yn - y) * (yn - y));
    cplx ph = cexp(-I * 2.0 * ORC_PI * r / lambda);
    if (model == ORC_PNUSW) {
        /* Eq. (3): sqrt(beta0) e^{-j 2 pi r / lambda} / r * sqrt(x / r). */
        return sqrt(beta0) * ph / r * sqrt(x / r);
    }
    /* Free-space spherical wave: (lambda / (4 pi r)) e^{-j 2 pi r / lambda}. */
    return lambda / (4.0 * ORC_PI * r) * ph;
}

/* h[n] for one user, n = 0..N-1, written as (re, im) pairs. */
int oracle_channel(int model, int64_t N, double lambda, double spacing, double beta0,
                   double x, double y, double* h) {
    for (int64_t n = 0; n < N; ++n) {
        cplx v = channel_entry(model, lambda, beta0, x, y, element_y(n, N, spacing));
        h[2 * n] = creal(v);
        h[2 * n + 1] = cimag(v);
    }
    return 0;
}

/* Exact Gram matrix H^H H by explicit inner products over the N elements
 * (Sec. III definition of received power and correlation; Sec. IV Eq. 9). */
int oracle_gram(int model, int64_t N, double lambda, double spacing, double beta0,
                const double* users, int K, int B, double* gram) {
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int b = 0; b < B; ++b) {
        cplx* H = (cplx*)malloc(sizeof(cplx) * (size_t)N * (size_t)K);
        if (!H) { bad = 1; continue; }
        for (int64_t n = 0; n < N; ++n) {
            double yn = element_y(n, N, spacing);
            for (int k = 0; k < K; ++k) {
                const double* u = users + ((size_t)b * K + k) * 2;
                H[(size_t)n * K + k] = channel_entry(model, lambda, beta0, u[0], u[1], yn);
            }
        }
        for (int i = 0; i < K; ++i) {
            for (int j = 0; j < K; ++j) {
                cplx acc = 0.0;
                for (int64_t n = 0; n < N; ++n)
                    acc += conj(H[(size_t)n * K + i]) * H[(size_t)n * K + j];
                double* g = gram + (((size_t)b * K + i) * K + j) * 2;
                g[0] = creal(acc);
                g[1] = cimag(acc);
            }
        }
        free(H);
    }
    return bad ? 3 : 0;
}

/* Uniform rectangular array (URA), the planar-array extension the paper
 * names in the footnote of Sec. II: R rows of N elements on the square
 * lattice of the given spacing in the y-z plane, element (row q, column n) at
 * (0, y_n, z_q) with z_q = (q - (R-1)/2) * spacing, so R = 1 is the ULA of
 * Sec. II-A.  Users stay in the horizontal plane z = 0 through the array
 * centre.  With the 3-D distance r = sqrt(x^2 + (y_n - y)^2 + z_q^2):
 *   PNUSW       sqrt(beta0) e^{-j 2 pi r / lambda} / r * sqrt(x / r)
 *               (Eq. 3: the projection of the element aperture on the
 *               direction of arrival, cos = x / r, x along the array normal);
 *   free space  (lambda / (4 pi r)) e^{-j 2 pi r / lambda};
 *   UPW         the planar wave of the user's direction (elevation 0), whose
 *               path difference across the aperture is y_n sin(theta) for
 *               every row. */
static cplx channel_entry_ura(int model, double lambda, double beta0, double x, double y, double yn,
                              double zq) {
    if (model == ORC_UPW) return channel_entry(model, lambda, beta0, x, y, yn);
    double r = sqrt(x * x + (yn - y) * (yn - y) + zq * zq);
    cplx ph = cexp(-I * 2.0 * ORC_PI * r / lambda);
    if (model == ORC_PNUSW) return sqrt(beta0) * ph / r * sqrt(x / r);
    return lambda / (4.0 * ORC_PI * r) * ph;
}

/* Exact Gram H^H H of the URA by explicit inner products over all R * N
 * elements (row-major element order: row q, then column n). */
int oracle_gram_ura(int model, int64_t N, int64_t R, double lambda, double spacing, double beta0,
                    const double* users, int K, int B, double* gram) {
    int bad = 0;
    int64_t M = N * R;
#pragma omp parallel for schedule(dynamic, 1)
    for (int b = 0; b < B; ++b) {
        cplx* H = (cplx*)malloc(sizeof(cplx) * (size_t)M * (size_t)K);
        if (!H) { bad = 1; continue; }
        for (int64_t q = 0; q < R; ++q) {
            double zq = ((double)q - 0.5 * (double)(R - 1)) * spacing;
            for (int64_t n = 0; n < N; ++n) {
                double yn = element_y(n, N, spacing);
                for (int k = 0; k < K; ++k) {
                    const double* u = users + ((size_t)b * K + k) * 2;
                    H[(size_t)(q * N + n) * K + k] = channel_entry_ura(model, lambda, beta0, u[0], u[1], yn, zq);
                }
            }
        }
        for (int i = 0; i < K; ++i) {
            for (int j = 0; j < K; ++j) {
                cplx acc = 0.0;
                for (int64_t m = 0; m < M; ++m)
                    acc += conj(H[(size_t)m * K + i]) * H[(size_t)m * K + j];
                double* g = gram + (((size_t)b * K + i) * K + j) * 2;
                g[0] = creal(acc);
                g[1] = cimag(acc);
            }
        }
        free(H);
    }
    return bad ? 3 : 0;
}

/* The bracket of Eq. (4), written with the aperture length N*spacing in
 * place of M*lambda/2 (identical for half-wavelength spacing):
 *   (ML - 4y)/sqrt(16x^2 + (ML-4y)^2) + (ML + 4y)/sqrt(16x^2 + (ML+4y)^2),
 * ML = 2 N spacing.  It tends to 2 as N grows (Eq. 5). */
static double power_bracket(int64_t N, double spacing, double x, double y) {
    double ML = 2.0 * (double)N * spacing;
    double a = ML - 4.0 * y, b = ML + 4.0 * y;
    return a / sqrt(16.0 * x * x + a * a) + b / sqrt(16.0 * x * x + b * b);
}

/* sgn of Eq. (7): -1 for x <= 0, +1 for x > 0. */
static double sgn7(double v) { return v > 0.0 ? 1.0 : -1.0; }

/* Closed-form Gram used by "modified ZF" (Sec. V-B):
 *   G~(i,i) = P_i / P from Eq. (4), G~(i,j) = rho_ij sqrt(P_i P_j) / P with
 *   rho_ij from Eq. (6).
 * PNUSW follows Eqs. (4) and (6) with the element spacing generalised
 * (2/lambda -> 1/spacing).  The free-space model uses the same two steps
 * (Riemann integral for the diagonal, stationary phase for the off-diagonal)
 * carried out for the amplitude lambda/(4 pi r) without the projection
 * factor: the diagonal becomes an arctangent pair and the off-diagonal equals
 * the PNUSW one divided by |cos gamma_ij| = ||x_i|-|x_j|| / d_ij.
 * UPW has an exact closed form: the Dirichlet kernel of the angular offset. */
int oracle_closed_form(int model, int64_t N, double lambda, double spacing, double beta0,
                       const double* users, int K, int B, double* gram) {
#pragma omp parallel for schedule(static)
    for (int b = 0; b < B; ++b) {
        const double* U = users + (size_t)b * K * 2;
        for (int i = 0; i < K; ++i) {
            for (int j = 0; j < K; ++j) {
                double xi = U[2 * i], yi = U[2 * i + 1], xj = U[2 * j], yj = U[2 * j + 1];
                cplx g;
                if (model == ORC_UPW) {
                    double ri = sqrt(xi * xi + yi * yi), rj = sqrt(xj * xj + yj * yj);
                    double si = yi / ri, sj = yj / rj;
                    double alpha = 2.0 * ORC_PI * spacing * (sj - si) / lambda;
                    double dir;
                    if (fabs(sin(0.5 * alpha)) < 1e-300)
                        dir = (double)N;
                    else
                        dir = sin(0.5 * (double)N * alpha) / sin(0.5 * alpha);
                    g = beta0 / (ri * rj) * cexp(I * 2.0 * ORC_PI * (ri - rj) / lambda) * dir;
                } else if (model == ORC_PNUSW) {
                    double Pi = beta0 / (spacing * fabs(xi)) * power_bracket(N, spacing, xi, yi);
                    double Pj = beta0 / (spacing * fabs(xj)) * power_bracket(N, spacing, xj, yj);
                    if (i == j) {
                        g = Pi;
                    } else {
                        double dx = fabs(xi) - fabs(xj), dy = yi - yj;
                        double d = sqrt(dx * dx + dy * dy);
                        double rho_mag = sqrt(lambda) * fabs(dx) / pow(dx * dx + dy * dy, 0.75) *
                                         pow(power_bracket(N, spacing, xi, yi), -0.5) *
                                         pow(power_bracket(N, spacing, xj, yj), -0.5);
                        cplx rho = rho_mag * cexp(I * sgn7(dx) * (2.0 * ORC_PI * d / lambda - ORC_PI / 4.0));
                        g = rho * sqrt(Pi * Pj);
                    }
                } else { /* free-space spherical wave */
                    double c2 = (lambda / (4.0 * ORC_PI)) * (lambda / (4.0 * ORC_PI));
                    if (i == j) {
                        double h = 0.5 * (double)N * spacing;
                        g = c2 / (spacing * xi) * (atan((h - yi) / xi) + atan((h + yi) / xi));
                    } else {
                        double dx = fabs(xi) - fabs(xj), dy = yi - yj;
                        double d = sqrt(dx * dx + dy * dy);
                        g = c2 / spacing * sqrt(lambda / (d * xi * xj)) *
                            cexp(I * sgn7(dx) * (2.0 * ORC_PI * d / lambda - ORC_PI / 4.0));
                    }
                }
                double* o = gram + (((size_t)b * K + i) * K + j) * 2;
                o[0] = creal(g);
                o[1] = cimag(g);
            }
        }
    }
    return 0;
}

/* Textbook Gauss-Jordan inverse with partial pivoting, in place on a copy.
 * Returns 0 on success, 1 when a pivot is exactly zero or not finite. */
static int gj_inverse(int K, const cplx* A, cplx* Ainv) {
    int W = 2 * K;
    cplx* T = (cplx*)malloc(sizeof(cplx) * (size_t)K * W);
    if (!T) return 1;
    for (int i = 0; i < K; ++i)
        for (int j = 0; j < W; ++j)
            T[i * W + j] = (j < K) ? A[i * K + j] : (j - K == i ? 1.0 : 0.0);
    int fail = 0;
    for (int c = 0; c < K && !fail; ++c) {
        int p = c;
        for (int r = c + 1; r < K; ++r)
            if (cabs(T[r * W + c]) > cabs(T[p * W + c])) p = r;
        double pm = cabs(T[p * W + c]);
        if (!(pm > 0.0) || !isfinite(pm)) { fail = 1; break; }
        if (p != c)
            for (int j = 0; j < W; ++j) { cplx t = T[c * W + j]; T[c * W + j] = T[p * W + j]; T[p * W + j] = t; }
        cplx piv = T[c * W + c];
        for (int j = 0; j < W; ++j) T[c * W + j] /= piv;
        for (int r = 0; r < K; ++r) {
            if (r == c) continue;
            cplx f = T[r * W + c];
            if (f == 0.0) continue;
            for (int j = 0; j < W; ++j) T[r * W + j] -= f * T[c * W + j];
        }
    }
    if (!fail)
        for (int i = 0; i < K; ++i)
            for (int j = 0; j < K; ++j) Ainv[i * K + j] = T[i * W + K + j];
    free(T);
    return fail;
}

/* log2 det of a Hermitian positive-definite matrix as the sum of log2 of
 * the pivots of Gaussian elimination with partial pivoting. */
static int gauss_log2det(int K, const cplx* A, double* out) {
    cplx* T = (cplx*)malloc(sizeof(cplx) * (size_t)K * K);
    if (!T) return 1;
    memcpy(T, A, sizeof(cplx) * (size_t)K * K);
    cplx det = 1.0;
    double logabs = 0.0;
    int fail = 0;
    for (int c = 0; c < K; ++c) {
        int p = c;
        for (int r = c + 1; r < K; ++r)
            if (cabs(T[r * K + c]) > cabs(T[p * K + c])) p = r;
        if (!(cabs(T[p * K + c]) > 0.0)) { fail = 1; break; }
        if (p != c) {
            for (int j = 0; j < K; ++j) { cplx t = T[c * K + j]; T[c * K + j] = T[p * K + j]; T[p * K + j] = t; }
            det = -det;
        }
        cplx piv = T[c * K + c];
        logabs += log2(cabs(piv));
        det *= piv / cabs(piv);
        for (int r = c + 1; r < K; ++r) {
            cplx f = T[r * K + c] / piv;
            for (int j = c; j < K; ++j) T[r * K + j] -= f * T[c * K + j];
        }
    }
    free(T);
    *out = logabs;
    (void)det;
    return fail;
}

/* Linear receivers from the Gram matrix alone (Sec. V).
 * A linear receiver W^H = M H^H gives, per user k,
 *   w_k^H h_j = (M G)_kj,     ||w_k||^2 = (M G M^H)_kk,
 * so SINR_k = p_k |(MG)_kk|^2 / (sum_{j!=k} p_j |(MG)_kj|^2 + sigma^2 (M G M^H)_kk)
 * with G the true Gram matrix and
 *   ZF   (Eq. 21): M = Gf^{-1}
 *   MMSE          : M = (Gf + sigma^2 diag(p)^{-1})^{-1}
 *   MRC           : M = I
 * where Gf is the Gram matrix the receiver was built from (the exact one, or
 * the closed form of Sec. V-B for modified ZF).
 * ZF_DL: downlink ZF precoding under a total power constraint (the downlink
 * the paper leaves to the reader, Sec. II): W = beta H M with M = Gf^{-1} and
 * beta^2 = P_T / tr(M G M^H), P_T = sum_k p_k; user k receives
 * beta (G M)_kj s_j, so SINR_k = beta^2 |(MG)_kk|^2 / (beta^2 sum_{j!=k}
 * |(MG)_jk|^2 + sigma^2)  (G M = (M G)^H for Hermitian M and G).
 * power_mode 0: power[b][k] is the transmit power p_k.
 * power_mode 1: power[b][k] is the received SNR p_k G_kk / sigma^2 of user k
 *               alone (G = the true Gram matrix), so p_k = snr_k sigma^2 / G_kk.
 * capacity (nullable): log2 det(I + sigma^{-2} diag(p)^{1/2} G diag(p)^{1/2})
 * (Eq. 9 with per-user powers).
 * status[b] = 0 ok, 4 singular receiver matrix (SINR set to 0). */
int oracle_beamform(const double* gram_filter, const double* gram_true, const double* power,
                    const double* noise, int K, int B, int scheme, int power_mode,
                    double* sinr, int* status, double* capacity) {
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 4)
    for (int b = 0; b < B; ++b) {
        size_t kk = (size_t)K * K;
        cplx* Gf = (cplx*)malloc(sizeof(cplx) * kk);
        cplx* G = (cplx*)malloc(sizeof(cplx) * kk);
        cplx* Z = (cplx*)malloc(sizeof(cplx) * kk);
        cplx* M = (cplx*)malloc(sizeof(cplx) * kk);
        cplx* A = (cplx*)malloc(sizeof(cplx) * kk);
        cplx* Q = (cplx*)malloc(sizeof(cplx) * kk);
        double* p = (double*)malloc(sizeof(double) * K);
        if (!Gf || !G || !Z || !M || !A || !Q || !p) { bad = 1; goto done; }
        const double* gf = gram_filter + (size_t)b * kk * 2;
        const double* gt = (gram_true ? gram_true : gram_filter) + (size_t)b * kk * 2;
        for (size_t e = 0; e < kk; ++e) {
            Gf[e] = gf[2 * e] + I * gf[2 * e + 1];
            G[e] = gt[2 * e] + I * gt[2 * e + 1];
        }
        double s2 = noise[b];
        for (int k = 0; k < K; ++k) {
            double v = power[(size_t)b * K + k];
            p[k] = (power_mode == ORC_POWER_RXSNR) ? v * s2 / creal(G[k * K + k]) : v;
        }
        int st = 0;
        if (scheme == ORC_MRC) {
            for (int i = 0; i < K; ++i)
                for (int j = 0; j < K; ++j) M[i * K + j] = (i == j) ? 1.0 : 0.0;
        } else {
            for (size_t e = 0; e < kk; ++e) Z[e] = Gf[e];
            if (scheme == ORC_MMSE)
                for (int k = 0; k < K; ++k) Z[k * K + k] += s2 / p[k];
            if (gj_inverse(K, Z, M)) st = 4;
        }
        if (!st) {
            /* A = M G */
            for (int i = 0; i < K; ++i)
                for (int j = 0; j < K; ++j) {
                    cplx acc = 0.0;
                    for (int l = 0; l < K; ++l) acc += M[i * K + l] * G[l * K + j];
                    A[i * K + j] = acc;
                }
            /* Q = A M^H = M G M^H, only its diagonal is used */
            for (int i = 0; i < K; ++i) {
                cplx acc = 0.0;
                for (int l = 0; l < K; ++l) acc += A[i * K + l] * conj(M[i * K + l]);
                Q[i * K + i] = acc;
            }
            if (scheme == ORC_ZF_DL) {
                /* downlink: W = beta H M, beta^2 = P_T / tr(W^H W / beta^2) = P_T / tr(M G M^H)
                   = P_T / sum_k Q_kk (P_T = sum_k p_k); user k receives beta (G M)_k. s with
                   G M = A^H, so SINR_k = beta^2 |A_kk|^2 / (beta^2 sum_{j != k} |A_jk|^2 + s2) */
                double pt = 0.0, tq = 0.0;
                for (int k = 0; k < K; ++k) {
                    pt += p[k];
                    tq += creal(Q[k * K + k]);
                }
                const double b2 = pt / tq;
                for (int k = 0; k < K; ++k) {
                    double sig = b2 * creal(A[k * K + k] * conj(A[k * K + k]));
                    double itf = 0.0;
                    for (int j = 0; j < K; ++j)
                        if (j != k) itf += b2 * creal(A[j * K + k] * conj(A[j * K + k]));
                    sinr[(size_t)b * K + k] = sig / (itf + s2);
                }
            } else {
                for (int k = 0; k < K; ++k) {
                    double sig = p[k] * creal(A[k * K + k] * conj(A[k * K + k]));
                    double itf = 0.0;
                    for (int j = 0; j < K; ++j)
                        if (j != k) itf += p[j] * creal(A[k * K + j] * conj(A[k * K + j]));
                    double den = itf + s2 * creal(Q[k * K + k]);
                    sinr[(size_t)b * K + k] = sig / den;
                }
            }
        } else {
            for (int k = 0; k < K; ++k) sinr[(size_t)b * K + k] = 0.0;
        }
        status[b] = st;
        if (capacity) {
            for (int i = 0; i < K; ++i)
                for (int j = 0; j < K; ++j)
                    Z[i * K + j] = (i == j ? 1.0 : 0.0) + sqrt(p[i]) * G[i * K + j] * sqrt(p[j]) / s2;
            double ld = 0.0;
            if (gauss_log2det(K, Z, &ld)) ld = NAN;
            capacity[b] = ld;
        }
    done:
        free(Gf); free(G); free(Z); free(M); free(A); free(Q); free(p);
    }
    return bad ? 3 : 0;
}

/* Sum rate R_b = sum_k log2(1 + SINR_bk) and its mean and sum of squared
 * deviations over the trials (two plain passes). stats = {mean, M2, count}. */
int oracle_sumrate(const double* sinr, int K, int B, double* rate, double* stats) {
    for (int b = 0; b < B; ++b) {
        double r = 0.0;
        for (int k = 0; k < K; ++k) r += log2(1.0 + sinr[(size_t)b * K + k]);
        rate[b] = r;
    }
    if (stats) {
        double m = 0.0;
        for (int b = 0; b < B; ++b) m += rate[b];
        m = B > 0 ? m / B : 0.0;
        double m2 = 0.0;
        for (int b = 0; b < B; ++b) m2 += (rate[b] - m) * (rate[b] - m);
        stats[0] = m;
        stats[1] = m2;
        stats[2] = (double)B;
    }
    return 0;
}

/* Per-trial power-saturation interval (Sec. IV-A, Eqs. 13-16):
 *   y_up = max_k x_k t / sqrt(1-t^2) + y_k,  y_down = min_k -x_k t / sqrt(1-t^2) + y_k,
 * and the number of elements that spans it, ceil((y_up - y_down) / spacing).
 * sat[b] = {y_up, y_down, n_sat}. */
int oracle_saturation(const double* users, int K, int B, double t, double spacing, double* sat) {
    double a = t / sqrt(1.0 - t * t);
    for (int b = 0; b < B; ++b) {
        double up = -INFINITY, dn = INFINITY;
        for (int k = 0; k < K; ++k) {
            double x = users[((size_t)b * K + k) * 2], y = users[((size_t)b * K + k) * 2 + 1];
            double u = x * a + y, d = -x * a + y;
            if (u > up) up = u;
            if (d < dn) dn = d;
        }
        sat[(size_t)b * 3] = up;
        sat[(size_t)b * 3 + 1] = dn;
        sat[(size_t)b * 3 + 2] = ceil((up - dn) / spacing);
    }
    return 0;
}
