// Gram matrices of a uniform rectangular array (URA), the planar-array
// extension named in the footnote of Sec. II, by row decomposition.
//
// R rows of N elements on the square lattice of the spacing d in the y-z
// plane, row q at height z_q = (q - (R-1)/2) d; users in the plane z = 0.
// With r = sqrt(x^2 + (y_n - y)^2 + z_q^2) = sqrt(x'^2 + (y_n - y)^2),
// x' = sqrt(x^2 + z_q^2), row q sees user (x, y) exactly as the ULA of
// Sec. II-A sees a user at (x', y), except that the PNUSW amplitude of Eq. (3)
// projects on the array normal: sqrt(x / r) = sqrt(x' / r) sqrt(x / x').  So
//   G = sum_q m_q diag(w_q) G_ULA(x'_q, y) diag(w_q),
// w_q = sqrt(x / x'_q) for PNUSW and 1 in free space, where rows at +-z_q are
// folded into one evaluation of multiplicity m_q = 2 (1 for the centre row of
// an odd R).  The planar wave of a user at elevation 0 is the same on every
// row: one ULA Gram times R.
//
// At BF16 hi/lo with rows of a multiple of 128 elements, at most 1024
// (spherical-wave models), the tensor-core Gram runs the identity itself, all
// row pairs of a trial in one accumulation (its URA mode).  Otherwise:
// the per-row Grams are the library's ULA Gram launchers (any precision) over
// B * Q virtual trials, Q = ceil(R / 2), in stream-ordered workspace, chunk
// by chunk; a combine kernel sums them in increasing q.  Work is R/2 row
// evaluations of N elements per user instead of R.
#include <math.h>

#include "common.cuh"

namespace xl {

__global__ void ura_rows_kernel(const double2* __restrict__ users, int K, int Bc, int Q, int R, double spacing,
                                int model, double2* __restrict__ vusers, double* __restrict__ w) {
    int64_t total = (int64_t)Bc * Q * K;
    double off = (R & 1) ? 0.0 : 0.5;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int k = (int)(e % K);
        int64_t t = e / K;
        int q = (int)(t % Q);
        int64_t b = t / Q;
        double2 u = users[b * K + k];
        if (!user_ok(u.x, u.y)) {
            // an invalid user stays invalid on every row (x' > 0 would hide x <= 0)
            vusers[e] = make_double2(nan(""), nan(""));
            w[e] = nan("");
            continue;
        }
        double z = ((double)q + off) * spacing;
        double xp = model == XLMIMO_UPW ? u.x : sqrt(fma(u.x, u.x, z * z));
        vusers[e] = make_double2(xp, u.y);
        w[e] = model == XLMIMO_PNUSW ? sqrt(u.x / xp) : 1.0;
    }
}

__global__ void ura_combine_kernel(const double2* __restrict__ gv, const double* __restrict__ w, int K, int Bc,
                                   int Q, int R, int model, double2* __restrict__ gram) {
    int64_t kk = (int64_t)K * K;
    int64_t total = (int64_t)Bc * kk;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t b = e / kk;
        int ij = (int)(e - b * kk);
        int i = ij / K, j = ij - i * K;
        double re = 0.0, im = 0.0;
#pragma unroll 8
        for (int q = 0; q < Q; ++q) {
            int64_t t = b * Q + q;
            double m = model == XLMIMO_UPW ? (double)R : ((R & 1) && q == 0) ? 1.0 : 2.0;
            // w_i w_j before m: the same product for (i, j) and (j, i), so G stays exactly Hermitian
            double s = m * (w[t * K + i] * w[t * K + j]);
            double2 g = gv[t * kk + ij];
            re = fma(s, g.x, re);
            im = fma(s, g.y, im);
        }
        gram[e] = make_double2(re, im);
    }
}

static int launch_gram_prec(const Geom& g, const double* users, int K, int B, int prec, double* gram,
                            cudaStream_t st) {
    switch (prec) {
        case XLMIMO_F64: return launch_gram_f64(g, users, K, B, gram, st);
        case XLMIMO_F32: return launch_gram_f32(g, users, K, B, gram, st);
        default: return launch_gram_tc(g, users, K, B, prec, gram, st);
    }
}

static int grid_for(int64_t total) {
    int64_t blocks = (total + 255) / 256;
    if (blocks > 16LL * num_sms()) blocks = 16LL * num_sms();
    return (int)(blocks < 1 ? 1 : blocks);
}

int launch_gram_ura(const Geom& g, int64_t rows, const double* users, int K, int B, int prec, double* gram,
                    cudaStream_t st) {
    if (rows == 1) return launch_gram_prec(g, users, K, B, prec, gram, st);
    // measured at 10^4 trials, K = 32, 16384 elements: the URA mode takes 4.42 ms for
    // every shape, the row pairs as ULA trials 18.4 (128 columns), 5.1-5.5 (1024)
    // and 3.8 (4096): long rows amortise the per-trial cost of the ULA kernel
    if (g.N <= 1024 && gram_tc_ura_supported(g, g.N, prec))
        return launch_gram_tc_ura(g, g.N, rows, users, K, B, gram, st);
    int Q = g.model == XLMIMO_UPW ? 1 : (int)((rows + 1) / 2);
    // Workspace per trial: Q ULA Grams, Q virtual user sets and weights; up
    // to 1 GiB a chunk.  (Chunks small enough for the per-row Grams to stay in
    // L2 were slower: more launches with their ramp and tail, and combine
    // grids too small to keep the loads in flight.)  Chunks are rounded to
    // whole waves of Gram CTAs (three per SM for K <= 32, two above).
    size_t per_trial = (size_t)Q * K * ((size_t)K * sizeof(double2) + sizeof(double2) + sizeof(double));
    const size_t budget = size_t(1) << 30;
    int64_t bc = (int64_t)(budget / per_trial);
    const int64_t wave = (int64_t)num_sms() * (K <= 32 ? 3 : 2);
    int64_t a = wave, c = Q;  // trials per whole wave of virtual trials: wave / gcd(wave, Q)
    while (c) { int64_t t = a % c; a = c; c = t; }
    const int64_t step = wave / a;
    if (bc >= step) bc -= bc % step;
    if (bc < 1) bc = 1;
    if (bc > B) bc = B;
    if (bc * Q > INT32_MAX) bc = INT32_MAX / Q;
    double2* gv = nullptr;
    double2* vu = nullptr;
    double* w = nullptr;
    int rc = cuda_status(cudaMallocAsync((void**)&gv, (size_t)bc * Q * K * K * sizeof(double2), st),
                         "workspace allocation");
    if (!rc) rc = cuda_status(cudaMallocAsync((void**)&vu, (size_t)bc * Q * K * sizeof(double2), st),
                              "workspace allocation");
    if (!rc) rc = cuda_status(cudaMallocAsync((void**)&w, (size_t)bc * Q * K * sizeof(double), st),
                              "workspace allocation");
    for (int64_t b0 = 0; !rc && b0 < B; b0 += bc) {
        int n = (int)((B - b0 < bc) ? B - b0 : bc);
        ura_rows_kernel<<<grid_for((int64_t)n * Q * K), 256, 0, st>>>((const double2*)users + b0 * K, K, n, Q,
                                                                       (int)rows, g.spacing, g.model, vu, w);
        rc = cuda_status(cudaGetLastError(), "ura_rows launch");
        if (!rc) rc = launch_gram_prec(g, (const double*)vu, K, n * Q, prec, (double*)gv, st);
        if (!rc) {
            ura_combine_kernel<<<grid_for((int64_t)n * K * K), 256, 0, st>>>(
                gv, w, K, n, Q, (int)rows, g.model, (double2*)gram + b0 * K * K);
            rc = cuda_status(cudaGetLastError(), "ura_combine launch");
        }
    }
    if (w) cudaFreeAsync(w, st);
    if (vu) cudaFreeAsync(vu, st);
    if (gv) cudaFreeAsync(gv, st);
    return rc;
}

}  // namespace xl
