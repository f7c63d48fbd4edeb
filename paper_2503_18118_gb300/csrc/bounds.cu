// Appendix A: how much the off-diagonal Gram entries matter.  Per trial,
// with R the users' correlation matrix (r_ij = h_i^H h_j / (|h_i| |h_j|)) and
// the same receive SNR a for every user:
//   log2 det R,
//   C = log2 det(I + a R)            (the capacity),
//   log2 U = K log2(1 + a)            (Hadamard's upper bound),
//   log2 L = log2 det R + log2 U      (the Schur-Horn lower bound),
// and -(1/K) log2 det R is the negative empirical expectation of Fig. 5.
// K reaches 1000 there, beyond the K <= 64 receivers, so the path is:
//   1. channel entries into HBM (FP32, the span-referenced generator of
//      chan_gen.cuh), one CTA per (trial, user);
//   2. the lower 64 x 64 user tiles of G = H^H H: FP32 products summed over
//      32-element chunks, chunk sums in double-float, FP64 once per entry;
//   3. R and I + a R, FP64, padded to a multiple of 64 with identity rows;
//   4. a right-looking blocked Cholesky of all 2B matrices at once, 32
//      columns a step: diagonal block, panel solve, trailing update, each a
//      batched launch; the log-determinant adds 2 log2 L_kk block by block.
// Matrices are column-major (element (i, j) at j * Kp + i), lower triangle.
#include <math.h>

#include "chan_gen.cuh"
#include "common.cuh"

namespace xl {

constexpr int BT = 32;  // tile and Cholesky block size

// -------------------------------------------------------------- channels
// H[(b K + k) N + n] = h_k(n) of trial b (FP32 complex).  One CTA per (trial,
// user): the user's geometry once (FP64), then 256 span references at a time
// (one per thread) and the entries of those spans, written contiguously.
constexpr int CH_THREADS = 256;

__global__ void __launch_bounds__(CH_THREADS) bounds_channel_kernel(Geom g, GenParams gp, const double* __restrict__ users,
                                                                    int K, float2* __restrict__ H) {
    __shared__ UserGeo ug;
    __shared__ UserRef refs[CH_THREADS];
    const int64_t b = blockIdx.y;
    const int k = blockIdx.x, tid = threadIdx.x;
    if (tid == 0) ug = make_user_geo(g, users[(b * K + k) * 2], users[(b * K + k) * 2 + 1]);
    __syncthreads();
    const int64_t nspans = (g.N + REF_SPAN - 1) / REF_SPAN;
    float2* Hk = H + (b * K + k) * g.N;
    for (int64_t s0 = 0; s0 < nspans; s0 += CH_THREADS) {
        if (s0 + tid < nspans) refs[tid] = make_user_ref(gp, ug, (long long)((s0 + tid) * REF_SPAN + REF_SPAN / 2));
        __syncthreads();
        const int64_t nb0 = s0 * REF_SPAN;
        const int64_t cnt = min((int64_t)CH_THREADS * REF_SPAN, g.N - nb0);
        for (int64_t i = tid; i < cnt; i += CH_THREADS) {
            const int sp = (int)(i / REF_SPAN), m = (int)(i - (int64_t)sp * REF_SPAN) - REF_SPAN / 2;
            float2 h = gen_entry_f32(g.model, gp.dprime_f, ug.xl2, ug.x2x2, ug.ampc, refs[sp], (float)m);
            if (!ug.ok) h = make_float2(nanf(""), nanf(""));
            Hk[nb0 + i] = h;
        }
        __syncthreads();
    }
}

// -------------------------------------------------------------- Gram tiles
// (hi, lo) += v by Knuth's two-sum on the high part (double-float accumulator).
__device__ __forceinline__ void ff_acc(float& hi, float& lo, float v) {
    const float t = __fadd_rn(hi, v);
    const float bb = __fsub_rn(t, hi);
    lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bb)), __fsub_rn(v, bb)));
    hi = t;
}

// Tile (ti, tj), ti >= tj, of GT x GT users of trial b: G[j Kp + i] =
// sum_n conj(h_i(n)) h_j(n).  256 threads; thread (ri, cj) = (tid / 16,
// tid % 16) owns rows ri + 16 qa and columns cj + 16 qb (qa, qb < 4), so a
// warp's column reads fall in distinct bank pairs and each element loaded
// from shared memory feeds four complex MACs.  The products and the sum over
// a 32-element chunk are FP32 (worst relative error 32 x 2^-24 of the chunk's
// sum of magnitudes); chunk sums go into double-float accumulators, so the
// sum over N loses nothing further, and the FP64 pipe is used once per entry.
constexpr int GT = 64;

__global__ void __launch_bounds__(256) bounds_gram_kernel(const float2* __restrict__ H, int K, int64_t N, int Kp,
                                                          double2* __restrict__ G) {
    __shared__ float2 Hi[GT][BT + 1], Hj[GT][BT + 1];  // [user][element of the chunk]
    const int64_t b = blockIdx.y;
    int ti, tj;
    tri_index(blockIdx.x, &ti, &tj);
    const int tid = threadIdx.x, ri = tid >> 4, cj = tid & 15;
    const float2* Hb = H + b * K * N;
    float hx[4][4], lx[4][4], hy[4][4], ly[4][4];
#pragma unroll
    for (int qa = 0; qa < 4; ++qa)
#pragma unroll
        for (int qb = 0; qb < 4; ++qb) hx[qa][qb] = lx[qa][qb] = hy[qa][qb] = ly[qa][qb] = 0.f;
    for (int64_t n0 = 0; n0 < N; n0 += BT) {
#pragma unroll
        for (int l = 0; l < GT * BT / 256; ++l) {
            const int idx = tid + 256 * l, u = idx >> 5, e = idx & 31;  // user, element
            const int64_t n = n0 + e;
            const int ui = ti * GT + u, uj = tj * GT + u;
            Hi[u][e] = (ui < K && n < N) ? Hb[(int64_t)ui * N + n] : make_float2(0.f, 0.f);
            Hj[u][e] = (uj < K && n < N) ? Hb[(int64_t)uj * N + n] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        float sx[4][4], sy[4][4];
#pragma unroll
        for (int qa = 0; qa < 4; ++qa)
#pragma unroll
            for (int qb = 0; qb < 4; ++qb) sx[qa][qb] = sy[qa][qb] = 0.f;
#pragma unroll 4
        for (int e = 0; e < BT; ++e) {
            float2 a[4], v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = Hi[ri + 16 * q][e];
                v[q] = Hj[cj + 16 * q][e];
            }
#pragma unroll
            for (int qa = 0; qa < 4; ++qa)
#pragma unroll
                for (int qb = 0; qb < 4; ++qb) {  // += conj(a) v
                    sx[qa][qb] = fmaf(a[qa].x, v[qb].x, fmaf(a[qa].y, v[qb].y, sx[qa][qb]));
                    sy[qa][qb] = fmaf(a[qa].x, v[qb].y, fmaf(-a[qa].y, v[qb].x, sy[qa][qb]));
                }
        }
#pragma unroll
        for (int qa = 0; qa < 4; ++qa)
#pragma unroll
            for (int qb = 0; qb < 4; ++qb) {
                ff_acc(hx[qa][qb], lx[qa][qb], sx[qa][qb]);
                ff_acc(hy[qa][qb], ly[qa][qb], sy[qa][qb]);
            }
        __syncthreads();
    }
    double2* Gb = G + b * (int64_t)Kp * Kp;
#pragma unroll
    for (int qa = 0; qa < 4; ++qa)
#pragma unroll
        for (int qb = 0; qb < 4; ++qb)
            Gb[(int64_t)(tj * GT + cj + 16 * qb) * Kp + ti * GT + ri + 16 * qa] =
                make_double2((double)hx[qa][qb] + (double)lx[qa][qb], (double)hy[qa][qb] + (double)ly[qa][qb]);
}

// -------------------------------------------------------------- R, I + aR
// A[2b] = R, A[2b+1] = I + a R (lower triangles), padded with identity rows.
__global__ void bounds_normalize_kernel(const double2* __restrict__ G, int K, int Kp, double a, int B,
                                        double2* __restrict__ A) {
    const int64_t per = (int64_t)Kp * Kp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)B * per;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = e / per;
        const int64_t w = e - b * per;
        const int j = (int)(w / Kp), i = (int)(w - (int64_t)j * Kp);
        if (i < j) continue;
        double2 r = make_double2(i == j ? 1.0 : 0.0, 0.0), m = r;
        if (i < K && j < K) {
            const double2* Gb = G + b * per;
            if (i == j) {
                m = make_double2(1.0 + a, 0.0);
            } else {
                const double2 v = Gb[w];
                const double s = 1.0 / sqrt(Gb[(int64_t)i * Kp + i].x * Gb[(int64_t)j * Kp + j].x);
                r = make_double2(v.x * s, v.y * s);
                m = make_double2(a * r.x, a * r.y);
            }
        }
        A[2 * b * per + w] = r;
        A[(2 * b + 1) * per + w] = m;
    }
}

// -------------------------------------------------------------- blocked Cholesky
// Diagonal block p of matrix m: factor in shared memory, write L_pp back and
// add sum_k log2 L_kk^2 to logdet[m] (NaN when a pivot is not positive).
__global__ void __launch_bounds__(256) bounds_chol_diag_kernel(double2* __restrict__ A, int Kp, int p,
                                                               double* __restrict__ logdet) {
    __shared__ double2 T[BT][BT + 1];
    __shared__ double piv[BT];
    __shared__ int bad;
    double2* Am = A + (int64_t)blockIdx.x * Kp * Kp;
    const int tid = threadIdx.x, o = p * BT;
    if (tid == 0) bad = 0;
    for (int e = tid; e < BT * BT; e += 256) {
        const int c = e >> 5, r = e & 31;
        if (r >= c) T[r][c] = Am[(int64_t)(o + c) * Kp + o + r];
    }
    __syncthreads();
    for (int k = 0; k < BT; ++k) {
        if (tid == 0) {
            const double d = T[k][k].x;
            piv[k] = d;
            if (!(d > 0.0) || !isfinite(d)) bad = 1;
            T[k][k] = make_double2(sqrt(d), 0.0);
        }
        __syncthreads();
        const double inv = 1.0 / T[k][k].x;
        for (int r = k + 1 + tid; r < BT; r += 256) T[r][k] = make_double2(T[r][k].x * inv, T[r][k].y * inv);
        __syncthreads();
        const int m = BT - k - 1, tri = m * (m + 1) / 2;
        for (int q = tid; q < tri; q += 256) {
            int rr, cc;
            tri_index(q, &rr, &cc);
            const int r = k + 1 + rr, c = k + 1 + cc;
            const double2 x = T[r][k], y = T[c][k];  // T[r][c] -= x conj(y)
            T[r][c].x -= fma(x.x, y.x, x.y * y.y);
            T[r][c].y -= fma(x.y, y.x, -x.x * y.y);
        }
        __syncthreads();
    }
    for (int e = tid; e < BT * BT; e += 256) {
        const int c = e >> 5, r = e & 31;
        if (r >= c) Am[(int64_t)(o + c) * Kp + o + r] = T[r][c];
    }
    if (tid == 0) {
        double s = 0.0;
        for (int k = 0; k < BT; ++k) s += log2(piv[k]);  // log2 L_kk^2, in column order
        logdet[blockIdx.x] = bad ? nan("") : logdet[blockIdx.x] + s;
    }
}

// Panel below block p: L_ip = A_ip L_pp^-H for block row i = p + 1 + blockIdx.x;
// thread r solves row r of the block by forward substitution.
__global__ void __launch_bounds__(BT) bounds_chol_panel_kernel(double2* __restrict__ A, int Kp, int p) {
    __shared__ double2 L[BT][BT + 1], X[BT][BT + 1];
    double2* Am = A + (int64_t)blockIdx.y * Kp * Kp;
    const int r = threadIdx.x, o = p * BT, io = (p + 1 + blockIdx.x) * BT;
    for (int c = 0; c < BT; ++c) {
        L[r][c] = Am[(int64_t)(o + c) * Kp + o + r];   // rows r >= c used
        X[r][c] = Am[(int64_t)(o + c) * Kp + io + r];
    }
    __syncthreads();
    for (int c = 0; c < BT; ++c) {
        double2 s = X[r][c];
        for (int l = 0; l < c; ++l) {  // s -= X_rl conj(L_cl)
            const double2 x = X[r][l], y = L[c][l];
            s.x -= fma(x.x, y.x, x.y * y.y);
            s.y -= fma(x.y, y.x, -x.x * y.y);
        }
        const double inv = 1.0 / L[c][c].x;
        X[r][c] = make_double2(s.x * inv, s.y * inv);
    }
    for (int c = 0; c < BT; ++c) Am[(int64_t)(o + c) * Kp + io + r] = X[r][c];
}

// Trailing update after block p: A_ij -= L_ip L_jp^H for p < j <= i, tile
// blockIdx.x of that lower triangle; row r = tid / 8, columns 4 (tid % 8)..+3.
__global__ void __launch_bounds__(256) bounds_chol_update_kernel(double2* __restrict__ A, int Kp, int p) {
    __shared__ double2 Li[BT][BT + 1], Lj[BT][BT + 1];
    double2* Am = A + (int64_t)blockIdx.y * Kp * Kp;
    int ti, tj;
    tri_index(blockIdx.x, &ti, &tj);
    const int o = p * BT, io = (p + 1 + ti) * BT, jo = (p + 1 + tj) * BT;
    const int tid = threadIdx.x;
    for (int e = tid; e < BT * BT; e += 256) {
        const int c = e >> 5, r = e & 31;
        Li[r][c] = Am[(int64_t)(o + c) * Kp + io + r];
        Lj[r][c] = Am[(int64_t)(o + c) * Kp + jo + r];
    }
    __syncthreads();
    const int r = tid >> 3, c0 = (tid & 7) * 4;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int c = c0 + q;
        double2 s = make_double2(0.0, 0.0);
#pragma unroll 8
        for (int l = 0; l < BT; ++l) {  // s += Li_rl conj(Lj_cl)
            const double2 x = Li[r][l], y = Lj[c][l];
            s.x = fma(x.x, y.x, fma(x.y, y.y, s.x));
            s.y = fma(x.y, y.x, fma(-x.x, y.y, s.y));
        }
        double2* t = Am + (int64_t)(jo + c) * Kp + io + r;
        const double2 v = *t;
        *t = make_double2(v.x - s.x, v.y - s.y);
    }
}

__global__ void bounds_finish_kernel(const double* __restrict__ logdet, int K, int B, double a,
                                     double* __restrict__ out) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
        const double lu = (double)K * log2(1.0 + a);
        out[4 * b + 0] = logdet[2 * b];
        out[4 * b + 1] = logdet[2 * b + 1];
        out[4 * b + 2] = lu;
        out[4 * b + 3] = logdet[2 * b] + lu;
    }
}

}  // namespace xl

using namespace xl;

extern "C" int xlmimo_capacity_bounds(const xlmimo_array* arr, const double* users, int K, int B, double snr,
                                      double* out, void* stream) {
    clear_error();
    Geom g;
    int rc = check_array(arr, &g);
    if (rc) return rc;
    if (K < 1 || K > XLMIMO_MAX_BOUNDS_USERS || B < 0) {
        set_error("K must be in [1, %d] and B >= 0", XLMIMO_MAX_BOUNDS_USERS);
        return XLMIMO_EINVAL;
    }
    if (!(snr >= 0.0) || !isfinite(snr)) {
        set_error("snr must be a finite number >= 0");
        return XLMIMO_EINVAL;
    }
    if (B == 0) return XLMIMO_OK;
    if (!users || !out) {
        set_error("users and out must be non-NULL");
        return XLMIMO_EINVAL;
    }
    cudaStream_t st = as_stream(stream);
    const int Kp = (K + GT - 1) / GT * GT;  // multiple of the Gram tile and of the Cholesky block
    const int nb = Kp / BT, ng = Kp / GT;
    const int64_t N = g.N, per = (int64_t)Kp * Kp;
    float2* H = nullptr;
    double2 *G = nullptr, *A = nullptr;
    double* ld = nullptr;
    rc = cuda_status(cudaMallocAsync((void**)&H, (size_t)B * K * N * sizeof(float2), st), "workspace allocation");
    if (!rc) rc = cuda_status(cudaMallocAsync((void**)&G, (size_t)B * per * sizeof(double2), st), "workspace allocation");
    if (!rc) rc = cuda_status(cudaMallocAsync((void**)&A, (size_t)2 * B * per * sizeof(double2), st), "workspace allocation");
    if (!rc) rc = cuda_status(cudaMallocAsync((void**)&ld, (size_t)2 * B * sizeof(double), st), "workspace allocation");
    if (!rc) {
        bounds_channel_kernel<<<dim3((unsigned)K, (unsigned)B), CH_THREADS, 0, st>>>(g, make_gen_params(g), users, K, H);
        rc = cuda_status(cudaGetLastError(), "bounds channel launch");
    }
    if (!rc) {
        bounds_gram_kernel<<<dim3((unsigned)(ng * (ng + 1) / 2), (unsigned)B), 256, 0, st>>>(H, K, N, Kp, G);
        rc = cuda_status(cudaGetLastError(), "bounds gram launch");
    }
    if (!rc) {
        int64_t blocks = ((int64_t)B * per + 255) / 256;
        if (blocks > 16LL * num_sms()) blocks = 16LL * num_sms();
        bounds_normalize_kernel<<<(unsigned)blocks, 256, 0, st>>>(G, K, Kp, snr, B, A);
        rc = cuda_status(cudaGetLastError(), "bounds normalize launch");
    }
    if (!rc) rc = cuda_status(cudaMemsetAsync(ld, 0, (size_t)2 * B * sizeof(double), st), "workspace clear");
    for (int p = 0; p < nb && !rc; ++p) {
        bounds_chol_diag_kernel<<<2 * B, 256, 0, st>>>(A, Kp, p, ld);
        rc = cuda_status(cudaGetLastError(), "bounds cholesky launch");
        const int m = nb - p - 1;
        if (!rc && m > 0) {
            bounds_chol_panel_kernel<<<dim3((unsigned)m, (unsigned)(2 * B)), BT, 0, st>>>(A, Kp, p);
            bounds_chol_update_kernel<<<dim3((unsigned)(m * (m + 1) / 2), (unsigned)(2 * B)), 256, 0, st>>>(A, Kp, p);
            rc = cuda_status(cudaGetLastError(), "bounds cholesky launch");
        }
    }
    if (!rc) {
        bounds_finish_kernel<<<(B + 255) / 256, 256, 0, st>>>(ld, K, B, snr, out);
        rc = cuda_status(cudaGetLastError(), "bounds finish launch");
    }
    if (ld) cudaFreeAsync(ld, st);
    if (A) cudaFreeAsync(A, st);
    if (G) cudaFreeAsync(G, st);
    if (H) cudaFreeAsync(H, st);
    return rc;
}
