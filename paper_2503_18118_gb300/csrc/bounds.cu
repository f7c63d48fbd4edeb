// Appendix A: how much the off-diagonal Gram entries matter.  Per trial,
// with R the users' correlation matrix (r_ij = h_i^H h_j / (|h_i| |h_j|)) and
// the same receive SNR a for every user:
//   log2 det R,
//   C = log2 det(I + a R)            (the capacity),
//   log2 U = K log2(1 + a)            (Hadamard's upper bound),
//   log2 L = log2 det R + log2 U      (the Schur-Horn lower bound),
// and -(1/K) log2 det R is the negative empirical expectation of Fig. 5.
// K reaches 1000 there, beyond the K <= 64 receivers, so the path is:
//   1. channel entries into HBM as a BF16 split of X = [Re H ; Im H] (the
//      span-referenced FP32 generator of chan_gen.cuh), one CTA per (trial,
//      user), users padded to Kp (a multiple of 64) and elements to Np (a
//      multiple of 64) with zeros;
//   2. the real Gram X X^T on the tensor cores, 128 x 128 tiles of the lower
//      triangle, hi*hi + lo*hi + hi*lo with FP32 totals (gram_hilo_tc.cuh);
//   3. the complex Gram from the real one, then R and I + a R, FP64, padded to
//      a multiple of 64 with identity rows;
//   4. a right-looking blocked Cholesky of all 2B matrices at once, 32
//      columns a step: diagonal block in FP64, panel solve and trailing
//      update in double-float on the FP32 pipe (~2^-48; the panel hands its
//      result to the update as float pairs), each a batched launch; the
//      log-determinant adds 2 log2 L_kk block by block.
// Matrices are column-major (element (i, j) at j * Kp + i), lower triangle.
#include <math.h>

#include <cudaTypedefs.h>

#include "chan_gen.cuh"
#include "common.cuh"
#include "gram_hilo_tc.cuh"

namespace xl {

constexpr int BT = 32;  // tile and Cholesky block size

// -------------------------------------------------------------- channels
// X_hi, X_lo of trial b: row k = Re h_k, row Kp + k = Im h_k (elements
// contiguous, Np per row), h = hi + lo with hi = RN_bf16(h) and lo =
// RN_bf16(h - hi).  One CTA per (trial, user k < Kp): the user's geometry
// once (FP64), then 256 span references at a time (one per thread) and the
// entries of those spans.  Padding users and elements are zero.
constexpr int CH_THREADS = 256;

__global__ void __launch_bounds__(CH_THREADS) bounds_channel_kernel(Geom g, GenParams gp, const double* __restrict__ users,
                                                                    int K, int Kp, int64_t Np,
                                                                    __nv_bfloat16* __restrict__ Xhi,
                                                                    __nv_bfloat16* __restrict__ Xlo) {
    __shared__ UserGeo ug;
    __shared__ UserRef refs[CH_THREADS];
    const int64_t b = blockIdx.y;
    const int k = blockIdx.x, tid = threadIdx.x;
    const int64_t ro = (b * 2 * Kp + k) * Np, io = (b * 2 * Kp + Kp + k) * Np;  // rows of Re and Im
    const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
    if (k >= K) {
        for (int64_t n = tid; n < Np; n += CH_THREADS) {
            Xhi[ro + n] = z;
            Xlo[ro + n] = z;
            Xhi[io + n] = z;
            Xlo[io + n] = z;
        }
        return;
    }
    if (tid == 0) ug = make_user_geo(g, users[(b * K + k) * 2], users[(b * K + k) * 2 + 1]);
    __syncthreads();
    const int64_t nspans = (g.N + REF_SPAN - 1) / REF_SPAN;
    for (int64_t s0 = 0; s0 < nspans; s0 += CH_THREADS) {
        if (s0 + tid < nspans) refs[tid] = make_user_ref(gp, ug, (long long)((s0 + tid) * REF_SPAN + REF_SPAN / 2));
        __syncthreads();
        const int64_t nb0 = s0 * REF_SPAN;
        const int64_t cnt = min((int64_t)CH_THREADS * REF_SPAN, g.N - nb0);
        for (int64_t i = tid; i < cnt; i += CH_THREADS) {
            const int sp = (int)(i / REF_SPAN), m = (int)(i - (int64_t)sp * REF_SPAN) - REF_SPAN / 2;
            float2 h = gen_entry_f32(g.model, gp.dprime_f, ug.xl2, ug.x2x2, ug.ampc, refs[sp], (float)m);
            if (!ug.ok) h = make_float2(nanf(""), nanf(""));
            const __nv_bfloat16 rh = __float2bfloat16_rn(h.x), ih = __float2bfloat16_rn(h.y);
            Xhi[ro + nb0 + i] = rh;
            Xlo[ro + nb0 + i] = __float2bfloat16_rn(h.x - __bfloat162float(rh));
            Xhi[io + nb0 + i] = ih;
            Xlo[io + nb0 + i] = __float2bfloat16_rn(h.y - __bfloat162float(ih));
        }
        __syncthreads();
    }
    for (int64_t n = g.N + tid; n < Np; n += CH_THREADS) {
        Xhi[ro + n] = z;
        Xlo[ro + n] = z;
        Xhi[io + n] = z;
        Xlo[io + n] = z;
    }
}

// -------------------------------------------------------------- R, I + aR
// The complex Gram G_ij = h_i^H h_j from the real X X^T (Rr, 2Kp x 2Kp FP32,
// row-major, tiles on or below the diagonal written):
//   Re G_ij = Rr(i, j) + Rr(Kp + i, Kp + j),  Im G_ij = Rr(i, Kp + j) - Rr(Kp + i, j).
__device__ __forceinline__ double rr_at(const float* Rr, int K2, int r, int c) {
    return (r / GH_TILE >= c / GH_TILE) ? (double)Rr[(int64_t)r * K2 + c] : (double)Rr[(int64_t)c * K2 + r];
}

// A[2b] = R, A[2b+1] = I + a R (lower triangles), padded with identity rows.
__global__ void bounds_normalize_kernel(const float* __restrict__ Rr, int K, int Kp, double a, int B,
                                        double2* __restrict__ A) {
    const int64_t per = (int64_t)Kp * Kp;
    const int K2 = 2 * Kp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)B * per;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = e / per;
        const int64_t w = e - b * per;
        const int j = (int)(w / Kp), i = (int)(w - (int64_t)j * Kp);
        if (i < j) continue;
        double2 r = make_double2(i == j ? 1.0 : 0.0, 0.0), m = r;
        if (i < K && j < K) {
            const float* Rb = Rr + b * (int64_t)K2 * K2;
            if (i == j) {
                m = make_double2(1.0 + a, 0.0);
            } else {
                const double gre = rr_at(Rb, K2, i, j) + rr_at(Rb, K2, Kp + i, Kp + j);
                const double gim = rr_at(Rb, K2, i, Kp + j) - rr_at(Rb, K2, Kp + i, j);
                const double gii = rr_at(Rb, K2, i, i) + rr_at(Rb, K2, Kp + i, Kp + i);
                const double gjj = rr_at(Rb, K2, j, j) + rr_at(Rb, K2, Kp + j, Kp + j);
                const double s = 1.0 / sqrt(gii * gjj);
                r = make_double2(gre * s, gim * s);
                m = make_double2(a * r.x, a * r.y);
            }
        }
        A[2 * b * per + w] = r;
        A[(2 * b + 1) * per + w] = m;
    }
}

// cuTensorMapEncodeTiled from the driver, looked up once.
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// Tensor map of B trials of 2Kp rows x Np BF16 elements, boxes of 128 rows x
// 64 elements (128 bytes: the swizzle atom), 128-byte swizzle.
static int x_tensor_map(CUtensorMap* map, void* base, int64_t Np, int Kp, int B) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return XLMIMO_ECUDA;
    }
    const cuuint64_t dims[3] = {(cuuint64_t)Np, (cuuint64_t)(2 * Kp), (cuuint64_t)B};
    const cuuint64_t strides[2] = {(cuuint64_t)Np * 2, (cuuint64_t)(2 * Kp) * (cuuint64_t)Np * 2};
    const cuuint32_t box[3] = {(cuuint32_t)GH_BK, (cuuint32_t)GH_TILE, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return XLMIMO_ECUDA;
    }
    return XLMIMO_OK;
}

// -------------------------------------------------------------- blocked Cholesky
// Diagonal block p of matrix m: factor in shared memory, write L_pp back and
// add sum_k log2 L_kk^2 to logdet[m] (NaN when a pivot is not positive).
__global__ void __launch_bounds__(256) bounds_chol_diag_kernel(double2* __restrict__ A, int Kp, int p,
                                                               double* __restrict__ logdet) {
    __shared__ double2 T[BT][BT + 1];
    __shared__ double piv[BT];
    __shared__ double yk;  // 1 / L_kk of the current column
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
            // one FP64 reciprocal square root per column (a few FP64
            // instructions), shared: each FP64 instruction costs a warp's issue
            const double d = T[k][k].x;
            piv[k] = d;
            double y = 0.0;
            if (!rsqrt_pivot(d, y)) {
                bad = 1;
                y = 0.0;
            }
            yk = y;
            T[k][k] = make_double2(d * y, 0.0);
        }
        __syncthreads();
        const double inv = yk;
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
    if (tid < 32) {
        // log2 L_kk^2, one column per lane, summed in a fixed shuffle order
        double s = bad ? 0.0 : log2(piv[tid]);
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (tid == 0) logdet[blockIdx.x] = bad ? nan("") : logdet[blockIdx.x] + s;
    }
}

// Panel below block p: L_ip = A_ip L_pp^-H for block row i = p + 1 + blockIdx.x,
// by forward substitution in double-float on the FP32 pipe (FMA-exact
// products, two-sums; the 32 pivot reciprocals are formed once in FP64).
// 256 threads: the two blocks are loaded and stored coalesced, and row r of
// the block is solved by the 8 threads 8 r .. 8 r + 7 of one warp, thread j
// summing the terms l = j, j + 8, ... of each column's sum and the 8 partial
// sums added by a fixed shuffle tree.  The result is written in place as float
// pairs (re hi, im hi, re lo, im lo: the same 16 bytes as the FP64 entry): the
// trailing update of this step is its only reader.
constexpr int PANEL_THREADS = 256;
constexpr int PANEL_SPLIT = PANEL_THREADS / BT;  // threads per row

__global__ void __launch_bounds__(PANEL_THREADS) bounds_chol_panel_kernel(double2* __restrict__ A, int Kp, int p) {
    __shared__ float4 L[BT][BT + 1], X[BT][BT + 1];
    __shared__ float2 rinv[BT];
    double2* Am = A + (int64_t)blockIdx.y * Kp * Kp;
    const int tid = threadIdx.x, o = p * BT, io = (p + 1 + blockIdx.x) * BT;
    auto split2 = [](double2 v) {
        float rh, rl, ih, il;
        split_f64(v.x, rh, rl);
        split_f64(v.y, ih, il);
        return make_float4(rh, ih, rl, il);
    };
    for (int e = tid; e < BT * BT; e += PANEL_THREADS) {
        const int c = e >> 5, r = e & 31;
        L[r][c] = split2(Am[(int64_t)(o + c) * Kp + o + r]);  // rows r >= c used
        X[r][c] = split2(Am[(int64_t)(o + c) * Kp + io + r]);
    }
    if (tid < BT) {
        float h, l;
        split_f64(1.0 / Am[(int64_t)(o + tid) * Kp + o + tid].x, h, l);
        rinv[tid] = make_float2(h, l);
    }
    __syncthreads();
    const int r = tid / PANEL_SPLIT, j = tid % PANEL_SPLIT;
    for (int c = 0; c < BT; ++c) {
        float2 sh = make_float2(0.f, 0.f), sl = sh;
        if (j == 0) {
            const float4 x0 = X[r][c];
            sh = make_float2(x0.x, x0.y);
            sl = make_float2(x0.z, x0.w);
        }
        for (int l = j; l < c; l += PANEL_SPLIT) {  // s -= X_rl conj(L_cl)
            const float4 x = X[r][l], y = L[c][l];
            ff2_mac(sh, sl, make_float2(-x.x, -x.y), make_float2(-x.z, -x.w), make_float2(y.x, y.x),
                    make_float2(y.z, y.z));
            ff2_mac(sh, sl, make_float2(-x.y, x.x), make_float2(-x.w, x.z), make_float2(y.y, y.y),
                    make_float2(y.w, y.w));
        }
        for (int off = PANEL_SPLIT / 2; off > 0; off >>= 1) {
            const float2 oh = make_float2(__shfl_xor_sync(0xffffffffu, sh.x, off), __shfl_xor_sync(0xffffffffu, sh.y, off));
            const float2 ol = make_float2(__shfl_xor_sync(0xffffffffu, sl.x, off), __shfl_xor_sync(0xffffffffu, sl.y, off));
            ff2_add(sh, sl, oh, ol);
        }
        if (j == 0) {
            const float2 t = __fadd2_rn(sh, sl);
            const float2 tl = __fadd2_rn(__fadd2_rn(sh, make_float2(-t.x, -t.y)), sl);
            const float2 ri = rinv[c];
            float2 qh = make_float2(0.f, 0.f), ql = qh;
            ff2_mac(qh, ql, t, tl, make_float2(ri.x, ri.x), make_float2(ri.y, ri.y));
            const float2 u = __fadd2_rn(qh, ql);
            X[r][c] = make_float4(u.x, u.y, __fadd_rn(__fadd_rn(qh.x, -u.x), ql.x), __fadd_rn(__fadd_rn(qh.y, -u.y), ql.y));
        }
        __syncwarp();  // the row's 8 threads read X[r][c] from the next column on
    }
    __syncthreads();
    for (int e = tid; e < BT * BT; e += PANEL_THREADS) {
        const int c = e >> 5, rr = e & 31;
        reinterpret_cast<float4*>(Am)[(int64_t)(o + c) * Kp + io + rr] = X[rr][c];
    }
}

// Trailing update after block p: A_ij -= L_ip L_jp^H for p < j <= i, tile
// blockIdx.x of that lower triangle, in double-float on the FP32 pipe (the
// FP64 pipe issues one warp instruction per ~64 cycles per scheduler): the
// two 32 x 32 blocks come as float pairs from the panel kernel, each
// entry's 32 products are accumulated with FMA-exact products and two-sums
// (~2^-48 of the terms' magnitudes), and the sum is subtracted from the FP64
// entry in FP64.  Thread: row r = tid / 8, columns c = tid % 8 + 8 q
// (q = 0..3, interleaved so that a warp's 16-byte loads of Lj fill all banks).
// part: 0 every tile of the trailing triangle; 1 the first block column of
// it only (tile blockIdx.x, 0: the look-ahead's next panel); 2 the others.
__global__ void __launch_bounds__(256) bounds_chol_update_kernel(double2* __restrict__ A, int Kp, int p, int part) {
    __shared__ float4 Li[BT][BT + 1], Lj[BT][BT + 1];  // (re hi, im hi, re lo, im lo)
    double2* Am = A + (int64_t)blockIdx.y * Kp * Kp;
    int ti, tj;
    if (part == 1) {
        ti = blockIdx.x;
        tj = 0;
    } else {
        tri_index(blockIdx.x, &ti, &tj);
        if (part == 2) {
            ++ti;
            ++tj;
        }
    }
    const int o = p * BT, io = (p + 1 + ti) * BT, jo = (p + 1 + tj) * BT;
    const int tid = threadIdx.x;
    const float4* Lf = reinterpret_cast<const float4*>(Am);
    for (int e = tid; e < BT * BT; e += 256) {
        const int c = e >> 5, r = e & 31;
        Li[r][c] = Lf[(int64_t)(o + c) * Kp + io + r];
        Lj[r][c] = Lf[(int64_t)(o + c) * Kp + jo + r];
    }
    __syncthreads();
    const int r = tid >> 3, c0 = tid & 7;
    float2 sh[4], sl[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) sh[q] = sl[q] = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int l = 0; l < BT; ++l) {
        const float4 x = Li[r][l];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            // s += x conj(y): lanes (re x re y, im x re y), then (im x im y, -re x im y)
            const float4 y = Lj[c0 + 8 * q][l];
            ff2_mac(sh[q], sl[q], make_float2(x.x, x.y), make_float2(x.z, x.w), make_float2(y.x, y.x),
                    make_float2(y.z, y.z));
            ff2_mac(sh[q], sl[q], make_float2(x.y, -x.x), make_float2(x.w, -x.z), make_float2(y.y, y.y),
                    make_float2(y.w, y.w));
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int c = c0 + 8 * q;
        double2* t = Am + (int64_t)(jo + c) * Kp + io + r;
        const double2 v = *t;
        *t = make_double2(v.x - ((double)sh[q].x + (double)sl[q].x), v.y - ((double)sh[q].y + (double)sl[q].y));
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

// The whole path; ev (NULL, or 6 events) is recorded on the stream before the
// channels and after each of the five phases.
static int capacity_bounds_impl(const xlmimo_array* arr, const double* users, int K, int B, double snr, double* out,
                                void* stream, cudaEvent_t* ev) {
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
    const int Kp = (K + 63) / 64 * 64;  // 2 Kp rows: whole 128-row Gram tiles; a multiple of the Cholesky block
    const int nb = Kp / BT, nt = 2 * Kp / GH_TILE;
    const int64_t N = g.N, Np = (N + GH_BK - 1) / GH_BK * GH_BK, per = (int64_t)Kp * Kp;
    const int64_t K2 = 2 * Kp;
    __nv_bfloat16 *Xhi = nullptr, *Xlo = nullptr;
    float* Rr = nullptr;
    double2* A = nullptr;
    double* ld = nullptr;
    rc = cuda_status(cudaMallocAsync((void**)&Xhi, (size_t)B * K2 * Np * 2, st), "workspace allocation");
    if (!rc) rc = cuda_status(cudaMallocAsync((void**)&Xlo, (size_t)B * K2 * Np * 2, st), "workspace allocation");
    if (!rc) rc = cuda_status(cudaMallocAsync((void**)&Rr, (size_t)B * K2 * K2 * sizeof(float), st), "workspace allocation");
    if (!rc) rc = cuda_status(cudaMallocAsync((void**)&A, (size_t)2 * B * per * sizeof(double2), st), "workspace allocation");
    if (!rc) rc = cuda_status(cudaMallocAsync((void**)&ld, (size_t)2 * B * sizeof(double), st), "workspace allocation");
    CUtensorMap mhi, mlo;
    if (!rc) rc = x_tensor_map(&mhi, Xhi, Np, Kp, B);
    if (!rc) rc = x_tensor_map(&mlo, Xlo, Np, Kp, B);
    if (!rc)
        rc = cuda_status(cudaFuncSetAttribute(gram_hilo_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)gh_smem_bytes()),
                         "bounds gram attribute");
    if (!rc && ev) rc = cuda_status(cudaEventRecord(ev[0], st), "event record");
    if (!rc) {
        bounds_channel_kernel<<<dim3((unsigned)Kp, (unsigned)B), CH_THREADS, 0, st>>>(g, make_gen_params(g), users, K, Kp,
                                                                                     Np, Xhi, Xlo);
        rc = cuda_status(cudaGetLastError(), "bounds channel launch");
    }
    if (!rc && ev) rc = cuda_status(cudaEventRecord(ev[1], st), "event record");
    if (!rc) {
        gram_hilo_kernel<<<dim3((unsigned)(nt * (nt + 1) / 2), (unsigned)B), GH_THREADS, gh_smem_bytes(), st>>>(
            mhi, mlo, (int)Np, Kp, Rr);
        rc = cuda_status(cudaGetLastError(), "bounds gram launch");
    }
    if (!rc && ev) rc = cuda_status(cudaEventRecord(ev[2], st), "event record");
    if (!rc) {
        int64_t blocks = ((int64_t)B * per + 255) / 256;
        if (blocks > 16LL * num_sms()) blocks = 16LL * num_sms();
        bounds_normalize_kernel<<<(unsigned)blocks, 256, 0, st>>>(Rr, K, Kp, snr, B, A);
        rc = cuda_status(cudaGetLastError(), "bounds normalize launch");
    }
    if (!rc && ev) rc = cuda_status(cudaEventRecord(ev[3], st), "event record");
    if (!rc) rc = cuda_status(cudaMemsetAsync(ld, 0, (size_t)2 * B * sizeof(double), st), "workspace clear");
    // Blocked Cholesky with a look-ahead of one block column: after step p's
    // panel, a library stream of the highest priority updates block column
    // p + 1 alone, factors its diagonal block and solves its panel (a few CTAs
    // per matrix, scheduled ahead of the bulk as SMs free up) while `st`
    // applies step p's update to the rest of the trailing triangle.  Events:
    // the rest of step p waits for panel p (the L it reads); the column update
    // of step p + 1 waits for the rest of step p (which updated that column).
    cudaStream_t sa = nullptr;  // the critical chain; st without a look-ahead
    cudaEvent_t evs[2 * (XLMIMO_MAX_BOUNDS_USERS / BT + 2)] = {};
    int nev = 0;
    auto event = [&](cudaStream_t from, cudaStream_t to) {
        cudaEvent_t e = nullptr;
        int r = cuda_status(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cholesky event");
        if (!r) evs[nev++] = e;
        if (!r) r = cuda_status(cudaEventRecord(e, from), "cholesky event");
        if (!r) r = cuda_status(cudaStreamWaitEvent(to, e, 0), "cholesky event");
        return r;
    };
    if (!rc && nb > 2) {
        int least = 0, greatest = 0;
        rc = cuda_status(cudaDeviceGetStreamPriorityRange(&least, &greatest), "stream priorities");
        if (!rc) rc = cuda_status(cudaStreamCreateWithPriority(&sa, cudaStreamNonBlocking, greatest), "cholesky stream");
        if (!rc) rc = event(st, sa);
    }
    cudaStream_t sc = sa ? sa : st;
    if (!rc) {
        bounds_chol_diag_kernel<<<2 * B, 256, 0, sc>>>(A, Kp, 0, ld);
        if (nb > 1) bounds_chol_panel_kernel<<<dim3((unsigned)(nb - 1), (unsigned)(2 * B)), PANEL_THREADS, 0, sc>>>(A, Kp, 0);
        rc = cuda_status(cudaGetLastError(), "bounds cholesky launch");
    }
    for (int p = 0; p + 1 < nb && !rc; ++p) {
        const int m = nb - p - 1;  // block columns after p
        if (sa && m > 1) {
            rc = event(sa, st);  // panel p is in place
            if (!rc) {
                bounds_chol_update_kernel<<<dim3((unsigned)(m * (m - 1) / 2), (unsigned)(2 * B)), 256, 0, st>>>(A, Kp, p, 2);
                bounds_chol_update_kernel<<<dim3((unsigned)m, (unsigned)(2 * B)), 256, 0, sa>>>(A, Kp, p, 1);
                rc = cuda_status(cudaGetLastError(), "bounds cholesky launch");
            }
        } else if (!rc) {
            bounds_chol_update_kernel<<<dim3((unsigned)(m * (m + 1) / 2), (unsigned)(2 * B)), 256, 0, sc>>>(A, Kp, p, 0);
            rc = cuda_status(cudaGetLastError(), "bounds cholesky launch");
        }
        if (!rc) {
            bounds_chol_diag_kernel<<<2 * B, 256, 0, sc>>>(A, Kp, p + 1, ld);
            if (m > 1) bounds_chol_panel_kernel<<<dim3((unsigned)(m - 1), (unsigned)(2 * B)), PANEL_THREADS, 0, sc>>>(A, Kp, p + 1);
            rc = cuda_status(cudaGetLastError(), "bounds cholesky launch");
        }
        // the next column update needs the rest of this step (the column it updates)
        if (!rc && sa && m > 1) rc = event(st, sa);
    }
    if (sa) {
        // joined even after an error, so that nothing on it outlives the call
        const int r = event(sa, st);
        if (!rc) rc = r;
        cudaStreamDestroy(sa);
    }
    for (int i = 0; i < nev; ++i) cudaEventDestroy(evs[i]);
    if (!rc && ev) rc = cuda_status(cudaEventRecord(ev[4], st), "event record");
    if (!rc) {
        bounds_finish_kernel<<<(B + 255) / 256, 256, 0, st>>>(ld, K, B, snr, out);
        rc = cuda_status(cudaGetLastError(), "bounds finish launch");
    }
    if (!rc && ev) rc = cuda_status(cudaEventRecord(ev[5], st), "event record");
    if (ld) cudaFreeAsync(ld, st);
    if (A) cudaFreeAsync(A, st);
    if (Rr) cudaFreeAsync(Rr, st);
    if (Xlo) cudaFreeAsync(Xlo, st);
    if (Xhi) cudaFreeAsync(Xhi, st);
    return rc;
}

extern "C" int xlmimo_capacity_bounds(const xlmimo_array* arr, const double* users, int K, int B, double snr,
                                      double* out, void* stream) {
    clear_error();
    return capacity_bounds_impl(arr, users, K, B, snr, out, stream, nullptr);
}

extern "C" int xlmimo_capacity_bounds_timed(const xlmimo_array* arr, const double* users, int K, int B, double snr,
                                            double* out, float* phase_ms, void* stream) {
    clear_error();
    if (!phase_ms) {
        set_error("phase_ms must be non-NULL");
        return XLMIMO_EINVAL;
    }
    cudaEvent_t ev[6] = {};
    int rc = XLMIMO_OK;
    for (int i = 0; i < 6 && !rc; ++i) rc = cuda_status(cudaEventCreate(&ev[i]), "event create");
    if (!rc) rc = capacity_bounds_impl(arr, users, K, B, snr, out, stream, ev);
    if (!rc && B == 0) {
        for (int i = 0; i < 5; ++i) phase_ms[i] = 0.0f;  // nothing was enqueued
    } else {
        if (!rc) rc = cuda_status(cudaEventSynchronize(ev[5]), "event synchronize");
        for (int i = 0; i < 5 && !rc; ++i)
            rc = cuda_status(cudaEventElapsedTime(&phase_ms[i], ev[i], ev[i + 1]), "event time");
    }
    for (int i = 0; i < 6; ++i)
        if (ev[i]) cudaEventDestroy(ev[i]);
    return rc;
}
