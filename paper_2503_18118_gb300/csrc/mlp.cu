// Training side of the correlation surrogate: pair features and targets,
// forward and backward passes, loss, Adam, and the BF16 packing of the
// inference image.
//
// The three 256 x 256 layers run on the tensor cores (mlp_train_tc.cu:
// BF16-rounded operands, the network's stated numerics, with the FP32
// gradient as a BF16 hi/lo pair); the 6 -> 256 and 256 -> 2 layers are FP32
// SIMT tiles here (64 x 64 outputs, 16-deep K steps, 4 x 4 outputs per
// thread).  Both have fused epilogues: bias + SiLU in the forward pass, the
// SiLU derivative in the backward pass.  Weight gradients contract over the
// batch, split into slices whose partial sums are added in slice order by a
// second kernel, so results do not depend on scheduling; the backward pass
// reuses the rounded values of the forward pass.
#include <math.h>

#include "aperture.cuh"
#include "mlp_common.cuh"

namespace xl {

constexpr int GT = 64;        // output tile edge
constexpr int GKS = 16;       // K step
constexpr int GTHREADS = 256;
constexpr int DW_SLICE = 512; // batch rows per weight-gradient slice

enum { EPI_HIDDEN = 0, EPI_LINEAR = 1, EPI_DSILU = 2, EPI_PARTIAL = 3 };

struct GemmArgs {
    const float* A;   // A(m, k): AT ? A[k * lda + m] : A[m * lda + k]
    int64_t lda;
    const float* B;   // B(k, n): BT ? B[n * ldb + k] : B[k * ldb + n]
    int64_t ldb;
    int M, N, Kd;
    int ones_row;     // AT only: row m == ones_row of A reads 1 (bias gradient)
    int k_slice;      // K rows per blockIdx.z slice (EPI_PARTIAL)
    const float* bias;
    float* Z;         // EPI_HIDDEN: pre-activation (may be NULL)
    float* C;         // output (activation, linear output, dz, or partials)
    int64_t ldc;
    const float* zprev;  // EPI_DSILU: pre-activation of the layer below
};


template <bool AT, bool BT, bool QA, bool QB, int EPI>
__global__ void __launch_bounds__(GTHREADS) mlp_gemm_kernel(GemmArgs a) {
    __shared__ __align__(16) float As[GKS][GT + 4];
    __shared__ __align__(16) float Bs[GKS][GT + 4];
    const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
    const int m0 = blockIdx.x * GT, n0 = blockIdx.y * GT;
    int kbeg = 0, kend = a.Kd;
    if (EPI == EPI_PARTIAL) {
        kbeg = blockIdx.z * a.k_slice;
        kend = min(a.Kd, kbeg + a.k_slice);
    }
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

    for (int k0 = kbeg; k0 < kend; k0 += GKS) {
        // A tile -> As[k][m]
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int m, k;
            if (AT) { k = t >> 4; m = (t & 15) * 4 + r; }
            else    { m = t >> 2; k = (t & 3) * 4 + r; }
            const int gm = m0 + m, gk = k0 + k;
            float v = 0.f;
            if (gm < a.M && gk < kend) {
                if (AT) v = (gm == a.ones_row) ? 1.0f : a.A[(int64_t)gk * a.lda + gm];
                else v = a.A[(int64_t)gm * a.lda + gk];
                if (QA && !(AT && gm == a.ones_row)) v = bf16_round(v);
            }
            As[k][m] = v;
        }
        // B tile -> Bs[k][n]
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int n, k;
            if (BT) { n = t >> 2; k = (t & 3) * 4 + r; }
            else    { k = t >> 4; n = (t & 15) * 4 + r; }
            const int gn = n0 + n, gk = k0 + k;
            float v = 0.f;
            if (gn < a.N && gk < kend) {
                v = BT ? a.B[(int64_t)gn * a.ldb + gk] : a.B[(int64_t)gk * a.ldb + gn];
                if (QB) v = bf16_round(v);
            }
            Bs[k][n] = v;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < GKS; ++k) {
            const float4 av = *reinterpret_cast<const float4*>(&As[k][ty * 4]);
            const float4 bv = *reinterpret_cast<const float4*>(&Bs[k][tx * 4]);
            const float ar[4] = {av.x, av.y, av.z, av.w}, br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(ar[i], br[j], acc[i][j]);
        }
        __syncthreads();
    }

#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= a.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n >= a.N) continue;
            const float v = acc[i][j];
            if (EPI == EPI_HIDDEN) {
                const float z = v + a.bias[n];
                if (a.Z) a.Z[(int64_t)m * a.ldc + n] = z;
                a.C[(int64_t)m * a.ldc + n] = silu_f(z);
            } else if (EPI == EPI_LINEAR) {
                a.C[(int64_t)m * a.ldc + n] = v + a.bias[n];
            } else if (EPI == EPI_DSILU) {
                a.C[(int64_t)m * a.ldc + n] = v * silu_grad_f(a.zprev[(int64_t)m * a.ldc + n]);
            } else {
                a.C[((int64_t)blockIdx.z * a.M + m) * a.N + n] = v;
            }
        }
    }
}

template <bool AT, bool BT, bool QA, bool QB, int EPI>
static int gemm(const GemmArgs& a, int slices, cudaStream_t st) {
    dim3 grid((a.M + GT - 1) / GT, (a.N + GT - 1) / GT, slices);
    mlp_gemm_kernel<AT, BT, QA, QB, EPI><<<grid, GTHREADS, 0, st>>>(a);
    return cuda_status(cudaGetLastError(), "mlp gemm launch");
}

// grad[e] = sum over slices s of part[s][e], e < n, in slice order
__global__ void sum_slices_kernel(const float* __restrict__ part, int S, int64_t n, float* __restrict__ grad) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int k = 0; k < S; ++k) s += part[(int64_t)k * n + e];
        grad[e] = s;
    }
}

__global__ void mlp_loss_kernel(const float2* __restrict__ out, const float2* __restrict__ tgt,
                                const float* __restrict__ w, int M, float2* __restrict__ dout, float* __restrict__ loss) {
    __shared__ float red[32];
    const float inv_m = 1.0f / (float)M;
    float s = 0.f;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        const float2 o = out[m], tg = tgt[m];
        const float wm = w ? w[m] : 1.0f;
        const float dx = o.x - tg.x, dy = o.y - tg.y;
        dout[m] = make_float2(wm * dx * inv_m, wm * dy * inv_m);
        s = fmaf(wm, dx * dx + dy * dy, s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0 && loss) *loss = 0.5f * s * inv_m;
    }
}

__global__ void mlp_adam_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                                const float* __restrict__ g, int64_t n, float lr, float b1, float omb1, float b2,
                                float omb2, float eps, float c1, float c2) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const float ge = g[e];
        const float me = b1 * m[e] + omb1 * ge;
        const float ve = b2 * v[e] + omb2 * ge * ge;
        m[e] = me;
        v[e] = ve;
        p[e] -= lr * (me * c1) / (sqrtf(ve * c2) + eps);
    }
}

__global__ void pair_features_kernel(FeatConst fc, int base, double H, double inv_lambda,
                                     const double2* __restrict__ users, int K, int64_t rows,
                                     const double2* __restrict__ gram, const double2* __restrict__ gcf,
                                     float* __restrict__ feat, float2* __restrict__ target, float* __restrict__ weight) {
    const int P = K * (K - 1) / 2;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = r / P;
        int i, j;
        pair_index((int)(r - b * P), K, i, j);
        const double2 ui = users[b * K + i], uj = users[b * K + j];
        float f[MLP_IN];
        pair_features_dev(fc, ui.x, ui.y, uj.x, uj.y, f);
#pragma unroll
        for (int c = 0; c < MLP_IN; ++c) feat[r * MLP_IN + c] = f[c];
        const int64_t g0 = b * K * K;
        if (target) {
            const double2 ge = gram[g0 + i * K + j], gc = gcf[g0 + i * K + j];
            const double den = gc.x * gc.x + gc.y * gc.y;
            const double re = (ge.x * gc.x + ge.y * gc.y) / den, im = (ge.y * gc.x - ge.x * gc.y) / den;
            const float2 f = aperture_factor(base, ui.x, ui.y, uj.x, uj.y, H, inv_lambda);
            target[r] = make_float2((float)(re - (double)f.x), (float)(im - (double)f.y));
        }
        if (weight) {
            const double2 gc = gcf[g0 + i * K + j];
            weight[r] = (float)((gc.x * gc.x + gc.y * gc.y) / (gcf[g0 + i * K + i].x * gcf[g0 + j * K + j].x));
        }
    }
}

// One thread per element of the BF16 tiles, then the FP32 block (layout in
// mlp_common.cuh).
__global__ void mlp_pack_kernel(const float* __restrict__ p, unsigned char* __restrict__ out) {
    const int64_t n_bf = (int64_t)MLP_TILES * 128 * 64;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_bf + MLP_PK_NF;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (e < n_bf) {
            const int tile = (int)(e / (128 * 64)), w = (int)(e % (128 * 64));
            const int row = w / 64, col = w % 64;  // row: output unit in the half, col: input in the tile
            __nv_bfloat16 v;
            if (tile < 2) {
                const int n = tile * 128 + row;
                float x = 0.0f;
                if (col < 3 * MLP_IN) x = 0.5f * p[mlp_off(0) + (int64_t)(col % MLP_IN) * MLP_W + n];
                const __nv_bfloat16 hi = __float2bfloat16_rn(x);
                v = col < 2 * MLP_IN ? hi : __float2bfloat16_rn(x - __bfloat162float(hi));
            } else {
                const int t = tile - 2;
                const int l = 1 + t / 8, nh = (t / 4) % 2, kc = t % 4;
                const int n = nh * 128 + row, k = kc * 64 + col;
                v = __float2bfloat16_rn(0.5f * p[mlp_off(l) + (int64_t)k * MLP_W + n]);
            }
            *reinterpret_cast<__nv_bfloat16*>(out + (int64_t)tile * MLP_TILE_BYTES + sw128_offset(row, col)) = v;
        } else {
            const int f = (int)(e - n_bf);
            float v;
            if (f < MLP_PK_W4) {
                const int l = f / MLP_W;  // b0/2 .. b3/2
                v = 0.5f * p[mlp_off(l) + (int64_t)mlp_in(l) * MLP_W + f % MLP_W];
            } else if (f < MLP_PK_B4) {
                v = p[mlp_off(4) + (f - MLP_PK_W4)];  // W4
            } else {
                v = p[mlp_off(4) + MLP_W * MLP_OUT + (f - MLP_PK_B4)];  // b4
            }
            reinterpret_cast<float*>(out + MLP_PK_F32)[f] = v;
        }
    }
}

static int grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    const int64_t cap = 16LL * num_sms();
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

static inline float* cache_z(float* cache, int l, int M) { return cache + (int64_t)(2 * l) * M * MLP_W; }
static inline float* cache_h(float* cache, int l, int M) { return cache + (int64_t)(2 * l + 1) * M * MLP_W; }

static int dw_slices(int M) { return (M + DW_SLICE - 1) / DW_SLICE; }
static int dw_slices_tc(int M) { return (M + MT_DW_SLICE - 1) / MT_DW_SLICE; }  // >= dw_slices(M)

// forward; with cache == NULL the hidden activations go to `tmp` ([2][M][256]);
// wpk: the packed weights of the 256 x 256 layers (mlp_tc_pack)
static int mlp_forward_impl(const float* params, const float* x, int M, float* out, float* cache, float* tmp,
                            const unsigned char* wpk, cudaStream_t st) {
    int rc = XLMIMO_OK;
    const float* h = x;
    for (int l = 0; l < MLP_LAYERS && !rc; ++l) {
        GemmArgs a{};
        a.A = h;
        a.lda = mlp_in(l);
        a.B = params + mlp_off(l);
        a.ldb = mlp_out(l);
        a.M = M;
        a.N = mlp_out(l);
        a.Kd = mlp_in(l);
        a.ones_row = -1;
        a.bias = params + mlp_off(l) + (int64_t)mlp_in(l) * mlp_out(l);
        a.ldc = mlp_out(l);
        if (l == MLP_LAYERS - 1) {
            a.C = out;
            rc = gemm<false, false, false, false, EPI_LINEAR>(a, 1, st);
        } else {
            a.Z = cache ? cache_z(cache, l, M) : nullptr;
            a.C = cache ? cache_h(cache, l, M) : tmp + (int64_t)(l & 1) * M * MLP_W;
            if (l == 0) rc = gemm<false, false, false, false, EPI_HIDDEN>(a, 1, st);
            else rc = mlp_tc_forward(h, wpk, l, a.bias, a.Z, a.C, M, st);
            h = a.C;
        }
    }
    return rc;
}

static int mlp_backward_impl(const float* params, const float* x, const float* cache, const float* dout, int M,
                             float* grad, float* work, const unsigned char* wpk, cudaStream_t st) {
    float* dz[2] = {work, work + (int64_t)M * MLP_W};
    float* part = work + 2LL * M * MLP_W;
    const int S = dw_slices(M);
    const float* g = dout;  // gradient at the output of layer l
    int rc = XLMIMO_OK;
    for (int l = MLP_LAYERS - 1; l >= 0 && !rc; --l) {
        const int in = mlp_in(l), outd = mlp_out(l);
        const float* hin = l == 0 ? x : cache_h(const_cast<float*>(cache), l - 1, M);
        // weight and bias gradient: [in + 1][out] = [h | 1]^T g, sliced over the batch
        GemmArgs a{};
        a.A = hin;
        a.lda = in;
        a.B = g;
        a.ldb = outd;
        a.M = in + 1;
        a.N = outd;
        a.Kd = M;
        a.ones_row = in;
        a.k_slice = DW_SLICE;
        a.C = part;
        const bool q = (l >= 1 && l <= 3);
        rc = q ? mlp_tc_weight_grad(hin, g, M, MT_DW_SLICE, part, st)
               : gemm<true, false, false, false, EPI_PARTIAL>(a, S, st);
        if (rc) break;
        const int64_t n = (int64_t)(in + 1) * outd;
        sum_slices_kernel<<<grid_for(n, 256), 256, 0, st>>>(part, q ? dw_slices_tc(M) : S, n, grad + mlp_off(l));
        rc = cuda_status(cudaGetLastError(), "mlp gradient reduce");
        if (rc || l == 0) break;
        // input gradient through W (rounded as in the forward pass) and SiLU'
        GemmArgs d{};
        d.A = g;
        d.lda = outd;
        d.B = params + mlp_off(l);  // B(k = out unit, n = in unit) = W[in][out]
        d.ldb = outd;
        d.M = M;
        d.N = in;
        d.Kd = outd;
        d.ones_row = -1;
        d.C = dz[l & 1];
        d.ldc = in;
        d.zprev = cache_z(const_cast<float*>(cache), l - 1, M);
        rc = q ? mlp_tc_input_grad(g, wpk, l, d.zprev, d.C, M, st)
               : gemm<false, true, false, false, EPI_DSILU>(d, 1, st);
        g = d.C;
    }
    return rc;
}

static int check_m(int M) {
    if (M < 0 || M > (1 << 24)) { set_error("M must be in [0, 2^24], got %d", M); return XLMIMO_EINVAL; }
    return XLMIMO_OK;
}

// Adam's scalar arguments, checked before a training step enqueues anything
static int check_adam(int64_t step, double lr, double beta1, double beta2, double eps) {
    if (step < 1) { set_error("step must be >= 1"); return XLMIMO_EINVAL; }
    if (!(lr >= 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0)) {
        set_error("need lr >= 0, beta1 and beta2 in [0, 1), eps > 0");
        return XLMIMO_EINVAL;
    }
    return XLMIMO_OK;
}

}  // namespace xl

using namespace xl;

extern "C" {

int xlmimo_pair_features(const xlmimo_array* arr, const double* users, int K, int B, int base, const double* gram,
                         const double* gram_cf, float* feat, float* target, float* weight, void* stream) {
    clear_error();
    Geom g;
    int rc = check_array(arr, &g);
    if (rc) return rc;
    if (K < 2 || K > XLMIMO_MAX_USERS || B < 0) { set_error("K must be in [2, 64] and B >= 0"); return XLMIMO_EINVAL; }
    if (base < XLMIMO_APERTURE_NONE || base > XLMIMO_APERTURE_FRESNEL) { set_error("unknown base %d", base); return XLMIMO_EINVAL; }
    if (target && (!gram || !gram_cf)) { set_error("targets need gram and gram_cf"); return XLMIMO_EINVAL; }
    if (weight && !gram_cf) { set_error("weights need gram_cf"); return XLMIMO_EINVAL; }
    if (B == 0) return XLMIMO_OK;
    if (!users || !feat) { set_error("users and feat must be non-NULL"); return XLMIMO_EINVAL; }
    const int64_t rows = (int64_t)B * (K * (K - 1) / 2);
    pair_features_kernel<<<grid_for(rows, 256), 256, 0, as_stream(stream)>>>(
        make_feat_const(g), base, 0.5 * (double)g.N * g.spacing, g.inv_lambda, (const double2*)users, K, rows,
        (const double2*)gram, (const double2*)gram_cf, feat, (float2*)target, weight);
    return cuda_status(cudaGetLastError(), "pair features launch");
}

int xlmimo_mlp_forward(const float* params, const float* x, int M, float* out, float* cache, void* stream) {
    clear_error();
    int rc = check_m(M);
    if (rc || M == 0) return rc;
    if (!params || !x || !out) { set_error("params, x and out must be non-NULL"); return XLMIMO_EINVAL; }
    float* tmp = nullptr;
    unsigned char* wpk = nullptr;
    cudaStream_t st = as_stream(stream);
    rc = cuda_status(cudaMallocAsync((void**)&wpk, (size_t)MT_PACK_BYTES, st), "forward workspace");
    if (!rc && !cache)
        rc = cuda_status(cudaMallocAsync((void**)&tmp, sizeof(float) * 2 * (size_t)M * MLP_W, st), "forward workspace");
    if (!rc) rc = mlp_tc_pack(params, wpk, st);
    if (!rc) rc = mlp_forward_impl(params, x, M, out, cache, tmp, wpk, st);
    if (tmp) cudaFreeAsync(tmp, st);
    if (wpk) cudaFreeAsync(wpk, st);
    return rc;
}

int xlmimo_mlp_loss(const float* out, const float* target, const float* weight, int M, float* dout, float* loss,
                    void* stream) {
    clear_error();
    int rc = check_m(M);
    if (rc || M == 0) return rc;
    if (!out || !target || !dout) { set_error("out, target and dout must be non-NULL"); return XLMIMO_EINVAL; }
    mlp_loss_kernel<<<1, 1024, 0, as_stream(stream)>>>((const float2*)out, (const float2*)target, weight, M,
                                                      (float2*)dout, loss);
    return cuda_status(cudaGetLastError(), "mlp loss launch");
}

// workspace: dZ [2][M][256], weight-gradient partials [S][257][256] (S for
// the 256-row slices of the tensor-core layers, which the FP32 layers' 512-row
// slices fit in), packed
// weights of the 256 x 256 layers (MT_PACK_BYTES)
static int64_t work_pack_off(int M) { return 2LL * M * MLP_W + (int64_t)dw_slices_tc(M) * (MLP_W + 1) * MLP_W; }

int64_t xlmimo_mlp_work_floats(int M) {
    if (M <= 0) return 0;
    return work_pack_off(M) + MT_PACK_BYTES / 4;
}

int xlmimo_mlp_backward(const float* params, const float* x, const float* cache, const float* dout, int M,
                        float* grad, float* work, void* stream) {
    clear_error();
    int rc = check_m(M);
    if (rc) return rc;
    if (!params || !grad) { set_error("params and grad must be non-NULL"); return XLMIMO_EINVAL; }
    if (M == 0) return cuda_status(cudaMemsetAsync(grad, 0, sizeof(float) * XLMIMO_MLP_PARAMS, as_stream(stream)), "grad clear");
    if (!x || !cache || !dout || !work) { set_error("x, cache, dout and work must be non-NULL"); return XLMIMO_EINVAL; }
    if (((uintptr_t)work & 15u) != 0) { set_error("work must be 16-byte aligned"); return XLMIMO_EINVAL; }
    cudaStream_t st = as_stream(stream);
    unsigned char* wpk = reinterpret_cast<unsigned char*>(work + work_pack_off(M));
    rc = mlp_tc_pack(params, wpk, st);
    return rc ? rc : mlp_backward_impl(params, x, cache, dout, M, grad, work, wpk, st);
}

int xlmimo_mlp_adam(float* params, float* m, float* v, const float* grad, int64_t step, double lr, double beta1,
                    double beta2, double eps, void* stream) {
    clear_error();
    if (!params || !m || !v || !grad) { set_error("params, m, v and grad must be non-NULL"); return XLMIMO_EINVAL; }
    int rc = check_adam(step, lr, beta1, beta2, eps);
    if (rc) return rc;
    const double c1 = 1.0 / (1.0 - pow(beta1, (double)step)), c2 = 1.0 / (1.0 - pow(beta2, (double)step));
    mlp_adam_kernel<<<grid_for(XLMIMO_MLP_PARAMS, 256), 256, 0, as_stream(stream)>>>(
        params, m, v, grad, XLMIMO_MLP_PARAMS, (float)lr, (float)beta1, (float)(1.0 - beta1), (float)beta2,
        (float)(1.0 - beta2), (float)eps, (float)c1, (float)c2);
    return cuda_status(cudaGetLastError(), "adam launch");
}

int xlmimo_mlp_train_step(float* params, float* m, float* v, float* grad, int64_t step, double lr, const float* x,
                          const float* target, const float* weight, int M, float* out, float* cache, float* work,
                          float* loss, void* stream) {
    clear_error();
    int rc = check_m(M);
    if (rc) return rc;
    if (M == 0) { set_error("M must be >= 1"); return XLMIMO_EINVAL; }
    if (!params || !m || !v || !grad || !x || !target || !out || !cache || !work) {
        set_error("params, m, v, grad, x, target, out, cache and work must be non-NULL");
        return XLMIMO_EINVAL;
    }
    if (((uintptr_t)work & 15u) != 0) { set_error("work must be 16-byte aligned"); return XLMIMO_EINVAL; }
    rc = check_adam(step, lr, 0.9, 0.999, 1e-8);
    if (rc) return rc;
    cudaStream_t st = as_stream(stream);
    // the output gradient reuses the head of the workspace's second slab
    float* dout = work + (int64_t)M * MLP_W;
    unsigned char* wpk = reinterpret_cast<unsigned char*>(work + work_pack_off(M));
    rc = mlp_tc_pack(params, wpk, st);
    if (!rc) rc = mlp_forward_impl(params, x, M, out, cache, nullptr, wpk, st);
    if (!rc) {
        mlp_loss_kernel<<<1, 1024, 0, st>>>((const float2*)out, (const float2*)target, weight, M, (float2*)dout, loss);
        rc = cuda_status(cudaGetLastError(), "mlp loss launch");
    }
    if (!rc) rc = mlp_backward_impl(params, x, cache, dout, M, grad, work, wpk, st);
    if (!rc) rc = xlmimo_mlp_adam(params, m, v, grad, step, lr, 0.9, 0.999, 1e-8, stream);
    return rc;
}

int xlmimo_mlp_pack(const float* params, void* packed, void* stream) {
    clear_error();
    if (!params || !packed) { set_error("params and packed must be non-NULL"); return XLMIMO_EINVAL; }
    if (((uintptr_t)packed & 15u) != 0) { set_error("packed must be 16-byte aligned"); return XLMIMO_EINVAL; }
    const int64_t n = (int64_t)MLP_TILES * 128 * 64 + MLP_PK_NF;
    mlp_pack_kernel<<<grid_for(n, 256), 256, 0, as_stream(stream)>>>(params, (unsigned char*)packed);
    return cuda_status(cudaGetLastError(), "mlp pack launch");
}

}  // extern "C"
