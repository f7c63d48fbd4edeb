// Fused tensor-core inference of the correlation surrogate: one CTA takes 128
// pair rows through the whole network and corrects their closed-form Gram
// entries in place.
//
//   rows warps 0-3 (thread = row): pair features, the 6 -> 256 layer in FP32,
//          SiLU, BF16 rows into the A tile (128 x 256, K-major, 128-byte
//          swizzle); after each tensor-core layer, TMEM -> registers, bias,
//          SiLU, BF16 back into the A tile; after the last, the 256 -> 2 layer
//          in FP32 and the complex correction G~_ij (1 + t_ij).
//   warp 4 streams the 24 weight tiles (16 KB: 128 output units x 64 inputs,
//          BF16, already in the swizzled operand layout) with bulk copies
//          through a two-stage ring.
//   warp 5 owns TMEM (256 columns: one FP32 128 x 256 accumulator) and issues
//          tcgen05.mma (M = N = 128, K = 16): per layer two output halves x
//          four 64-input chunks x four K steps.
// The A tile is rewritten only after the layer that reads it has completed
// (its commit is the rows' signal), and the accumulator only after the rows
// have read it (their arrival is the MMA warp's signal).  Every wait is
// bounded; a CTA that gives up writes NaN to its pairs.  Two CTAs fit on an
// SM (110 KB shared memory, 256 TMEM columns each), so one CTA's SiLU work
// overlaps the other's matrix products.
#include "mlp_common.cuh"
#include "tc_common.cuh"

namespace xl {

constexpr int MI_ROWS = 128;
constexpr int MI_THREADS = 192;
constexpr int MI_STAGES = 2;
constexpr uint32_t MI_TMEM_COLS = 256;
constexpr int MI_A_BYTES = 4 * MLP_TILE_BYTES;
constexpr int MI_F32_BYTES = (MLP_PK_NF * 4 + 15) / 16 * 16;

struct MiShared {
    uint64_t full[MI_STAGES];
    uint64_t empty[MI_STAGES];
    uint64_t a_ready;
    uint64_t d_ready;
    uint64_t fin;
    uint32_t tmem_base;
    int abort;
};

constexpr int MI_SMEM = 1024 + MI_A_BYTES + MI_STAGES * MLP_TILE_BYTES + MI_F32_BYTES + (int)sizeof(MiShared);

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Wait bounded by time only (used on the way out, after an abort).
__device__ __forceinline__ bool mbar_wait_timed(uint64_t* bar, uint32_t parity) {
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > TC_WAIT_NS) return false;
    return true;
}

__device__ __forceinline__ float tanh_approx(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// SiLU feeding a BF16 operand: z/2 (1 + tanh(z/2)), one MUFU op.
__device__ __forceinline__ float silu_tanh(float z) {
    const float hz = 0.5f * z;
    return fmaf(hz, tanh_approx(hz), hz);
}

// SiLU feeding the FP32 output layer.
__device__ __forceinline__ float silu_exp(float z) { return __fdividef(z, 1.0f + __expf(-z)); }

// 32 activations of row m (columns 32 cb .. 32 cb + 31) -> BF16 A tile
__device__ __forceinline__ void store_a_row(unsigned char* A, int m, int cb, const float* h) {
    unsigned char* tile = A + (cb >> 1) * MLP_TILE_BYTES + (m >> 3) * 1024 + (m & 7) * 128;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            __nv_bfloat162 p = __floats2bfloat162_rn(h[u * 8 + 2 * q], h[u * 8 + 2 * q + 1]);
            w[q] = *reinterpret_cast<uint32_t*>(&p);
        }
        const int unit = ((cb & 1) * 4 + u) ^ (m & 7);
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(smem_u32(tile + unit * 16)), "r"(w[0]),
                     "r"(w[1]), "r"(w[2]), "r"(w[3])
                     : "memory");
    }
}

__global__ void __launch_bounds__(MI_THREADS, 2)
    mlp_infer_tc_kernel(FeatConst fc, const double2* __restrict__ users, int K, int64_t rows,
                        const unsigned char* __restrict__ packed, double2* __restrict__ gram) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char* A = base;
    unsigned char* ring = A + MI_A_BYTES;
    float* pf = reinterpret_cast<float*>(ring + MI_STAGES * MLP_TILE_BYTES);
    MiShared* sh = reinterpret_cast<MiShared*>(reinterpret_cast<unsigned char*>(pf) + MI_F32_BYTES);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int P = K * (K - 1) / 2;

    if (tid == 0) {
        for (int s = 0; s < MI_STAGES; ++s) {
            mbar_init(&sh->full[s], 1);
            mbar_init(&sh->empty[s], 1);
        }
        mbar_init(&sh->a_ready, MI_ROWS);
        mbar_init(&sh->d_ready, 1);
        mbar_init(&sh->fin, 1);
        sh->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh->tmem_base)),
                     "r"(MI_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    const float* gpf = reinterpret_cast<const float*>(packed + MLP_PK_F32);
    for (int e = tid; e < MLP_PK_NF; e += MI_THREADS) pf[e] = gpf[e];
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh->tmem_base;
    volatile int* abort = &sh->abort;

    if (warp == 4) {
        // ---------------- weight tiles through the ring
        if (lane == 0) {
            int issued = 0;
            for (int c = 0; c < MLP_TILES; ++c) {
                const int s = c % MI_STAGES;
                if (c >= MI_STAGES && !mbar_wait(&sh->empty[s], ((c / MI_STAGES) - 1) & 1, abort)) break;
                bulk_load(smem_u32(ring + s * MLP_TILE_BYTES), packed + (int64_t)c * MLP_TILE_BYTES, MLP_TILE_BYTES,
                          &sh->full[s]);
                ++issued;
            }
            // no copy may still be landing when the CTA exits
            for (int c = issued - MI_STAGES; c < issued; ++c)
                if (c >= 0) mbar_wait_timed(&sh->full[c % MI_STAGES], (c / MI_STAGES) & 1);
        }
        __syncwarp();
    } else if (warp == 5) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = tc_idesc<TCP_BF16>();
            bool ok = true;
            for (int l = 0; l < 3 && ok; ++l) {
                if (!mbar_wait(&sh->a_ready, l & 1, abort)) { ok = false; break; }
                tc_fence_after();
                for (int nh = 0; nh < 2 && ok; ++nh) {
                    for (int kc = 0; kc < 4; ++kc) {
                        const int c = l * 8 + nh * 4 + kc, s = c % MI_STAGES;
                        if (!mbar_wait(&sh->full[s], (c / MI_STAGES) & 1, abort)) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t a0 = smem_u32(A + kc * MLP_TILE_BYTES);
                        const uint32_t b0 = smem_u32(ring + s * MLP_TILE_BYTES);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            umma(tmem + nh * 128, desc_sw128(a0 + kk * 32), desc_sw128(b0 + kk * 32), idesc,
                                 (kc | kk) ? 1u : 0u);
                        umma_commit(&sh->empty[s]);
                    }
                }
                if (ok) umma_commit(&sh->d_ready);
            }
            umma_commit(&sh->fin);  // arrives once every MMA issued above has completed
        }
        __syncwarp();
    } else {
        // ---------------- rows
        const int m = warp * 32 + lane;
        const int64_t r = (int64_t)blockIdx.x * MI_ROWS + m;
        const bool valid = r < rows;
        int64_t b = 0;
        int i = 0, j = 1;
        float f[MLP_IN] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (valid) {
            b = r / P;
            pair_index((int)(r - b * P), K, i, j);
            const double2 ui = users[b * K + i], uj = users[b * K + j];
            pair_features_dev(fc, ui.x, ui.y, uj.x, uj.y, f);
        }
        // layer 0 (FP32)
        for (int cb = 0; cb < 8; ++cb) {
            float h[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const int c = cb * 32 + q;
                float z = pf[MLP_PK_B0 + c];
#pragma unroll
                for (int e = 0; e < MLP_IN; ++e) z = fmaf(f[e], pf[MLP_PK_W0 + e * MLP_W + c], z);
                h[q] = silu_tanh(z);
            }
            store_a_row(A, m, cb, h);
        }
        fence_async_smem();
        mbar_arrive(&sh->a_ready);

        float o0 = pf[MLP_PK_B4], o1 = pf[MLP_PK_B4 + 1];
        bool ok = true;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        for (int l = 0; l < 3; ++l) {
            if (!mbar_wait(&sh->d_ready, l & 1, abort)) { ok = false; break; }
            tc_fence_after();
            const float* bias = pf + MLP_PK_B1 + l * MLP_W;
            for (int cb = 0; cb < 8; ++cb) {
                float v[32];
                tmem_ld32(trow + cb * 32, v);
                if (l < 2) {
#pragma unroll
                    for (int q = 0; q < 32; ++q) v[q] = silu_tanh(v[q] + bias[cb * 32 + q]);
                    store_a_row(A, m, cb, v);
                } else {
#pragma unroll
                    for (int q = 0; q < 32; ++q) {
                        const int c = cb * 32 + q;
                        const float hv = silu_exp(v[q] + bias[c]);
                        o0 = fmaf(hv, pf[MLP_PK_W4 + 2 * c], o0);
                        o1 = fmaf(hv, pf[MLP_PK_W4 + 2 * c + 1], o1);
                    }
                }
            }
            if (l < 2) {
                fence_async_smem();
                tc_fence_before();
                mbar_arrive(&sh->a_ready);
            }
        }
        if (valid) {
            const int64_t g0 = b * K * K;
            if (ok && !*abort) {
                const double2 gc = gram[g0 + i * K + j];
                const double t0 = (double)o0, t1 = (double)o1;
                const double re = gc.x + (gc.x * t0 - gc.y * t1), im = gc.y + (gc.x * t1 + gc.y * t0);
                gram[g0 + i * K + j] = make_double2(re, im);
                gram[g0 + j * K + i] = make_double2(re, -im);
            } else {
                const double nanv = __longlong_as_double(0x7ff8000000000000ULL);
                gram[g0 + i * K + j] = make_double2(nanv, nanv);
                gram[g0 + j * K + i] = make_double2(nanv, nanv);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 5) {
        if (lane == 0) mbar_wait_timed(&sh->fin, 0);
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(MI_TMEM_COLS) : "memory");
    }
}

static int mlp_infer_prepare() {
    static bool done[64] = {false};
    int dev = 0;
    int rc = cuda_status(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc) return rc;
    if (dev < 64 && done[dev]) return XLMIMO_OK;
    rc = cuda_status(cudaFuncSetAttribute(mlp_infer_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, MI_SMEM),
                     "surrogate kernel attribute");
    if (!rc && dev < 64) done[dev] = true;
    return rc;
}

}  // namespace xl

using namespace xl;

extern "C" int xlmimo_surrogate_gram(const xlmimo_array* arr, const double* users, int K, int B, const void* packed,
                                     double* gram, void* stream) {
    clear_error();
    Geom g;
    int rc = check_array(arr, &g);
    if (rc) return rc;
    if (K < 1 || K > XLMIMO_MAX_USERS || B < 0) { set_error("K must be in [1, 64] and B >= 0"); return XLMIMO_EINVAL; }
    if (B == 0) return XLMIMO_OK;
    if (!users || !gram || !packed) { set_error("users, packed and gram must be non-NULL"); return XLMIMO_EINVAL; }
    if (((uintptr_t)packed & 15u) != 0) { set_error("packed must be 16-byte aligned"); return XLMIMO_EINVAL; }
    cudaStream_t st = as_stream(stream);
    rc = launch_closed_form(g, users, K, B, gram, st);
    if (rc || K < 2) return rc;
    if ((rc = mlp_infer_prepare())) return rc;
    const int64_t rows = (int64_t)B * (K * (K - 1) / 2);
    const int64_t grid = (rows + MI_ROWS - 1) / MI_ROWS;
    if (grid > 0x7fffffffLL) { set_error("too many pairs for one launch (B * K(K-1)/2 > 2^38)"); return XLMIMO_EINVAL; }
    mlp_infer_tc_kernel<<<(unsigned)grid, MI_THREADS, MI_SMEM, st>>>(make_feat_const(g), (const double2*)users, K, rows,
                                                                      (const unsigned char*)packed, (double2*)gram);
    return cuda_status(cudaGetLastError(), "surrogate kernel launch");
}
