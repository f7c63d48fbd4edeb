// Tensor-core GEMMs of the surrogate's training, for its three 256 x 256
// layers (the 6 -> 256 and 256 -> 2 layers stay on the FP32 kernel of
// mlp.cu):
//   forward       Z = round(H) round(W) + b,  H' = silu(Z)          M x 256, K = 256
//   input grad    dZ = (G round(W)^T) silu'(Z_below)                 M x 256, K = 256
//   weight grad   dW_s = round(H_s)^T G_s per slice s of rows        256 x 256, K = slice
// round() is the network's BF16 rounding, so those products are exact on the
// tensor cores; G, the FP32 gradient, enters as a BF16 pair hi + lo (within
// 2^-16 of G, two MMAs), which keeps each product within 2^-16 of the FP32
// one.  The FP32 accumulator in TMEM rounds partial sums towards zero, over
// at most 64 steps here (K = 512 in 16-element steps of two MMAs): below
// 64 x 2^-23 ~ 8e-6 of the sum of magnitudes.
// One CTA per 128 x 128 output tile (M = N = 128 MMAs; 2-3 CTAs per SM, the
// operand loads being latency-bound): warps 0-3 turn
// FP32 operands into BF16 tiles (K-major, 128-byte swizzle) in a two-stage
// ring of 64 contraction elements per stage; the weight operand comes
// pre-packed (mlp_tc_pack) by a bulk copy; warp 4 owns 256 TMEM columns and
// issues tcgen05.mma; warps 0-3 then read their 32 accumulator rows each and
// apply the epilogue.  The weight-gradient kernel's first row tile also sums
// G's columns over its slice as it converts them (the bias gradient).  Every
// wait is bounded; a CTA that gives up writes NaN.
#include "gen_tc.cuh"
#include "mlp_common.cuh"
#include "tc_common.cuh"

namespace xl {

constexpr int MT_ROWS = 128;                       // output rows per CTA (the MMA's M)
constexpr int MT_COLS = 128;                       // output columns per CTA (the MMA's N)
constexpr int MT_BH_BYTES = MT_COLS * 64 * 2;      // 16 KB: half of a packed weight tile
constexpr int MT_BK = 64;                          // contraction elements per stage
constexpr int MT_A_BYTES = MT_ROWS * MT_BK * 2;    // 16 KB
constexpr int MT_STAGES = 2;
constexpr int MT_THREADS = 160;

enum { MT_FWD = 0, MT_DX = 1, MT_DW = 2 };

template <int MODE>
struct MtCfg {
    static constexpr int A_TERMS = MODE == MT_DX ? 2 : 1;  // BF16 terms of the A operand
    static constexpr int B_TERMS = MODE == MT_DW ? 2 : 1;
    static constexpr int STAGE = A_TERMS * MT_A_BYTES + B_TERMS * MT_BH_BYTES;
    static constexpr bool B_BULK = MODE != MT_DW;  // B: packed weight tiles
    static constexpr int SMEM = 1024 + MT_STAGES * STAGE + 128;
};

struct MtShared {
    uint64_t full[MT_STAGES];   // 128 producer arrivals
    uint64_t wtx[MT_STAGES];    // the weight tile's bulk copy
    uint64_t empty[MT_STAGES];  // commit: the stage's MMAs are complete
    uint64_t done;              // commit: every MMA is complete
    uint32_t tmem_base;
    int abort;
};

struct MtArgs {
    const float* a;            // FWD: H; DX: G; DW: H ([M][256], rows = batch)
    const float* b;            // DW: G [M][256]
    const unsigned char* wpk;  // FWD / DX: the layer's 4 packed weight tiles
    const float* bias;         // FWD
    const float* zprev;        // DX
    float* z;                  // FWD (may be NULL)
    float* c;                  // FWD: activation; DX: dZ; DW: partials [S][257][256]
    int M;
    int k_slice;               // DW
};

__device__ __forceinline__ uint32_t bf2(float x, float y) {
    __nv_bfloat162 v = __floats2bfloat162_rn(x, y);
    return *reinterpret_cast<uint32_t*>(&v);
}

// 8 consecutive contraction elements v[0..7] of row r into the tile at
// column c (a multiple of 8): BF16-rounded, or as a hi/lo pair (lo_tile).
template <bool SPLIT>
__device__ __forceinline__ void put8(unsigned char* tile, unsigned char* lo_tile, int r, int c, const float (&v)[8]) {
    uint4 hi;
    hi.x = bf2(v[0], v[1]);
    hi.y = bf2(v[2], v[3]);
    hi.z = bf2(v[4], v[5]);
    hi.w = bf2(v[6], v[7]);
    const int off = sw128_offset(r, c);
    *reinterpret_cast<uint4*>(tile + off) = hi;
    if (SPLIT) {
        const uint32_t h[4] = {hi.x, hi.y, hi.z, hi.w};
        uint32_t l[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float h0 = __uint_as_float(h[q] << 16), h1 = __uint_as_float(h[q] & 0xFFFF0000u);
            l[q] = bf2(v[2 * q] - h0, v[2 * q + 1] - h1);
        }
        *reinterpret_cast<uint4*>(lo_tile + off) = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

// Row-major operand rows (batch) r of the tile, contraction columns kb..kb+63
// of X [M][256]: thread r reads its row's 64 values (all loads issued first:
// the conversion is bound by the memory requests in flight).
template <bool SPLIT>
__device__ __forceinline__ void load_rows(const float* __restrict__ X, int M, int row0, int kb, int r,
                                          unsigned char* tile, unsigned char* lo_tile) {
    const int m = row0 + r;
    float4 buf[MT_BK / 4];
    if (m < M) {
        const float4* src = reinterpret_cast<const float4*>(X + (int64_t)m * MLP_W + kb);
#pragma unroll
        for (int i = 0; i < MT_BK / 4; ++i) buf[i] = src[i];
    } else {
#pragma unroll
        for (int i = 0; i < MT_BK / 4; ++i) buf[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < MT_BK / 8; ++j) {
        const float4 p = buf[2 * j], q = buf[2 * j + 1];
        const float v[8] = {p.x, p.y, p.z, p.w, q.x, q.y, q.z, q.w};
        put8<SPLIT>(tile, lo_tile, r, 8 * j, v);
    }
}

// Transposed operand: tile row r = feature f0 + r, contraction columns =
// batch rows kb..kb+63 (zero from kend on) of X [M][256]; a warp's lanes read
// 32 consecutive features of one batch row (128 bytes) per load, all 64
// loads of a thread issued first.  csum (if non-NULL) accumulates the
// feature's values over the batch rows in order.
template <bool SPLIT>
__device__ __forceinline__ void load_cols(const float* __restrict__ X, int f0, int kb, int kend, int r,
                                          unsigned char* tile, unsigned char* lo_tile, float* csum) {
    float v[MT_BK / 8][8];
#pragma unroll
    for (int j = 0; j < MT_BK / 8; ++j)
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int b = kb + 8 * j + q;
            v[j][q] = b < kend ? X[(int64_t)b * MLP_W + f0 + r] : 0.f;
        }
#pragma unroll
    for (int j = 0; j < MT_BK / 8; ++j) {
        put8<SPLIT>(tile, lo_tile, r, 8 * j, v[j]);
        if (csum)
#pragma unroll
            for (int q = 0; q < 8; ++q) *csum += v[j][q];
    }
}

template <int MODE>
__global__ void __launch_bounds__(MT_THREADS, 2) mlp_gemm_tc_kernel(MtArgs a) {
    using C = MtCfg<MODE>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    MtShared* sh = reinterpret_cast<MtShared*>(base + MT_STAGES * C::STAGE);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row0 = blockIdx.x * MT_ROWS;  // FWD / DX: batch rows; DW: input features
    const int nh = MODE == MT_DW ? blockIdx.z : blockIdx.y;  // output columns nh * 128 ..
    const int col0 = nh * MT_COLS;
    const int k0 = MODE == MT_DW ? blockIdx.y * a.k_slice : 0;
    const int kend = MODE == MT_DW ? min(a.M, k0 + a.k_slice) : MLP_W;
    const int nst = (kend - k0 + MT_BK - 1) / MT_BK;
    volatile int* abort = &sh->abort;

    if (tid == 0) {
        for (int i = 0; i < MT_STAGES; ++i) {
            mbar_init(&sh->full[i], 128);
            mbar_init(&sh->wtx[i], 1);
            mbar_init(&sh->empty[i], 1);
        }
        mbar_init(&sh->done, 1);
        sh->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh->tmem_base)),
                     "r"(MT_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh->tmem_base;
    const uint32_t sbase = smem_u32(base);

    if (warp < 4) {
        // ---------------- operands
        int issued = 0;
        float csum0 = 0.f;  // DW, first row tile: column sums of G (the bias gradient)
        for (int s = 0; s < nst; ++s) {
            const int slot = s % MT_STAGES;
            if (s >= MT_STAGES && !mbar_wait(&sh->empty[slot], (uint32_t)((s / MT_STAGES - 1) & 1), abort)) break;
            unsigned char* st = base + slot * C::STAGE;
            const int kb = k0 + s * MT_BK;
            if (C::B_BULK && tid == 0) {
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&sh->wtx[slot])),
                             "r"(MT_BH_BYTES)
                             : "memory");
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        sbase + (uint32_t)(slot * C::STAGE + C::A_TERMS * MT_A_BYTES)),
                    "l"(a.wpk + (int64_t)s * MT_B_TILE_BYTES + nh * MT_BH_BYTES), "r"(MT_BH_BYTES),
                    "r"(smem_u32(&sh->wtx[slot]))
                    : "memory");
                ++issued;
            }
            if (MODE == MT_FWD) {
                load_rows<false>(a.a, a.M, row0, kb, tid, st, nullptr);
            } else if (MODE == MT_DX) {
                load_rows<true>(a.a, a.M, row0, kb, tid, st, st + MT_A_BYTES);
            } else {
                unsigned char* bt = st + MT_A_BYTES;
                load_cols<false>(a.a, row0, kb, kend, tid, st, nullptr, nullptr);
                load_cols<true>(a.b, col0, kb, kend, tid, bt, bt + MT_BH_BYTES, row0 == 0 ? &csum0 : nullptr);
            }
            fence_async_smem();
            mbar_arrive(&sh->full[slot]);
        }
        if (MODE == MT_DW && row0 == 0) {
            float* bias_row = a.c + ((int64_t)blockIdx.y * (MLP_W + 1) + MLP_W) * MLP_W;
            bias_row[col0 + tid] = csum0;
        }
        // no bulk copy may still be landing when the CTA exits
        if (C::B_BULK && tid == 0)
            for (int s = issued - MT_STAGES; s < issued; ++s)
                if (s >= 0) {
                    const uint64_t t0 = global_ns();
                    while (!mbar_try_wait(&sh->wtx[s % MT_STAGES], (uint32_t)((s / MT_STAGES) & 1)))
                        if (global_ns() - t0 > TC_WAIT_NS) break;
                }

        // ---------------- epilogue: warp w reads accumulator rows 32 w .. 32 w + 31
        const bool ok = mbar_wait(&sh->done, 0u, abort) && !*abort;
        tc_fence_after();
        const int r = 32 * warp + lane;
        const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
        const float nanv = __int_as_float(0x7fc00000);
        float* out;
        if (MODE == MT_DW)
            out = a.c + ((int64_t)blockIdx.y * (MLP_W + 1) + row0 + r) * MLP_W + col0;
        else
            out = a.c + (int64_t)(row0 + r) * MLP_W + col0;
        const bool live = MODE == MT_DW || row0 + r < a.M;
#pragma unroll 1
        for (int c0 = 0; c0 < MT_COLS; c0 += 16) {
            uint32_t acc[16];
            tmem_ld16(trow + (uint32_t)c0, acc);
            tmem_wait_ld();
            if (!live) continue;
            float v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = ok ? __uint_as_float(acc[j]) : nanv;
            if (MODE == MT_FWD) {
                float zz[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    zz[j] = v[j] + a.bias[col0 + c0 + j];
                    v[j] = silu_f(zz[j]);
                }
                if (a.z) {
                    float* zr = a.z + (int64_t)(row0 + r) * MLP_W + col0 + c0;
#pragma unroll
                    for (int j = 0; j < 16; j += 4)
                        *reinterpret_cast<float4*>(zr + j) = make_float4(zz[j], zz[j + 1], zz[j + 2], zz[j + 3]);
                }
            } else if (MODE == MT_DX) {
                const float* zp = a.zprev + (int64_t)(row0 + r) * MLP_W + col0 + c0;
#pragma unroll
                for (int j = 0; j < 16; j += 4) {
                    const float4 q = *reinterpret_cast<const float4*>(zp + j);
                    v[j] *= silu_grad_f(q.x);
                    v[j + 1] *= silu_grad_f(q.y);
                    v[j + 2] *= silu_grad_f(q.z);
                    v[j + 3] *= silu_grad_f(q.w);
                }
            }
#pragma unroll
            for (int j = 0; j < 16; j += 4)
                *reinterpret_cast<float4*>(out + c0 + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        }
    } else if (lane == 0) {
        // ---------------- MMA issuer
        const uint32_t idesc = tc_idesc<TCP_BF16X3, (uint32_t)MT_COLS>();
        for (int s = 0; s < nst; ++s) {
            const int slot = s % MT_STAGES;
            const uint32_t ph = (uint32_t)((s / MT_STAGES) & 1);
            if (!mbar_wait(&sh->full[slot], ph, abort)) break;
            if (C::B_BULK && !mbar_wait(&sh->wtx[slot], ph, abort)) break;
            tc_fence_after();
            const uint32_t st = sbase + (uint32_t)(slot * C::STAGE);
            const uint32_t bt = st + (uint32_t)(C::A_TERMS * MT_A_BYTES);
#pragma unroll
            for (int kk = 0; kk < MT_BK / 16; ++kk) {
                const uint32_t first = (s == 0 && kk == 0) ? 0u : 1u;
                const uint64_t da = desc_sw128(st + kk * 32), db = desc_sw128(bt + kk * 32);
                umma(tmem, da, db, idesc, first);
                if (C::A_TERMS == 2) umma(tmem, desc_sw128(st + MT_A_BYTES + kk * 32), db, idesc, 1u);
                if (C::B_TERMS == 2) umma(tmem, da, desc_sw128(bt + MT_BH_BYTES + kk * 32), idesc, 1u);
            }
            umma_commit(&sh->empty[slot]);
        }
        umma_commit(&sh->done);
        const uint64_t t0 = global_ns();  // nothing in flight once the tensor memory is released
        while (!mbar_try_wait(&sh->done, 0u))
            if (global_ns() - t0 > TC_WAIT_NS) break;
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 4) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(MT_COLS) : "memory");
    }
}

// One thread per packed element: layer l = 1..3, operand (0 forward: row =
// output unit, K = input; 1 input gradient: row = input unit, K = output),
// K chunk, row, column.
__global__ void mlp_tc_pack_kernel(const float* __restrict__ p, unsigned char* __restrict__ out) {
    const int64_t per_tile = 256 * 64, n = 3LL * 2 * 4 * per_tile;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int t = (int)(e / per_tile), w = (int)(e % per_tile);
        const int l = 1 + t / 8, op = (t / 4) % 2, kc = t % 4;
        const int row = w / 64, col = w % 64, k = kc * 64 + col;
        const float v = op == 0 ? p[mlp_off(l) + (int64_t)k * MLP_W + row] : p[mlp_off(l) + (int64_t)row * MLP_W + k];
        *reinterpret_cast<__nv_bfloat16*>(out + (int64_t)t * MT_B_TILE_BYTES + sw128_offset(row, col)) =
            __float2bfloat16_rn(v);
    }
}

template <int MODE>
static int launch_mt(const MtArgs& a, dim3 grid, cudaStream_t st) {
    constexpr int smem = MtCfg<MODE>::SMEM;
    static_assert(smem <= 227 * 1024, "shared memory");
    int rc = cuda_status(cudaFuncSetAttribute(mlp_gemm_tc_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                         "mlp tensor-core attribute");
    if (rc) return rc;
    mlp_gemm_tc_kernel<MODE><<<grid, MT_THREADS, smem, st>>>(a);
    return cuda_status(cudaGetLastError(), "mlp tensor-core gemm launch");
}

int mlp_tc_pack(const float* params, unsigned char* wpk, cudaStream_t st) {
    mlp_tc_pack_kernel<<<4 * num_sms(), 256, 0, st>>>(params, wpk);
    return cuda_status(cudaGetLastError(), "mlp training pack launch");
}

int mlp_tc_forward(const float* h, const unsigned char* wpk, int l, const float* bias, float* z, float* c, int M,
                   cudaStream_t st) {
    MtArgs a{};
    a.a = h;
    a.wpk = wpk + (int64_t)(l - 1) * MT_PACK_LAYER_BYTES;
    a.bias = bias;
    a.z = z;
    a.c = c;
    a.M = M;
    return launch_mt<MT_FWD>(a, dim3((unsigned)((M + MT_ROWS - 1) / MT_ROWS), MLP_W / MT_COLS), st);
}

int mlp_tc_input_grad(const float* g, const unsigned char* wpk, int l, const float* zprev, float* dz, int M,
                      cudaStream_t st) {
    MtArgs a{};
    a.a = g;
    a.wpk = wpk + (int64_t)(l - 1) * MT_PACK_LAYER_BYTES + 4LL * MT_B_TILE_BYTES;
    a.zprev = zprev;
    a.c = dz;
    a.M = M;
    return launch_mt<MT_DX>(a, dim3((unsigned)((M + MT_ROWS - 1) / MT_ROWS), MLP_W / MT_COLS), st);
}

int mlp_tc_weight_grad(const float* h, const float* g, int M, int k_slice, float* part, cudaStream_t st) {
    const int S = (M + k_slice - 1) / k_slice;
    MtArgs a{};
    a.a = h;
    a.b = g;
    a.c = part;
    a.M = M;
    a.k_slice = k_slice;
    return launch_mt<MT_DW>(a, dim3(2, (unsigned)S, MLP_W / MT_COLS), st);
}

}  // namespace xl
