// Fused tensor-core inference of the correlation surrogate: a persistent CTA
// takes tiles of 128 pair rows through the whole network and corrects their
// closed-form Gram entries in place.  The barrier set-up, TMEM allocation and
// parameter load happen once per CTA; a tile's pair indices, positions and
// closed-form entries are fetched while the previous tile is in flight, and
// the weight stream runs on into the next tile.
//
// Two CTAs per SM, one tile of 128 pair rows in flight each, a two-stage
// weight ring each.  Measured on a per-CTA clock64 timeline, each layer's
// MMAs waited ~800 cycles per 16 KB weight tile (L2 latency with two tiles in
// flight, the crossbar at 15 % of its peak) and the SiLU epilogue was
// issue-bound with four row warps per scheduler.  Two lockstep tiles per CTA
// sharing each weight tile (five-stage ring) and one tile per CTA at one CTA
// per SM (nine-stage ring) were both measured slower: without a second CTA the
// SiLU epilogue of one half is not hidden behind the other half's products.
//
//   row warps (8): thread (m, h) owns output units 128 h .. 128 h + 127 of
//          row m of the tile (m = 32 (warp % 4) + lane, h = warp / 4).  It
//          writes the features (half 0:
//          [hi(f), lo(f), hi(f)] in BF16) into its tile's A (128 x 256 BF16,
//          K-major, 128-byte swizzle); after each layer it reads its 128
//          accumulators from TMEM, adds the bias and applies SiLU as
//          z/2 (1 + tanh(z/2)) (the packed weights hold W/2, so the
//          accumulator already is z/2), and writes BF16 back into its half of
//          A; after the last hidden layer it forms its half of the FP32
//          256 -> 2 product, the halves are added, and half 0 applies
//          G~_ij (1 + t_ij).
//   loader warp streams the 26 weight tiles (16 KB: 128 output units x 64
//          inputs, BF16, stored in the swizzled operand layout) through the
//          ring with bulk copies; a slot is refilled once the MMA warp has
//          released it.
//   MMA warp owns TMEM (256 columns: an FP32 128 x 256 accumulator) and
//          issues tcgen05.mma (M = N = 128, K = 16) half by half, committing
//          each half separately so half 0's epilogue runs while half 1
//          multiplies.
// SiLU uses the FP32 tanh (relative error ~2^-11) in every layer; in the last
// hidden layer, which feeds the FP32 output layer directly, the exact form
// (exp and divide, two MUFU ops) was measured to change neither the output
// error nor the sum rate, and cost 12 % of the kernel.
// Ordering: a layer's MMAs start once every row thread has written A and read
// the accumulator (one arrival each); half 0 overwrites its A columns only
// after half 1's MMAs have read them (a separate commit after half 1's first
// two input chunks); half 1's accumulator commit implies the whole layer is
// done.  Every wait is bounded; a CTA that gives up writes NaN to its pairs.
#include <algorithm>

#include "mlp_common.cuh"
#include "tc_common.cuh"

namespace xl {

constexpr int MI_ROWS = 128;  // pair rows per tile (the MMA's M)
constexpr int MI_A_BYTES = 4 * MLP_TILE_BYTES;
constexpr int MI_F32_BYTES = (MLP_PK_NF * 4 + 15) / 16 * 16;

// Warp roles, ring depth (what the shared memory of two CTAs per SM holds)
// and tensor memory of the inference kernel.
struct MiCfg {
    static constexpr int ROW_WARPS = 8;
    static constexpr int LOADER = ROW_WARPS, MMA = ROW_WARPS + 1;
    static constexpr int THREADS = 32 * (ROW_WARPS + 2);
    static constexpr int ROW_THREADS = 32 * ROW_WARPS;
    static constexpr int CTAS_PER_SM = 2;
    static constexpr int STAGES = 2;
    static constexpr uint32_t TMEM_COLS = 256;
};

struct MiShared {
    uint64_t full[MiCfg::STAGES];
    uint64_t empty[MiCfg::STAGES];
    uint64_t a_ready;    // one arrival per row thread: A tiles written, accumulators read
    uint64_t d_ready[2]; // commit: output half h of the layer complete (every tile)
    uint64_t a_free;     // commit: half 1 has read A columns 0-127 (every tile)
    uint64_t fin;        // commit after the last MMA
    uint32_t tmem_base;
    int abort;
    float2 red[MI_ROWS];     // half 1's share of the output layer
};

constexpr int mi_smem() {
    return 1024 + MI_A_BYTES + MiCfg::STAGES * MLP_TILE_BYTES + MI_F32_BYTES + (int)sizeof(MiShared);
}

// Copy into this CTA's shared memory, completing bytes on `bar` (armed separately).
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// mbar_wait with suspension: same bound (TC_WAIT_NS) and abort protocol.
__device__ __forceinline__ bool mbar_wait_sleep(uint64_t* bar, uint32_t parity, volatile int* abort) {
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait_sleep(bar, parity, 2000u)) return true;
        if (*abort) return false;
        if (global_ns() - t0 > TC_WAIT_NS) {
            *abort = 1;
            return false;
        }
    }
}

// Wait bounded by time only (used on the way out, after an abort).
__device__ __forceinline__ bool mbar_wait_timed(uint64_t* bar, uint32_t parity) {
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > TC_WAIT_NS) return false;
    return true;
}

__device__ __forceinline__ float tanh_f32(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}


__device__ __forceinline__ uint32_t bf16x2_bits(float a, float b) {
    __nv_bfloat162 p = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&p);
}

// silu(z) of two accumulators holding z/2 (bias added here), as BF16x2: FP32
// tanh (measured faster than the packed-FP16 tanh, whose float/half
// conversions cost more than the MUFU op they save, and more accurate).
__device__ __forceinline__ uint32_t silu_pair_bf16(float2 hz) {
    const float2 h = __ffma2_rn(hz, make_float2(tanh_f32(hz.x), tanh_f32(hz.y)), hz);
    return bf16x2_bits(h.x, h.y);
}

// 16-byte unit u (0..7) of row m in A chunk kc
__device__ __forceinline__ uint32_t a_unit(const unsigned char* A, int kc, int m, int u) {
    return smem_u32(A + kc * MLP_TILE_BYTES + (m >> 3) * 1024 + (m & 7) * 128 + ((u ^ (m & 7)) << 4));
}

__device__ __forceinline__ void st_v4(uint32_t addr, const uint32_t* w) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3])
                 : "memory");
}

// Features of row r (if valid) as the layer-0 A row [hi(f), lo(f), hi(f), 0]
// of row m, from positions already in registers.
__device__ __forceinline__ void write_a0(unsigned char* A, int m, const FeatConst& fc, bool valid, double2 ui,
                                         double2 uj) {
    float f[MLP_IN] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (valid) pair_features_dev(fc, ui.x, ui.y, uj.x, uj.y, f);
    float a[32];
#pragma unroll
    for (int e = 0; e < MLP_IN; ++e) {
        const float hi = __bfloat162float(__float2bfloat16_rn(f[e]));
        a[e] = hi;
        a[MLP_IN + e] = f[e] - hi;
        a[2 * MLP_IN + e] = hi;
    }
#pragma unroll
    for (int e = 3 * MLP_IN; e < 32; ++e) a[e] = 0.f;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) w[q] = bf16x2_bits(a[u * 8 + 2 * q], a[u * 8 + 2 * q + 1]);
        st_v4(a_unit(A, 0, m, u), w);
    }
}

// Per-row inputs of one tile, fetched a tile ahead.
struct RowIn {
    bool valid;
    int i, j;
    int64_t g0;       // first entry of the trial's Gram
    double2 ui, uj;   // user positions
    double2 gc;       // closed-form G~_ij (upper triangle)
    double2 gf;       // G~_ij F_ij, the base (conjugate of the lower triangle)
};

template <bool HB>
__device__ __forceinline__ RowIn fetch_row(int64_t r, int64_t rows, int K, int P, const double2* __restrict__ users,
                                           const double2* __restrict__ gram) {
    RowIn in;
    in.valid = r < rows;
    in.i = 0;
    in.j = 1;
    in.g0 = 0;
    in.ui = in.uj = in.gc = in.gf = make_double2(1.0, 0.0);
    if (in.valid) {
        const int64_t b = r / P;
        pair_index((int)(r - b * P), K, in.i, in.j);
        in.ui = users[b * K + in.i];
        in.uj = users[b * K + in.j];
        in.g0 = b * K * K;
        in.gc = gram[in.g0 + in.i * K + in.j];
        if (HB) {
            const double2 lo = gram[in.g0 + in.j * K + in.i];
            in.gf = make_double2(lo.x, -lo.y);
        } else {
            in.gf = in.gc;
        }
    }
    return in;
}

// Persistent: CTA x takes tiles x, x + grid, x + 2 grid, ... (n_iter of them;
// tiles past the end have no valid rows).
// HB: the Gram holds a base G~ F below the diagonal (else the base is G~).
template <bool HB>
__global__ void __launch_bounds__(MiCfg::THREADS, MiCfg::CTAS_PER_SM)
    mlp_infer_tc_kernel(FeatConst fc, const double2* __restrict__ users, int K, int64_t rows, int n_iter,
                        const unsigned char* __restrict__ packed, double2* __restrict__ gram) {
    using C = MiCfg;
    constexpr int MI_STAGES = C::STAGES;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char* A = base;  // the tile's A operand
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
        mbar_init(&sh->a_ready, C::ROW_THREADS);
        mbar_init(&sh->d_ready[0], 1);
        mbar_init(&sh->d_ready[1], 1);
        mbar_init(&sh->a_free, 1);
        mbar_init(&sh->fin, 1);
        sh->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == C::MMA) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh->tmem_base)),
                     "r"(C::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    const float* gpf = reinterpret_cast<const float*>(packed + MLP_PK_F32);
    for (int e = tid; e < MLP_PK_NF; e += C::THREADS) pf[e] = gpf[e];
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh->tmem_base;
    volatile int* abort = &sh->abort;
    const int n_tiles_total = n_iter * MLP_TILES;

    if (warp == C::LOADER) {
        // ---------------- weight tiles through the ring
        if (lane == 0) {
            int armed = 0;
            for (int c = 0; c < n_tiles_total; ++c) {
                const int s = c % MI_STAGES;
                // the previous tile of this slot has landed here before the slot is re-armed
                if (c >= MI_STAGES && !mbar_wait_sleep(&sh->full[s], ((c / MI_STAGES) - 1) & 1, abort)) break;
                expect_tx(&sh->full[s], MLP_TILE_BYTES);
                ++armed;
                // ... and the MMA warp has consumed it before the slot is overwritten
                if (c >= MI_STAGES && !mbar_wait_sleep(&sh->empty[s], ((c / MI_STAGES) - 1) & 1, abort)) break;
                const uint32_t dst = smem_u32(ring + s * MLP_TILE_BYTES);
                const unsigned char* src = packed + (int64_t)(c % MLP_TILES) * MLP_TILE_BYTES;
                bulk_load(dst, src, MLP_TILE_BYTES, &sh->full[s]);
            }
            // no copy may still be landing when the CTA exits
            for (int c = armed - MI_STAGES; c < armed; ++c)
                if (c >= 0) mbar_wait_timed(&sh->full[c % MI_STAGES], (c / MI_STAGES) & 1);
        }
        __syncwarp();
    } else if (warp == C::MMA) {
        // ---------------- MMA issuer: the tile takes each weight tile in turn
        if (lane == 0) {
            const uint32_t idesc = tc_idesc<TCP_BF16>();
            bool ok = true;
            int c = 0;
            for (int it = 0; it < n_iter && ok; ++it) {
                for (int L = 0; L < 4 && ok; ++L) {
                    if (!mbar_wait_sleep(&sh->a_ready, L & 1, abort)) { ok = false; break; }  // 4 phases per tile
                    tc_fence_after();
                    const int nk = L == 0 ? 1 : 4, ksteps = L == 0 ? 2 : 4;
                    for (int nh = 0; nh < 2 && ok; ++nh) {
                        for (int kc = 0; kc < nk; ++kc, ++c) {
                            const int s = c % MI_STAGES;
                            if (!mbar_wait_sleep(&sh->full[s], (c / MI_STAGES) & 1, abort)) { ok = false; break; }
                            tc_fence_after();
                            const uint32_t b0 = smem_u32(ring + s * MLP_TILE_BYTES);
                            const uint32_t a0 = smem_u32(A + kc * MLP_TILE_BYTES);
                            for (int kk = 0; kk < ksteps; ++kk)
                                umma(tmem + nh * 128, desc_sw128(a0 + kk * 32), desc_sw128(b0 + kk * 32), idesc,
                                     (kc | kk) ? 1u : 0u);
                            umma_commit(&sh->empty[s]);
                            if (nh == 1 && kc == (nk - 1) / 2) umma_commit(&sh->a_free);  // chunks 0, 1 read
                        }
                        if (ok) umma_commit(&sh->d_ready[nh]);
                    }
                }
            }
            umma_commit(&sh->fin);  // arrives once every MMA issued above has completed
        }
        __syncwarp();
    } else {
        // ---------------- rows: warp (hf, quarter) = (warp / 4, warp % 4)
        const int m = (warp & 3) * 32 + lane, hf = warp >> 2;
        const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(hf * 128);
        const int64_t tile_rows = MI_ROWS;  // rows per CTA iteration
        const int64_t row_off = m;
        RowIn cur;
        cur.valid = false;
        if (hf == 0) {
            cur = fetch_row<HB>((int64_t)blockIdx.x * tile_rows + row_off, rows, K, P, users, gram);
            write_a0(A, m, fc, cur.valid, cur.ui, cur.uj);
        }
        fence_async_smem();
        mbar_arrive(&sh->a_ready);
        bool ok = true;
        for (int it = 0; it < n_iter; ++it) {
            RowIn nxt;
            nxt.valid = false;
            const bool more = it + 1 < n_iter;
            if (hf == 0 && more)  // loads for the next tile, in flight during this one
                nxt = fetch_row<HB>(((int64_t)blockIdx.x + (int64_t)(it + 1) * gridDim.x) * tile_rows + row_off, rows, K, P,
                                users, gram);
            float2 o = make_float2(0.f, 0.f);
            for (int L = 0; L < 4 && ok; ++L) {
                if (!mbar_wait_sleep(&sh->d_ready[hf], L & 1, abort)) { ok = false; break; }
                tc_fence_after();
                const float* bias = pf + MLP_PK_B0 + L * MLP_W + hf * 128;
                for (int cb = 0; cb < 4; ++cb) {
                    float v[32];
                    tmem_ld32(trow + cb * 32, v);
                    const float4* b4 = reinterpret_cast<const float4*>(bias + cb * 32);
                    if (L < 3) {
                        uint32_t w[16];
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const float4 bb = b4[q];
                            w[2 * q] =
                                silu_pair_bf16(__fadd2_rn(make_float2(v[4 * q], v[4 * q + 1]), make_float2(bb.x, bb.y)));
                            w[2 * q + 1] = silu_pair_bf16(
                                __fadd2_rn(make_float2(v[4 * q + 2], v[4 * q + 3]), make_float2(bb.z, bb.w)));
                        }
                        if (hf == 0 && cb == 0 && !mbar_wait_sleep(&sh->a_free, L & 1, abort)) { ok = false; break; }
                        const int col = hf * 128 + cb * 32;
#pragma unroll
                        for (int u = 0; u < 4; ++u) st_v4(a_unit(A, col >> 6, m, ((col & 63) >> 3) + u), w + 4 * u);
                    } else {
                        const float4* w4 = reinterpret_cast<const float4*>(pf + MLP_PK_W4 + 2 * (hf * 128 + cb * 32));
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            const float2 bb = q & 1 ? make_float2(b4[q >> 1].z, b4[q >> 1].w)
                                                    : make_float2(b4[q >> 1].x, b4[q >> 1].y);
                            const float2 hz = __fadd2_rn(make_float2(v[2 * q], v[2 * q + 1]), bb);
                            const float2 h = __ffma2_rn(hz, make_float2(tanh_f32(hz.x), tanh_f32(hz.y)), hz);
                            const float4 ww = w4[q];  // W4 rows of the two columns
                            o = __ffma2_rn(make_float2(h.x, h.x), make_float2(ww.x, ww.y), o);
                            o = __ffma2_rn(make_float2(h.y, h.y), make_float2(ww.z, ww.w), o);
                        }
                    }
                }
                if (!ok) break;
                if (L < 3) {
                    fence_async_smem();
                    tc_fence_before();
                    mbar_arrive(&sh->a_ready);
                }
            }
            // the accumulator has been read: the next tile's features go in (once
            // half 1 has read A chunk 0 for layer 3), and its layer 0 may start
            if (ok && more) {
                if (hf == 0) {
                    if (mbar_wait_sleep(&sh->a_free, 1, abort)) write_a0(A, m, fc, nxt.valid, nxt.ui, nxt.uj);
                    else ok = false;
                }
                fence_async_smem();
                tc_fence_before();
                if (ok) mbar_arrive(&sh->a_ready);
            }
            if (hf == 1) sh->red[m] = o;
            // barrier of the 256 row threads that also agrees on stopping, so
            // that all of them leave the loop together
            uint32_t stop;
            {
                const uint32_t mine = (!ok || *abort) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred p, 1, %2, q;\n selp.u32 %0, 1, 0, p;\n}\n"
                    : "=r"(stop)
                    : "r"(mine), "n"(C::ROW_THREADS)
                    : "memory");
            }
            if (hf == 0 && cur.valid) {
                const float2 o1 = sh->red[m];
                double2 v0, v1;
                if (!stop) {
                    // G~ F + G~ t
                    const double t0 = (double)(o.x + o1.x + pf[MLP_PK_B4]);
                    const double t1 = (double)(o.y + o1.y + pf[MLP_PK_B4 + 1]);
                    const double2 gc = cur.gc;
                    v0 = make_double2(cur.gf.x + (gc.x * t0 - gc.y * t1), cur.gf.y + (gc.x * t1 + gc.y * t0));
                    v1 = make_double2(v0.x, -v0.y);
                } else {
                    const double nanv = __longlong_as_double(0x7ff8000000000000ULL);
                    v0 = v1 = make_double2(nanv, nanv);
                }
                gram[cur.g0 + cur.i * K + cur.j] = v0;
                gram[cur.g0 + cur.j * K + cur.i] = v1;
            }
            // red[] is rewritten only after the next tile's output layer, which
            // cannot start before half 0 has passed its next epilogues
            cur = nxt;
            if (stop) {
                // the remaining tiles of this CTA are lost: mark them
                for (int k = it + 1; k < n_iter && hf == 0; ++k) {
                    const RowIn q = fetch_row<HB>(((int64_t)blockIdx.x + (int64_t)k * gridDim.x) * tile_rows + row_off, rows,
                                              K, P, users, gram);
                    if (q.valid) {
                        const double nanv = __longlong_as_double(0x7ff8000000000000ULL);
                        gram[q.g0 + q.i * K + q.j] = make_double2(nanv, nanv);
                        gram[q.g0 + q.j * K + q.i] = make_double2(nanv, nanv);
                    }
                }
                break;
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == C::MMA && lane == 0) mbar_wait_timed(&sh->fin, 0);
    __syncwarp();
    if (warp == C::MMA) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS) : "memory");
    }
}

template <bool HB>
static int mlp_infer_launch(const FeatConst& fc, const double* users, int K, int64_t rows, const void* packed,
                            double* gram, cudaStream_t st) {
    using C = MiCfg;
    constexpr int smem = mi_smem();
    static bool done[64] = {false};
    int dev = 0;
    int rc = cuda_status(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc) return rc;
    if (dev >= 64 || !done[dev]) {
        rc = cuda_status(cudaFuncSetAttribute(mlp_infer_tc_kernel<HB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                         "surrogate kernel attribute");
        if (rc) return rc;
        if (dev < 64) done[dev] = true;
    }
    const int64_t n_tiles = (rows + MI_ROWS - 1) / MI_ROWS;
    const int64_t grid = std::min<int64_t>(n_tiles, (int64_t)C::CTAS_PER_SM * num_sms());
    const int64_t n_iter = (n_tiles + grid - 1) / grid;
    if (n_iter * MLP_TILES > 0x7fffffffLL) { set_error("too many pairs for one launch"); return XLMIMO_EINVAL; }
    mlp_infer_tc_kernel<HB><<<(unsigned)grid, C::THREADS, smem, st>>>(fc, (const double2*)users, K, rows, (int)n_iter,
                                                                      (const unsigned char*)packed, (double2*)gram);
    return cuda_status(cudaGetLastError(), "surrogate kernel launch");
}

}  // namespace xl

using namespace xl;

extern "C" int xlmimo_surrogate_gram(const xlmimo_array* arr, const double* users, int K, int B, int base,
                                     const void* packed, double* gram, void* stream) {
    clear_error();
    Geom g;
    int rc = check_array(arr, &g);
    if (rc) return rc;
    if (K < 1 || K > XLMIMO_MAX_USERS || B < 0) { set_error("K must be in [1, 64] and B >= 0"); return XLMIMO_EINVAL; }
    if (base < XLMIMO_APERTURE_NONE || base > XLMIMO_APERTURE_FRESNEL) { set_error("unknown base %d", base); return XLMIMO_EINVAL; }
    if (B == 0) return XLMIMO_OK;
    if (!users || !gram || !packed) { set_error("users, packed and gram must be non-NULL"); return XLMIMO_EINVAL; }
    if (((uintptr_t)packed & 15u) != 0) { set_error("packed must be 16-byte aligned"); return XLMIMO_EINVAL; }
    cudaStream_t st = as_stream(stream);
    rc = launch_closed_form(g, users, K, B, gram, st);
    if (rc || K < 2) return rc;
    // the base G~ F goes into the lower triangle (conjugated); the network's
    // kernel reads G~ above the diagonal and G~ F below, and writes G~ F + G~ t
    if ((rc = launch_aperture_base(g, base, users, K, B, gram, st))) return rc;
    const int64_t rows = (int64_t)B * (K * (K - 1) / 2);
    const FeatConst fc = make_feat_const(g);
    return base != XLMIMO_APERTURE_NONE ? mlp_infer_launch<true>(fc, users, K, rows, packed, gram, st)
                                        : mlp_infer_launch<false>(fc, users, K, rows, packed, gram, st);
}
