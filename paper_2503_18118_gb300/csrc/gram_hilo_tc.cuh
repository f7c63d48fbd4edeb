// Real Gram tiles R = X X^T on the tensor cores for rows stored in HBM as a
// BF16 split X = X_hi + X_lo (the channels of Appendix A's K up to 1000
// users, too many for the generate-in-shared-memory pipeline).
//
// X of trial b is 2Kp rows (Re of users 0 .. Kp-1, then Im) of Np elements,
// K-major (elements contiguous), in two arrays X_hi and X_lo; Kp is a
// multiple of 64 and Np of 64.  One CTA per (128 x 128 tile pair ti >= tj,
// trial): a TMA warp streams the four 128 x 64 tiles (A = rows of block ti,
// B = rows of block tj, hi and lo) of each 64-element stage through a ring of
// GH_NST stages with 128-byte swizzle; one thread issues per 16-element step
// the three tcgen05.mma (M = N = 128) of
//   R_tile += A_hi B_hi^T + A_lo B_hi^T + A_hi B_lo^T
// (X_lo X_lo^T, below 2^-18 relative, is dropped) into one of two TMEM
// accumulators, switching every GH_PER stages; four warps add each finished
// accumulator into a running FP32 total in TMEM (round to nearest) while the
// other one fills, and write the tile (FP32, row-major 2Kp x 2Kp per trial)
// after the last.  The FP32 accumulation of the tensor cores rounds towards
// zero; the per-period totals bound that bias by GH_PER stages.  Every wait
// is bounded; a CTA that gives up writes NaN to its tile.
#pragma once

#include <cuda.h>

#include "gen_tc.cuh"

namespace xl {

constexpr int GH_TILE = 128;                          // rows of A and B per tile
constexpr int GH_BK = 64;                             // elements per stage: one 128-byte swizzle atom of BF16
constexpr int GH_TILE_BYTES = GH_TILE * GH_BK * 2;    // 16 KB
constexpr int GH_STAGE_BYTES = 4 * GH_TILE_BYTES;     // A_hi, A_lo, B_hi, B_lo
constexpr int GH_NST = 3;
constexpr int GH_PER = 4;  // stages per accumulation period: 4 x 4 steps x 3 MMAs = 48 accumulations
constexpr int GH_THREADS = 192;  // warp 0 TMA, warp 1 MMA, warps 2-5 drain and epilogue

struct GhShared {
    uint64_t full[GH_NST];
    uint64_t empty[GH_NST];
    uint64_t wfull[2];  // commit: a period's MMAs into accumulator w are complete
    uint64_t wfree[2];  // 128 arrivals: accumulator w added into the total
    uint64_t done;      // commit: every MMA the thread issued is complete
    uint32_t tmem_base;
    int abort;
};

constexpr size_t gh_smem_bytes() { return 1024 + (size_t)GH_NST * GH_STAGE_BYTES + sizeof(GhShared); }

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Wait bounded by time only (on the way out, after an abort).
__device__ __forceinline__ bool gh_wait_timed(uint64_t* bar, uint32_t parity) {
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > TC_WAIT_NS) return false;
    return true;
}

// R[b] (2Kp x 2Kp FP32, row-major; tiles ti >= tj written) of X_hi, X_lo
// described by the two tensor maps (dims {Np, 2Kp, B}, box {64, 128, 1}).
__global__ void __launch_bounds__(GH_THREADS, 1)
    gram_hilo_kernel(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo, int Np,
                     int Kp, float* __restrict__ R) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    GhShared* sh = reinterpret_cast<GhShared*>(base + GH_NST * GH_STAGE_BYTES);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int b = blockIdx.y;
    int ti, tj;
    tri_index(blockIdx.x, &ti, &tj);
    const int nk = Np / GH_BK;
    const int nper = (nk + GH_PER - 1) / GH_PER;
    volatile int* abort = &sh->abort;

    if (tid == 0) {
        for (int i = 0; i < GH_NST; ++i) {
            mbar_init(&sh->full[i], 1);
            mbar_init(&sh->empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&sh->wfull[i], 1);
            mbar_init(&sh->wfree[i], 128);
        }
        mbar_init(&sh->done, 1);
        sh->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh->tmem_base)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh->tmem_base;  // W0: columns 0-127, W1: 128-255, total: 256-383
    const uint32_t sbase = smem_u32(base);

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            int issued = 0;
            for (int s = 0; s < nk; ++s) {
                const int slot = s % GH_NST;
                if (s >= GH_NST && !mbar_wait(&sh->empty[slot], (uint32_t)((s / GH_NST - 1) & 1), abort)) break;
                const uint32_t st = sbase + (uint32_t)slot * GH_STAGE_BYTES;
                arrive_expect_tx(&sh->full[slot], GH_STAGE_BYTES);
                const int x = s * GH_BK;
                tma_load_3d(st, &map_hi, x, ti * GH_TILE, b, &sh->full[slot]);
                tma_load_3d(st + GH_TILE_BYTES, &map_lo, x, ti * GH_TILE, b, &sh->full[slot]);
                tma_load_3d(st + 2 * GH_TILE_BYTES, &map_hi, x, tj * GH_TILE, b, &sh->full[slot]);
                tma_load_3d(st + 3 * GH_TILE_BYTES, &map_lo, x, tj * GH_TILE, b, &sh->full[slot]);
                ++issued;
            }
            // no copy may still be landing when the CTA exits
            for (int s = issued - GH_NST; s < issued; ++s)
                if (s >= 0) gh_wait_timed(&sh->full[s % GH_NST], (uint32_t)((s / GH_NST) & 1));
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = tc_idesc<TCP_BF16X3, 128u>();
            for (int s = 0; s < nk; ++s) {
                const int slot = s % GH_NST;
                if (!mbar_wait(&sh->full[slot], (uint32_t)((s / GH_NST) & 1), abort)) break;
                const int p = s / GH_PER, w = p & 1;
                const bool first = s % GH_PER == 0;
                // accumulator w was last used by period p - 2: its total must be taken
                if (first && p >= 2 && !mbar_wait(&sh->wfree[w], (uint32_t)(((p - 2) >> 1) & 1), abort)) break;
                tc_fence_after();
                const uint32_t st = sbase + (uint32_t)slot * GH_STAGE_BYTES;
                const uint32_t d = tmem + (uint32_t)(w * 128);
#pragma unroll
                for (int kk = 0; kk < GH_BK / 16; ++kk) {
                    const uint64_t ahi = desc_sw128(st + kk * 32), alo = desc_sw128(st + GH_TILE_BYTES + kk * 32);
                    const uint64_t bhi = desc_sw128(st + 2 * GH_TILE_BYTES + kk * 32);
                    const uint64_t blo = desc_sw128(st + 3 * GH_TILE_BYTES + kk * 32);
                    umma(d, ahi, bhi, idesc, (first && kk == 0) ? 0u : 1u);
                    umma(d, alo, bhi, idesc, 1u);
                    umma(d, ahi, blo, idesc, 1u);
                }
                umma_commit(&sh->empty[slot]);
                if (s % GH_PER == GH_PER - 1 || s == nk - 1) umma_commit(&sh->wfull[w]);
            }
            umma_commit(&sh->done);
            gh_wait_timed(&sh->done, 0);  // nothing in flight once the tensor memory is released
        }
        __syncwarp();
    } else {
        // ---------------- drain and epilogue: warps 2-5 own TMEM lane quarters 2, 3, 0, 1
        const int q = warp & 3;
        const uint32_t lrow = (uint32_t)(q * 32) << 16;
        const int row = ti * GH_TILE + q * 32 + lane;  // row of R
        float* out = R + ((int64_t)b * 2 * Kp + row) * (2 * Kp) + tj * GH_TILE;
        bool ok = true;
        for (int p = 0; p < nper; ++p) {
            const int w = p & 1;
            if (!mbar_wait(&sh->wfull[w], (uint32_t)((p >> 1) & 1), abort)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const bool last = p == nper - 1;
#pragma unroll 1
            for (int c = 0; c < GH_TILE; c += 16) {
                uint32_t a[16], t[16];
                tmem_ld16(tmem + lrow + (uint32_t)(w * 128 + c), a);
                if (p > 0) tmem_ld16(tmem + lrow + (uint32_t)(256 + c), t);
                tmem_wait_ld();
                if (p > 0) {
#pragma unroll
                    for (int j = 0; j < 16; j += 2) {
                        const float2 s2 = __fadd2_rn(make_float2(__uint_as_float(a[j]), __uint_as_float(a[j + 1])),
                                                     make_float2(__uint_as_float(t[j]), __uint_as_float(t[j + 1])));
                        a[j] = __float_as_uint(s2.x);
                        a[j + 1] = __float_as_uint(s2.y);
                    }
                }
                if (last) {
#pragma unroll
                    for (int j = 0; j < 16; j += 4)
                        *reinterpret_cast<float4*>(out + c + j) =
                            make_float4(__uint_as_float(a[j]), __uint_as_float(a[j + 1]), __uint_as_float(a[j + 2]),
                                        __uint_as_float(a[j + 3]));
                } else {
                    tmem_st16(tmem + lrow + (uint32_t)(256 + c), a);
                }
            }
            if (!last) {
                tmem_wait_st();
                tc_fence_before();
                mbar_arrive(&sh->wfree[w]);
            }
        }
        if (!ok || *abort) {
            const float nanv = __int_as_float(0x7fc00000);
            for (int c = 0; c < GH_TILE; c += 4) *reinterpret_cast<float4*>(out + c) = make_float4(nanv, nanv, nanv, nanv);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

}  // namespace xl
