// tcgen05 building blocks shared by the tensor-core Gram kernels: stage
// layout, mbarrier and TMEM helpers, descriptors, the 16-bit hi/lo split.
// See gram_tc.cu for the method.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "chan_gen.cuh"
#include "common.cuh"

namespace xl {

constexpr int TC_STAGES = 3;
constexpr int TC_T = 64;              // elements per stage
constexpr int TC_THREADS = 288;
constexpr int TC_GEN_THREADS = 256;
constexpr int TC_REF_SPAN = 256;      // elements per phase reference (4 stages)
constexpr uint64_t TC_WAIT_NS = 4000000000ull;  // 4 s

enum { TCP_BF16 = 0, TCP_BF16X3 = 1, TCP_F16X3 = 2 };

template <int KMAX>
struct TcCfg {
    static constexpr int ROWS = 4 * KMAX;                   // hi and lo rows of Re and Im
    static constexpr int STAGE_BYTES = ROWS * TC_T * 2;     // 16-bit entries
    static constexpr int LO_OFFSET = 2 * KMAX * 128;        // bytes to the lo block
    static constexpr int SLOTS = KMAX / 32;                 // users per generator lane
    static constexpr int FOLD_LD = KMAX == 32 ? 65 : 129;   // epilogue row stride (floats)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ uint32_t mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok;
}

// try_wait that lets the hardware suspend the thread for up to `ns` while the
// phase is incomplete, so that waiting warps give their issue slots to the
// working ones (measured: 1.8 % faster Gram kernel than polling).
__device__ __forceinline__ uint32_t mbar_try_wait_sleep(uint64_t* bar, uint32_t parity, uint32_t ns) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for the phase with the given parity.  Every wait in this
// kernel is a per-stage hand-off (microseconds); after TC_WAIT_NS of wall
// time, or once another thread has aborted, it gives up, sets *abort and
// returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
    if (mbar_try_wait(bar, parity)) return true;  // usual case: no timer read
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait_sleep(bar, parity, 1000u)) return true;
        if ((it & 63u) == 63u) {
            if (*abort) return false;
            if (global_ns() - t0 > TC_WAIT_NS) {
                *abort = 1;
                return false;
            }
        }
    }
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// SMEM matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;              // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
    d |= (uint64_t)1 << 46;              // descriptor version
    d |= (uint64_t)2 << 61;              // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: 16-bit A and B (format 1 = BF16, 0 = F16),
// FP32 accumulator, both K-major, M = 128, N = 128 or 64.
template <int PREC, uint32_t N = 128>
__device__ __forceinline__ uint32_t tc_idesc() {
    const uint32_t fmt = PREC == TCP_F16X3 ? 0u : 1u;
    return (1u << 4)               // D format F32
           | (fmt << 7)            // A format
           | (fmt << 10)           // B format
           | ((N >> 3) << 17)      // N / 8
           | ((128u >> 4) << 24);  // M / 16
}

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                     uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// hi/lo (or hi only) 16-bit conversion of two values, packed.  TRUNC (BF16
// hi/lo only): hi by truncation (one byte permute packs both), lo the exact
// remainder rounded; otherwise hi is rounded to nearest, whose remainder is
// a quarter as large in square (what a product that drops lo*lo gives up).
template <int PREC, bool TRUNC = false>
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
    if (PREC == TCP_F16X3) {
        __half2 h = __floats2half2_rn(a, b);
        float2 hf = __half22float2(h);
        __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
        hi = *reinterpret_cast<uint32_t*>(&h);
        lo = *reinterpret_cast<uint32_t*>(&l);
    } else if (PREC == TCP_BF16X3 && TRUNC) {
        // hi = the upper 16 bits of each float (truncation: one byte permute
        // packs both), lo = the exact remainder rounded to BF16; |lo| < 2^-7 |x|,
        // so hi + lo carries x to ~2^-16 relative
        const uint32_t xa = __float_as_uint(a), xb = __float_as_uint(b);
        hi = __byte_perm(xa, xb, 0x7632);
        const float2 r = __fadd2_rn(make_float2(a, b), make_float2(-__uint_as_float(xa & 0xFFFF0000u),
                                                                    -__uint_as_float(xb & 0xFFFF0000u)));
        __nv_bfloat162 l = __floats2bfloat162_rn(r.x, r.y);
        lo = *reinterpret_cast<uint32_t*>(&l);
    } else {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        hi = *reinterpret_cast<uint32_t*>(&h);
        if (PREC == TCP_BF16X3) {
            // exact remainders a - hi, b - hi in one packed FMA
            const float2 hf = __bfloat1622float2(h);
            const float2 r = __fadd2_rn(make_float2(a, b), make_float2(-hf.x, -hf.y));
            __nv_bfloat162 l = __floats2bfloat162_rn(r.x, r.y);
            lo = *reinterpret_cast<uint32_t*>(&l);
        } else {
            lo = 0u;
        }
    }
}

}  // namespace xl
