// The exact-Gram pipeline of one CTA on the 5th-generation tensor cores
// (tcgen05), shared by the one-launch-per-batch kernel (gram_tc.cu) and the
// persistent ragged-batch kernel (batched.cu).
//
// The complex Gram G = H^H H of K users is a real contraction over the
// elements: with X = [Re H ; Im H] (2K rows, one column per element),
//   Re G_ij = (X X^T)_{i,j} + (X X^T)_{K+i,K+j},  Im G_ij = (X X^T)_{i,K+j} - (X X^T)_{K+i,j}.
// Each FP32 channel entry is split v = hi + lo in BF16 (|v - hi - lo| <=
// 2^-16 |v|) or, after scaling user k's entries by s_k = 1/|h_k| at the
// array centre so that they sit near 1, in FP16 (<= 2^-22 |v|; the scale is
// divided out in FP64 at the end).  Two layouts:
//   narrow (K <= 32): Y = [X_hi ; X_lo] has 128 rows and M = 128, N = 64 MMAs
//            accumulate D = Y X_hi^T = [P ; Q], P = X_hi X_hi^T, Q = X_lo X_hi^T,
//            so that X X^T = P + Q + Q^T up to X_lo X_lo^T (below 2^-18
//            relative with the round-to-nearest hi).  Stages of 128 elements
//            (two 64-element sub-tiles).
//   wide (K <= 64): X_hi and X_lo have 128 rows each; two M = N = 128 MMAs
//            per k-step accumulate D = X_hi X_hi^T + (2 X_lo) X_hi^T = P + 2Q
//            (the lo tile holds 2 X_lo, an exponent increment), and
//            X X^T = (D + D^T) / 2.  Stages of 64 elements.
// The single-term BF16 variant keeps X_hi only.  Channel entries come from
// the slice expansion of gen_tc.cuh, or, for an item with a user closer than
// NEAR_DIST, from the exact per-entry formula of chan_gen.cuh.
//
// Roles (9 warps):
//   warps 0-7  generate ring stages: lane = user, warp = one 8-element slice
//              per 64-element sub-tile; each thread writes 8-byte halves of
//              the 16-byte rows of the K-major, 128-byte-swizzled 16-bit
//              tile, fences the async proxy and arrives on the stage's "full"
//              barrier.  They also drain the accumulator (below);
//   warp 8     one thread waits for each full stage, issues the K = 16
//              tcgen05.mma of its sub-tiles into the working accumulator W
//              and commits to the stage's "empty" barrier (generators reuse
//              the stage once it fires) and, at the end of an item, to "done";
//   warps 0-3  read the accumulators back (tcgen05.ld), fold the blocks and
//              write the complex Gram in FP64.
// Periodic drain (gen_tc.cuh): every DRAIN stages the MMA thread commits to
// "wfull"; at the start of the stage after next the generators add W into
// the running total T (tcgen05.ld / FP32 add / tcgen05.st) and arrive on
// "wfree", which the MMA thread awaits before it starts the next period in W
// afresh.  The final period stays in W; the epilogue adds W and T.
// Ring slots and barrier phases are indexed by counters that run on across
// the items of a persistent CTA (gs: stages, gd: drains, items done).
// Every wait is bounded; a wait that gives up sets the CTA's abort flag, the
// item is written as NaN, and outstanding MMAs drain before exit.
#pragma once

#include <math.h>

#include <type_traits>

#include "gen_tc.cuh"

namespace xl {

// URA mode (uniform rectangular array, users in the plane z = 0): a trial's
// elements are its ceil(R/2) mirrored row pairs one after another, ncol per
// row, ncol a multiple of URA_SPAN so that no reference span crosses a row.
// Row q, at height z_q = (q + zoff) spacing, sees user (x, y) as the ULA sees
// (x', y), x' = sqrt(x^2 + z_q^2): each span takes its phase reference and
// distances from x'.  The amplitude constant stays the true user's (PNUSW
// projects on the array normal: sqrt(beta0 x) r^{-3/2}) in the FP64 factor,
// which also carries the factor 2 of the mirrored pair; the centre row of an
// odd R (counted once) is generated with amplitude 1/sqrt(2).
struct UraRows {
    long long ncol;  // elements per row (0: ULA mode)
    double zoff;     // 0 for odd R, 1/2 for even R
    double spacing;
    int odd;
};
constexpr int URA_SPAN = 128;

// Span constants in flight: the span being generated, the one being made
// and up to two spans of warps that lag behind (a warp can run at most
// NRING - 1 stages ahead of the slowest, and a span is at least one stage).
constexpr int NREF = 4;

// Shared state of the pipeline for up to KCAP users and an NRING-stage ring.
template <int KCAP, int NRING>
struct EngShared {
    uint64_t full[NRING];
    uint64_t empty[NRING];
    uint64_t done;
    uint64_t wfull;  // commit: the period's MMAs into W are complete
    uint64_t wfree;  // 256 arrivals: W added into T
    uint32_t tmem_base;
    int abort;
    int bad;
    int near;          // a user too close for the slice expansion
    int item;          // persistent kernels: the current work item
    UserGeo ug[KCAP];
    double fac[KCAP];  // per-user factor of the Gram: G_ij = fac_i fac_j (accumulated sum)
    double ux[KCAP];   // URA: the users' true x
    uint64_t refok[NREF];     // one arrival: the span constants of a ring slot are written
    float4 sref_a[NREF][KCAP];  // span constants (SpanC, first half) of a ring of spans
    float4 sref_b[NREF][KCAP];  // (second half)
};

template <int KCAP, int NRING>
__device__ __forceinline__ void eng_init_barriers(EngShared<KCAP, NRING>* sh) {
    for (int i = 0; i < NRING; ++i) {
        mbar_init(&sh->full[i], TC_GEN_THREADS);
        mbar_init(&sh->empty[i], 1);
    }
    mbar_init(&sh->done, 1);
    mbar_init(&sh->wfull, 1);
    mbar_init(&sh->wfree, TC_GEN_THREADS);
    for (int i = 0; i < NREF; ++i) mbar_init(&sh->refok[i], 1);
    sh->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ SpanC span_c_of(float4 a, float4 b) {
    SpanC s;
    s.frac0 = a.x;
    s.ah = a.y;
    s.al = a.z;
    s.e0 = a.w;
    s.r0 = b.x;
    s.kx = b.y;
    s.xl2 = b.z;
    s.aw = b.w;
    return s;
}

// Exact per-entry generator constants from the span constants (the fallback
// for users too close for the slice expansion).
__device__ __forceinline__ PairConst pair_const_of(const SpanC& s, float dprime) {
    PairConst c;
    c.frac0 = s.frac0;
    c.ah = s.ah;
    c.al = s.al;
    c.af = f2(__fadd_rn(s.ah, s.al));
    c.e0 = f2(s.e0);
    c.r0 = f2(s.r0);
    c.xl2 = f2(s.xl2);
    c.kx = f2(s.kx);
    c.dp = f2(dprime);
    c.ampc = f2(s.aw);
    return c;
}

// Entries 4h .. 4h + 3 of one 8-element slice by the exact per-entry
// formula, as words w[comp][q].
template <int MODEL, int PREC, bool TRUNC>
__device__ __forceinline__ void exact_slice_words(const PairConst& pc, float mfs, int h, int rs, uint32_t (&w)[4][2]) {
    const float base = slice_base(pc, mfs + 3.5f);  // phase at the slice centre
    const float dp = pc.dp.x, u0 = mfs * dp;         // u = m spacing/lambda
    const float fh = (float)(4 * h);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int i = 4 * h + 2 * q;
        const float fi = fh + (float)(2 * q);
        float2 re, im;
        gen_pair<MODEL, false>(pc, make_float2(fmaf(fi, dp, u0), fmaf(fi + 1.0f, dp, u0)),
                               make_float2(fi - 3.5f, fi - 2.5f), base, re, im);
        if (i >= rs) { re.x = 0.f; im.x = 0.f; }
        if (i + 1 >= rs) { re.y = 0.f; im.y = 0.f; }
        split2<PREC, TRUNC>(re.x, re.y, w[0][q], w[2][q]);
        split2<PREC, TRUNC>(im.x, im.y, w[1][q], w[3][q]);
    }
}

// One user's set-up: geometry, factor of the Gram (G_ij = fac_i fac_j times
// the accumulated sum) and the amplitude weight of its generated entries
// (ug.ampc; 0 for padding); bad: an invalid position; near: too close to the
// array for the slice expansion.
struct UserSetup {
    UserGeo ug;
    double fac;
    int bad, near;
};

template <int MODEL, int PREC, bool URA>
__device__ __forceinline__ UserSetup user_setup(const Geom& g, const GenParams& gp, double x, double y, bool valid) {
    UserSetup s;
    s.ug = make_user_geo(g, x, y);
    s.bad = valid && !s.ug.ok;
    s.near = valid && !(x * g.inv_lambda >= (double)NEAR_DIST * (double)gp.dprime_f);
    // the BF16 paths generate entries without the amplitude constant and
    // apply it to the Gram in FP64; the FP16 path scales user k's entries by
    // 1/|h_k| at the array centre so that they sit near 1, and divides it out
    double fac = amp_const(g, x, y);
    float aw = 1.0f;
    if (URA) fac *= 1.4142135623730951;  // fac_i fac_j carries the 2 of a mirrored row pair
    if (PREC == TCP_F16X3) {
        const double rc = sqrt(x * x + y * y) * g.inv_lambda;  // distance in wavelengths
        double amp_c = (MODEL == XLMIMO_UPW) ? fac : (MODEL == XLMIMO_PNUSW) ? fac / (rc * sqrt(rc)) : fac / rc;
        const float sc = (float)(1.0 / amp_c);
        aw = (float)(fac * (double)sc);  // entries c s_k / r^p ~ 1, c the model's constant
        fac = 1.0 / (double)sc;
    }
    s.ug.ampc = valid ? aw : 0.f;
    s.fac = fac;
    return s;
}

template <int MODEL, int KMAX, int PREC, bool URA, int NRING>
struct GramEngine {
    using C = TcCfg<KMAX>;
    static constexpr int KM = KMAX;
    static constexpr int SUBS = KMAX == 32 ? 2 : 1;
    static constexpr int T = TC_T * SUBS;                                // elements per stage
    static constexpr uint32_t BYTES = (uint32_t)C::STAGE_BYTES * SUBS;  // per ring stage (32 KB)
    static constexpr int WCOLS = KMAX == 32 ? 64 : 128;                 // accumulator columns
    // stages per accumulation period: 64 MMA accumulations into W (narrow:
    // 8 per stage; wide: 2 x 4 per stage).  Measured at the headline: a
    // period of 32 accumulations costs 1.7 % more time for a bias of
    // ~2e-6 instead of ~4e-6.
    static constexpr int DRAIN = 8;
    // both layouts drop X_lo X_lo^T, so hi is rounded to nearest (a remainder
    // below 2^-9 relative; a truncated hi leaves up to 2^-7, and the dropped
    // term then biased the diagonal by -1.2e-5)
    static constexpr bool TRUNC = false;
    static constexpr bool LO2 = KMAX == 64;
    static constexpr int SPAN = URA ? URA_SPAN : TC_REF_SPAN;
    static constexpr int SPAN_ST = SPAN / T;  // stages per reference span
    static constexpr int NCOMP = (PREC == TCP_BF16 && KMAX == 64) ? 2 : 4;  // the one-term wide MMA reads hi only

    static __device__ __forceinline__ int stages(int64_t nbeg, int64_t nend) { return (int)((nend - nbeg + T - 1) / T); }
    static __device__ __forceinline__ int drains(int nst) { return (nst - 1) / DRAIN; }
    static __device__ __forceinline__ int spans(int nst) { return (nst + SPAN_ST - 1) / SPAN_ST; }

    // Threads tid < KMAX: user tid of the item (users [K][2] doubles): its
    // geometry, Gram factor and amplitude weight; flags invalid positions
    // (bad) and users too close for the slice expansion (near).  Users K ..
    // KMAX - 1 are padding at (1, 0) with weight 0.
    template <class SH>
    static __device__ __forceinline__ void setup_user(SH* sh, const Geom& g, const GenParams& gp, const double* users, int K, int tid) {
        const bool valid = tid < K;
        const double x = valid ? users[tid * 2] : 1.0, y = valid ? users[tid * 2 + 1] : 0.0;
        const UserSetup u = user_setup<MODEL, PREC, URA>(g, gp, x, y, valid);
        if (u.bad) atomicOr(&sh->bad, 1);
        if (u.near) atomicOr(&sh->near, 1);
        if (URA) sh->ux[tid] = x;
        sh->ug[tid] = u.ug;
        sh->fac[tid] = u.fac;
    }

    // Generator warps 0-7 over the item's elements [nbeg, nend).  gs0 / gd0:
    // stages and drains of the CTA before this item.  Returns true if a wait
    // gave up.  PACKED: the user slots belong to instances of their own; slot
    // k's elements are lane_n0[k] + [0, lane_len[k]) (the stages cover the
    // longest, shorter slots generate zeros past their end), nbeg = 0 and
    // nend = the longest length.
    template <class SH, bool PACKED = false>
    static __device__ __forceinline__ bool generate(SH* sh, uint32_t sbase, uint32_t tmem, const Geom& g, const GenParams& gp,
                                    int64_t nbeg, int64_t nend, const UraRows& ura, int gs0, int gd0, int gsp0,
                                    bool fast, const long long* lane_n0 = nullptr, const int* lane_len = nullptr) {
        static_assert(!PACKED || !URA, "packed user slots: ULA only");
        // the thread's coordinates read afresh (an opaque read): in a
        // persistent kernel the values derived from them below are then made
        // per item instead of being hoisted across the whole item loop, where
        // they would stay live through the epilogue and spill
        uint32_t tidx;
        asm volatile("mov.u32 %0, %%tid.x;" : "=r"(tidx));
        const int warp = (int)(tidx >> 5), lane = (int)(tidx & 31u);
        volatile int* abort = &sh->abort;
        const int nst = stages(nbeg, nend);
        const int ndrain = drains(nst);
        // The double-float phase references of a span (SPAN elements) are
        // made once per CTA: at the start of span sp, warp (sp + 1) % 8
        // prepares span sp + 1 into the next slot of a ring of NREF spans and
        // arrives on the slot's barrier, which every warp awaits at the start
        // of that span.  Warps do not wait for one another otherwise (the
        // stage ring bounds how far they drift apart).  gsp0: spans of the CTA
        // before this item (slots and phases run on across items).
        const int nsp = (nst + SPAN_ST - 1) / SPAN_ST;
        auto make_refs = [&](int sp) {
            const int slot = (gsp0 + sp) % NREF;
            const long long m0 = (long long)(nbeg + (int64_t)sp * SPAN);
            if (URA) {
                const long long q = m0 / ura.ncol;
                const long long ncs = m0 - q * ura.ncol + SPAN / 2;  // span centre, column index in the row
                const double z = ((double)q + ura.zoff) * ura.spacing;
                const float roww = (ura.odd && q == 0) ? 0.70710678118654752f : 1.0f;
                for (int kk = lane; kk < KMAX; kk += 32) {
                    // the spherical-wave reference reads y, x^2 and 2 (x/lambda)^2 only:
                    // the user's own geometry with x'^2 = x^2 + z^2 in their place
                    const double x = sh->ux[kk];
                    const double x2 = fma(x, x, z * z);
                    const double xl2 = x2 * (g.inv_lambda * g.inv_lambda);
                    UserGeo ug = sh->ug[kk];
                    ug.x2 = ff_from_double(x2);
                    ug.xl2 = (float)xl2;
                    ug.x2x2 = (float)(2.0 * xl2);
                    const SpanC c = make_span_c(make_user_ref(gp, ug, ncs), ug.xl2, ug.ampc * roww);
                    sh->sref_a[slot][kk] = make_float4(c.frac0, c.ah, c.al, c.e0);
                    sh->sref_b[slot][kk] = make_float4(c.r0, c.kx, c.xl2, c.aw);
                }
            } else {
                for (int kk = lane; kk < KMAX; kk += 32) {
                    const long long ncs = (PACKED ? lane_n0[kk] + (long long)sp * SPAN : m0) + SPAN / 2;
                    const UserGeo& ug = sh->ug[kk];
                    const SpanC c = make_span_c(make_user_ref(gp, ug, ncs), ug.xl2, ug.ampc);
                    sh->sref_a[slot][kk] = make_float4(c.frac0, c.ah, c.al, c.e0);
                    sh->sref_b[slot][kk] = make_float4(c.r0, c.kx, c.xl2, c.aw);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh->refok[slot]);
        };
        if (warp == 0 && nsp > 0) make_refs(0);
        // stage-tile offset of this lane's component-0 row, lane 0 and lane 1
        // of the packed arithmetic (narrow: sub-tiles 0 and 1 of user `lane`;
        // wide: users lane and lane + 32); component c sits KMAX * c rows on
        const int rin = lane & 7;
        const uint32_t soff0 = (uint32_t)((lane >> 3) * 1024 + rin * 128 + ((warp ^ rin) << 4));
        const uint32_t soff1 = KMAX == 32 ? soff0 + (uint32_t)C::STAGE_BYTES : soff0 + 4u * 1024u;
        // drain: this warp's lane quarter and half of W's columns
        const uint32_t tq = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((warp >> 2) * (WCOLS / 2));
        int drained = 0;
        // T += W of period `drained` (returns false if the wait gave up)
        auto drain = [&]() -> bool {
            const bool ok = mbar_wait(&sh->wfull, (uint32_t)((gd0 + drained) & 1), abort);
            if (ok) {
                tc_fence_after();
                drain_cols<WCOLS / 2>(tq, tq + WCOLS, drained == 0);
                tc_fence_before();
                mbar_arrive(&sh->wfree);
            }
            ++drained;
            return ok;
        };
        // stage bookkeeping kept incremental: ring slot st and its wrap count,
        // this warp's slice offset from the span centre (mf0, an exact small
        // integer in FP32), valid elements of the last stage
        const int last_rem = (int)(nend - nbeg - (int64_t)(nst - 1) * T) - warp * 8;
        const float dp = gp.dprime_f;
        // the stage loop, with the slice expansion (FAST) or the exact
        // per-entry formula; CTA-uniform, so each loop keeps its own
        // registers.  Returns whether a wait gave up.
        // packed: the lengths of this thread's user slots (slot lane, and lane + 32 wide)
        const int len0 = PACKED ? lane_len[lane] : 0;
        const int len1 = PACKED && KMAX == 64 ? lane_len[lane + 32] : 0;
        auto gen_loop = [&](auto fast_tag) -> bool {
            constexpr bool FAST = decltype(fast_tag)::value;
            bool dead = false;
            int st = gs0 % NRING;
            int wraps = gs0 / NRING;
            float mf0 = 0.f;
            int rslot = gsp0 % NREF;  // ring slot of the current span's constants
            for (int it = 0; it < nst; ++it) {
                const int sp = it / SPAN_ST;
                if (it % SPAN_ST == 0) {
                    if (dead || *abort) {
                        dead = true;
                        break;
                    }
                    if (sp > 0 && ++rslot == NREF) rslot = 0;
                    mf0 = (float)(warp * 8 - SPAN / 2);
                    if (warp == ((sp + 1) & 7) && sp + 1 < nsp) make_refs(sp + 1);
                    if (!mbar_wait(&sh->refok[rslot], (uint32_t)(((gsp0 + sp) / NREF) & 1), abort)) {
                        dead = true;
                        break;
                    }
                } else {
                    mf0 += (float)T;
                }
                // the period that ended two stages ago goes into T
                if (it >= DRAIN + 1 && (it - 1) % DRAIN == 0 && !dead && !drain()) dead = true;
                const int cur = st;
                const int wcur = wraps;
                if (++st == NRING) { st = 0; ++wraps; }
                if (dead) continue;
                if (wcur > 0 && !mbar_wait(&sh->empty[cur], (uint32_t)((wcur - 1) & 1), abort)) {
                    dead = true;
                    continue;
                }
                const int rem = it == nst - 1 ? last_rem : T;  // valid elements from this warp's first slice on
                const uint32_t sb = sbase + (uint32_t)cur * BYTES;
                int rem0 = rem, rem1 = KMAX == 32 ? rem - TC_T : rem;
                if (PACKED) {
                    // slot k's elements from this warp's first slice of the stage on
                    // (item lengths below 2^31)
                    const int e0 = len0 - it * T;
                    rem0 = e0 >= T ? T : max(e0, -T) - warp * 8;
                    if (KMAX == 64) {
                        const int e1 = len1 - it * T;
                        rem1 = e1 >= T ? T : max(e1, -T) - warp * 8;
                    } else {
                        rem1 = rem0 - TC_T;
                    }
                }
                const int k1 = KMAX == 32 ? lane : lane + 32;
                SliceCo co;
                if (FAST)
                    co = slice_co<MODEL>(span_c_of(sh->sref_a[rslot][lane], sh->sref_b[rslot][lane]),
                                         span_c_of(sh->sref_a[rslot][k1], sh->sref_b[rslot][k1]),
                                         KMAX == 32 ? make_float2(mf0 + 3.5f, mf0 + (float)(TC_T + 3.5)) : f2(mf0 + 3.5f), dp);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    // lanes 8-15 and 24-31 take the other half of the slice in each
                    // pass, so that one 8-byte store of the warp fills all 32 banks
                    const int hs = h ^ ((lane >> 3) & 1);
                    uint32_t w[2][4][2];
                    if (FAST) {
                        // packed lanes end at different elements: one warp-wide choice, the
                        // partial form zeroing each lane's entries past its own end
                        const bool full = PACKED ? __all_sync(0xffffffffu, rem0 >= 8 && rem1 >= 8) : (rem0 >= 8 && rem1 >= 8);
                        if (full) slice_words<MODEL, PREC, TRUNC, LO2, false>(co, hs, 8, 8, w);
                        else slice_words<MODEL, PREC, TRUNC, LO2, true>(co, hs, rem0, rem1, w);
                    } else {
#pragma unroll
                        for (int l = 0; l < 2; ++l) {
                            const int kl = l == 0 ? lane : k1;
                            exact_slice_words<MODEL, PREC, TRUNC>(
                                pair_const_of(span_c_of(sh->sref_a[rslot][kl], sh->sref_b[rslot][kl]), dp),
                                KMAX == 32 ? mf0 + (float)(TC_T * l) : mf0, hs, l == 0 ? rem0 : rem1, w[l]);
                            if (LO2 && PREC != TCP_BF16) {
#pragma unroll
                                for (int q = 0; q < 2; ++q) {
                                    w[l][2][q] = double_halves<PREC>(w[l][2][q]);
                                    w[l][3][q] = double_halves<PREC>(w[l][3][q]);
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int c = 0; c < NCOMP; ++c) {
                        const uint32_t off = (uint32_t)(c * KMAX * 128 + 8 * hs);
                        asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(sb + soff0 + off), "r"(w[0][c][0]),
                                     "r"(w[0][c][1])
                                     : "memory");
                        asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(sb + soff1 + off), "r"(w[1][c][0]),
                                     "r"(w[1][c][1])
                                     : "memory");
                    }
                }
                fence_async_smem();
                mbar_arrive(&sh->full[cur]);
            }
            return dead;
        };
        bool dead = fast ? gen_loop(std::true_type()) : gen_loop(std::false_type());
        // a period whose drain point lies past the last stage
        while (drained < ndrain && !dead)
            if (!drain()) dead = true;
        return dead;
    }

    // The MMA thread (warp 8, lane 0) over the item's nst stages; commits
    // "done" at the end whatever happened.
    template <class SH>
    static __device__ __forceinline__ void mma(SH* sh, uint32_t sbase, uint32_t tmem, int nst, int gs0, int gd0) {
        volatile int* abort = &sh->abort;
        const uint32_t idesc = tc_idesc<PREC, KMAX == 32 ? 64u : 128u>();
        int st = gs0 % NRING;
        uint32_t ph = (uint32_t)(gs0 / NRING) & 1u;
        for (int it = 0; it < nst; ++it) {
            if (!mbar_wait(&sh->full[st], ph, abort)) break;
            const bool first = it % DRAIN == 0;  // first stage of a period: W starts afresh
            if (first && it > 0 && !mbar_wait(&sh->wfree, (uint32_t)((gd0 + it / DRAIN - 1) & 1), abort)) break;
            tc_fence_after();
            const uint32_t sa0 = sbase + (uint32_t)st * BYTES;
#pragma unroll
            for (int sub = 0; sub < SUBS; ++sub) {
                const uint32_t sa = sa0 + (uint32_t)(sub * C::STAGE_BYTES);
#pragma unroll
                for (int kk = 0; kk < TC_T / 16; ++kk) {
                    const uint64_t hi = desc_sw128(sa + kk * 32);
                    const uint32_t acc = (first && sub == 0 && kk == 0) ? 0u : 1u;
                    // narrow: D += Y X_hi^T (A the whole sub-tile, B its first 64 rows);
                    // wide: D += X_hi X_hi^T + (2 X_lo) X_hi^T
                    umma(tmem, hi, hi, idesc, acc);
                    if (KMAX == 64 && PREC != TCP_BF16) umma(tmem, desc_sw128(sa + C::LO_OFFSET + kk * 32), hi, idesc, 1u);
                }
            }
            umma_commit(&sh->empty[st]);
            if (it % DRAIN == DRAIN - 1 && it + 1 < nst) umma_commit(&sh->wfull);
            if (++st == NRING) { st = 0; ph ^= 1u; }
        }
        umma_commit(&sh->done);  // fires once every issued MMA has completed
    }

    // All threads, after the item's "done" wait and a CTA barrier (with the
    // tcgen05 fences around it): W (+ T) to the fold buffer, then the complex
    // Gram of K users times the per-user factors, or NaN if !ok.
    template <class SH>
    static __device__ __forceinline__ void epilogue(SH* sh, float* fold, uint32_t tmem, int K, int ndrain, bool ok, double2* o,
                                    int tid, int warp, int lane) {
        epilogue_fold(fold, tmem, ndrain, ok, warp, lane);
        epilogue_write(sh, fold, K, 0, ok, o, tid);
    }

    // W (+ T) of the accumulator to the fold buffer (warps 0-3), then a CTA
    // barrier.
    static __device__ __forceinline__ void epilogue_fold(float* fold, uint32_t tmem, int ndrain, bool ok, int warp, int lane) {
        if (ok && warp < 4) {
            const int m = warp * 32 + lane;  // row of D
            const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
            for (int cb = 0; cb < WCOLS / 16; ++cb) {
                uint32_t v[16], u[16];
                tmem_ld16(trow + cb * 16, v);
                if (ndrain > 0) tmem_ld16(trow + WCOLS + cb * 16, u);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    fold[m * C::FOLD_LD + cb * 16 + j] =
                        ndrain > 0 ? __uint_as_float(v[j]) + __uint_as_float(u[j]) : __uint_as_float(v[j]);
            }
        }
        tc_fence_before();
        __syncthreads();
    }

    // The complex Gram of the K users in lanes u0 .. u0 + K - 1 from the fold
    // (R = X X^T, 2 KMAX square) times their per-user factors, or NaN if !ok.
    template <class SH>
    static __device__ __forceinline__ void epilogue_write(const SH* sh, const float* fold, int K, int u0, bool ok, double2* o,
                                          int tid) {
        if (ok) {
            const int P = K * (K + 1) / 2;
            for (int q = tid; q < P; q += TC_THREADS) {
                int i = 0, rl = K, p = q;
                while (p >= rl) { p -= rl; ++i; --rl; }
                const int j = i + p;
                auto R = [&](int r, int c) {  // (X X^T)_rc
                    return KMAX == 32 ? fold[r * C::FOLD_LD + c] + fold[(r + 64) * C::FOLD_LD + c] +
                                            fold[(c + 64) * C::FOLD_LD + r]
                                      : 0.5f * (fold[r * C::FOLD_LD + c] + fold[c * C::FOLD_LD + r]);
                };
                const int a = u0 + i, b = u0 + j;
                double re = (double)(R(a, b) + R(KMAX + a, KMAX + b));
                double im = (double)(R(a, KMAX + b) - R(KMAX + a, b));
                const double us = sh->fac[a] * sh->fac[b];
                re *= us;
                im *= us;
                if (i == j) {
                    o[i * K + i] = make_double2(re, 0.0);
                } else {
                    o[i * K + j] = make_double2(re, im);
                    o[j * K + i] = make_double2(re, -im);
                }
            }
        } else {
            for (int e = tid; e < K * K; e += TC_THREADS) o[e] = make_double2(nan(""), nan(""));
        }
    }
};

}  // namespace xl
