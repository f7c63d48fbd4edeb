// Exact Gram matrices on the 5th-generation tensor cores (tcgen05) with FP32
// accumulation in tensor memory: BF16 (one term), BF16 hi/lo split, or FP16
// hi/lo split of per-user scaled entries.
//
// The complex Gram G = H^H H of K users is a real contraction over the
// elements: with X = [Re H ; Im H] (2K rows, one column per element),
//   Re G_ij = (X X^T)_{i,j} + (X X^T)_{K+i,K+j},  Im G_ij = (X X^T)_{i,K+j} - (X X^T)_{K+i,j}.
// Each FP32 channel entry is split v = hi + lo in BF16 (|v - hi - lo| <=
// 2^-16 |v|) or, after scaling user k's entries by s_k = 1/|h_k| at the
// array centre so that they sit near 1, in FP16 (<= 2^-22 |v|; the scale is
// divided out in FP64 at the end).  For K <= 32, Y = [X_hi ; X_lo] has 128
// rows and M = 128, N = 64 MMAs accumulate D = Y X_hi^T = [P ; Q], P =
// X_hi X_hi^T and Q = X_lo X_hi^T, so that X X^T = P + Q + Q^T up to
// X_lo X_lo^T (below 2^-18 relative with the round-to-nearest split).  Even
// and odd 64-element sub-tiles go to two accumulators (TMEM columns 0-63 and
// 64-127) summed at the end: tcgen05 rounds each accumulation towards zero,
// and halving the steps per accumulator halves that bias.
// For 32 < K <= 64, X_hi and X_lo have 128 rows each and three MMAs per
// k-step accumulate X_hi X_hi^T + X_lo X_hi^T + X_hi X_lo^T into one
// 128 x 128 accumulator.  The single-term BF16 variant keeps X_hi only.
//
// Pipeline (one CTA per trial chunk, 9 warps):
//   warps 0-7  generate ring stages (two of 128 elements for K <= 32, three
//              of 64 for K <= 64): lane = user, warp = one 8-element slice
//              per 64-element sub-tile; each thread writes 16-byte rows of
//              the K-major, 128-byte-swizzled 16-bit tile, fences the async
//              proxy and arrives on the stage's "full" barrier;
//   warp 8     allocates 128 TMEM columns; one thread waits for each full
//              stage, issues four K=16 tcgen05.mma per sub-tile into TMEM and
//              commits to the stage's "empty" barrier (generators reuse the
//              stage once it fires) and, at the end, to "done";
//   warps 0-3  read the accumulator back (tcgen05.ld), fold the blocks and
//              write the complex Gram in FP64.
// Every wait is bounded; a wait that gives up marks the trial (NaN output),
// lets outstanding MMAs drain and frees the tensor memory.
#include <math.h>

#include <type_traits>

#include "tc_common.cuh"

namespace xl {

// Ring of the Gram kernel: NRING stages of T elements, each SUBS 64-element
// sub-tiles of the K-major swizzled layout (TcCfg::STAGE_BYTES each).  K <= 32
// uses two stages of 128 elements, so the per-stage bookkeeping of a
// generator thread is paid once per 16 entries; K <= 64 three of 64.
template <int KMAX>
struct GtRing {
    static constexpr int SUBS = KMAX == 32 ? 2 : 1;
    static constexpr int T = TC_T * SUBS;
    static constexpr int NRING = KMAX == 32 ? 2 : TC_STAGES;
    static constexpr uint32_t BYTES = (uint32_t)TcCfg<KMAX>::STAGE_BYTES * SUBS;  // per ring stage
};

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

template <int KMAX>
struct UraShared {
    double ux[KMAX];            // the users' true x
    float2 rowc[2][KMAX];       // (x'/lambda)^2 and 2 (x'/lambda)^2 of the current and the next span's row
    float roww[2];              // amplitude weight of those rows
};

template <int MODEL, int KMAX, int PREC, bool URA>
__global__ void __launch_bounds__(TC_THREADS, KMAX == 32 ? 3 : 2)
    gram_tc_kernel(Geom g, GenParams gp, const double* __restrict__ users, int K, int S, int64_t chunk,
                   double2* __restrict__ out, UraRows ura) {
    using C = TcCfg<KMAX>;
    static_assert(!URA || PREC == TCP_BF16X3, "the URA mode generates weighted entries for the BF16 hi/lo split");
    using RG = GtRing<KMAX>;
    extern __shared__ unsigned char smem_raw[];
    // stages must be 1024-byte aligned for the 128-byte swizzle
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char* stages = base;
    TcShared<KMAX>* sh = reinterpret_cast<TcShared<KMAX>*>(base + RG::NRING * RG::BYTES);
    float* fold = reinterpret_cast<float*>(base);  // epilogue reuses the stages
    UraShared<KMAX>* ush = reinterpret_cast<UraShared<KMAX>*>(reinterpret_cast<unsigned char*>(sh) + sizeof(TcShared<KMAX>));

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int b = blockIdx.x, s = blockIdx.y;

    if (tid == 0) {
        for (int i = 0; i < RG::NRING; ++i) {
            mbar_init(&sh->full[i], TC_GEN_THREADS);
            mbar_init(&sh->empty[i], 1);
        }
        mbar_init(&sh->done, 1);
        sh->abort = 0;
        sh->bad = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh->tmem_base)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid < KMAX) {
        double x = 1.0, y = 0.0;
        if (tid < K) {
            x = users[((int64_t)b * K + tid) * 2];
            y = users[((int64_t)b * K + tid) * 2 + 1];
        }
        UserGeo u = make_user_geo(g, x, y);
        if (tid < K && !u.ok) atomicOr(&sh->bad, 1);
        // the BF16 paths generate entries without the amplitude constant and
        // apply it to the Gram in FP64; the FP16 path scales user k's entries by
        // 1/|h_k| at the array centre so that they sit near 1, and divides it out
        double fac = amp_const(g, x, y);
        if (URA) {
            ush->ux[tid] = x;
            fac *= 1.4142135623730951;  // fac_i fac_j carries the 2 of a mirrored row pair
        }
        if (PREC == TCP_F16X3) {
            const double rc = sqrt(x * x + y * y) * g.inv_lambda;  // distance in wavelengths
            double amp_c = (MODEL == XLMIMO_UPW) ? fac : (MODEL == XLMIMO_PNUSW) ? fac / (rc * sqrt(rc)) : fac / rc;
            const float sc = (float)(1.0 / amp_c);
            u.ampc *= sc;
            fac = 1.0 / (double)sc;
        }
        sh->ug[tid] = u;
        sh->fac[tid] = fac;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh->tmem_base;
    volatile int* abort = &sh->abort;

    const int64_t nbeg = (int64_t)s * chunk;
    const int64_t nend = min(g.N, nbeg + chunk);
    const int nst = (int)((nend - nbeg + RG::T - 1) / RG::T);

    if (warp < 8) {
        // ---------------- generators: lane = user (and user + 32), warp = 8-element slice.
        // The double-float phase references of a span (TC_REF_SPAN elements)
        // are made once per CTA: warp (sp + 1) % 8 prepares span sp + 1 into
        // the other half of a double buffer while span sp is generated, and
        // the eight generator warps meet at a named barrier at every span
        // start.  That barrier also votes on stopping, so that after an abort
        // all 256 generator threads leave the loop together.
        constexpr int SPAN = URA ? URA_SPAN : TC_REF_SPAN;
        constexpr int SPAN_ST = SPAN / RG::T;  // stages per span
        const int nsp = (nst + SPAN_ST - 1) / SPAN_ST;
        auto make_refs = [&](int sp) {
            const long long m0 = (long long)(nbeg + (int64_t)sp * SPAN);
            if (URA) {
                const long long q = m0 / ura.ncol;
                const long long ncs = m0 - q * ura.ncol + SPAN / 2;  // span centre, column index in the row
                const double z = ((double)q + ura.zoff) * ura.spacing;
                for (int kk = lane; kk < KMAX; kk += 32) {
                    // the spherical-wave reference reads y, x^2 and 2 (x/lambda)^2 only:
                    // the user's own geometry with x'^2 = x^2 + z^2 in their place
                    const double x = ush->ux[kk];
                    const double x2 = fma(x, x, z * z);
                    const double xl2 = x2 * (g.inv_lambda * g.inv_lambda);
                    UserGeo ug = sh->ug[kk];
                    ug.x2 = ff_from_double(x2);
                    ug.xl2 = (float)xl2;
                    ug.x2x2 = (float)(2.0 * xl2);
                    sh->ref[sp & 1][kk] = make_user_ref(gp, ug, ncs);
                    ush->rowc[sp & 1][kk] = make_float2(ug.xl2, ug.x2x2);
                }
                if (lane == 0) ush->roww[sp & 1] = (ura.odd && q == 0) ? 0.70710678118654752f : 1.0f;
            } else {
                const long long ncs = m0 + SPAN / 2;
                for (int kk = lane; kk < KMAX; kk += 32) sh->ref[sp & 1][kk] = make_user_ref(gp, sh->ug[kk], ncs);
            }
        };
        if (warp == 0 && nsp > 0) make_refs(0);
        // stage-tile offsets of this lane's four component rows (slot 0, slot 1)
        uint32_t soff[C::SLOTS][4];
#pragma unroll
        for (int slot = 0; slot < C::SLOTS; ++slot)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int f = KMAX * c + lane + 32 * slot;  // row of the stage tile
                const int rin = f & 7;
                soff[slot][c] = (uint32_t)((f >> 3) * 1024 + rin * 128 + ((warp ^ rin) << 4));
            }
        PairConst pc = make_pair_const(UserRef{0.f, 0.f, 0.f, 0.f, 1.f, 0.f}, gp.dprime_f, 0.f, 0.f, 0.f);
        // stage bookkeeping kept incremental and 32-bit: ring slot st and its
        // wrap count, this warp's slice offset from the span centre (mf0, an
        // exact small integer in FP32), valid elements of the last stage
        const uint32_t sbase = smem_u32(stages);
        const int last_rem = (int)(nend - nbeg - (int64_t)(nst - 1) * RG::T) - warp * 8;
        int st = 0, wraps = 0;
        float mf0 = 0.f;
        bool dead = false;
        for (int it = 0; it < nst; ++it) {
            const int sp = it / SPAN_ST;
            if ((it & (SPAN_ST - 1)) == 0) {
                uint32_t stop;
                const uint32_t mine = (dead || *abort) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred p, 1, 256, q;\n selp.u32 %0, 1, 0, p;\n}\n"
                    : "=r"(stop)
                    : "r"(mine)
                    : "memory");
                if (stop) break;
                mf0 = (float)(warp * 8 - SPAN / 2);
                if (C::SLOTS == 1) {
                    if (URA) {
                        const float2 rc = ush->rowc[sp & 1][lane];
                        pc = make_pair_const(sh->ref[sp & 1][lane], gp.dprime_f, rc.x, rc.y, lane < K ? ush->roww[sp & 1] : 0.f);
                    } else {
                        const UserGeo& u = sh->ug[lane];
                        pc = make_pair_const(sh->ref[sp & 1][lane], gp.dprime_f, u.xl2, u.x2x2, lane < K ? u.ampc : 0.f);
                    }
                }
                if (warp == ((sp + 1) & 7) && sp + 1 < nsp) make_refs(sp + 1);
            } else {
                mf0 += (float)RG::T;
            }
            const int cur = st;
            const int wcur = wraps;
            if (++st == RG::NRING) { st = 0; ++wraps; }
            if (dead) continue;
            if (wcur > 0 && !mbar_wait(&sh->empty[cur], (wcur - 1) & 1, abort)) {
                dead = true;
                continue;
            }
            const int rem = it == nst - 1 ? last_rem : RG::T;  // valid elements from this warp's first slice on
            const uint32_t sb = sbase + (uint32_t)cur * RG::BYTES;
#pragma unroll
            for (int slot = 0; slot < C::SLOTS; ++slot) {
                const int k = lane + 32 * slot;
                if (C::SLOTS > 1) {
                    if (URA) {
                        const float2 rc = ush->rowc[sp & 1][k];
                        pc = make_pair_const(sh->ref[sp & 1][k], gp.dprime_f, rc.x, rc.y, k < K ? ush->roww[sp & 1] : 0.f);
                    } else {
                        const UserGeo& u = sh->ug[k];
                        pc = make_pair_const(sh->ref[sp & 1][k], gp.dprime_f, u.xl2, u.x2x2, k < K ? u.ampc : 0.f);
                    }
                }
#pragma unroll
                for (int sub = 0; sub < RG::SUBS; ++sub) {
                    const float mfs = mf0 + (float)(sub * TC_T);  // this slice's first offset
                    const int rs = rem - sub * TC_T;              // its valid elements (<= 0: none)
                    uint32_t w[4][4];  // [component: Re hi, Im hi, Re lo, Im lo][packed pair]
                    // two instances of the slice: full (no per-element checks; every
                    // stage but a chunk's last) and partial (elements past the end are 0)
                    const float base = slice_base(pc, mfs + 3.5f);  // phase at the slice centre
                    const float dp = pc.dp.x, u0 = mfs * dp;        // u = m spacing/lambda
                    auto slice = [&](auto partial) {
#pragma unroll
                        for (int i = 0; i < 8; i += 2) {
                            float2 re, im;
                            gen_pair<MODEL, !URA && PREC != TCP_F16X3>(pc, make_float2(fmaf((float)i, dp, u0), fmaf((float)(i + 1), dp, u0)),
                                                                make_float2((float)i - 3.5f, (float)i - 2.5f), base, re, im);
                            if (decltype(partial)::value) {
                                if (i >= rs) { re.x = 0.f; im.x = 0.f; }
                                if (i + 1 >= rs) { re.y = 0.f; im.y = 0.f; }
                            }
                            split2<PREC>(re.x, re.y, w[0][i >> 1], w[2][i >> 1]);
                            split2<PREC>(im.x, im.y, w[1][i >> 1], w[3][i >> 1]);
                        }
                    };
                    if (rs >= 8) slice(std::integral_constant<bool, false>());
                    else slice(std::integral_constant<bool, true>());
                    const int ncomp = (PREC == TCP_BF16 && KMAX == 64) ? 2 : 4;  // the one-term K>32 MMA reads hi only
                    const uint32_t ss = sb + (uint32_t)(sub * C::STAGE_BYTES);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        if (c >= ncomp) break;
                        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(ss + soff[slot][c]), "r"(w[c][0]),
                                     "r"(w[c][1]), "r"(w[c][2]), "r"(w[c][3])
                                     : "memory");
                    }
                }
            }
            fence_async_smem();
            mbar_arrive(&sh->full[cur]);
        }
    } else {
        // ---------------- MMA issuer (one lane; the others wait at the warp barrier)
        if (lane == 0) {
            const uint32_t idesc = tc_idesc<PREC, KMAX == 32 ? 64u : 128u>();
            for (int it = 0; it < nst; ++it) {
                const int st = it % RG::NRING;
                if (!mbar_wait(&sh->full[st], (it / RG::NRING) & 1, abort)) break;
                tc_fence_after();
                const uint32_t sa0 = smem_u32(stages) + (uint32_t)st * RG::BYTES;
#pragma unroll
                for (int sub = 0; sub < RG::SUBS; ++sub) {
                    const uint32_t sa = sa0 + (uint32_t)(sub * C::STAGE_BYTES);
#pragma unroll
                    for (int kk = 0; kk < TC_T / 16; ++kk) {
                        const uint64_t hi = desc_sw128(sa + kk * 32);
                        if (KMAX == 32) {
                            // D_sub += Y X_hi^T: A is the whole sub-tile, B its first 64 rows
                            const uint32_t acc = (it > 0 || kk > 0) ? 1u : 0u;
                            umma(tmem + (uint32_t)sub * 64u, hi, hi, idesc, acc);
                        } else {
                            const uint32_t acc = (it > 0 || kk > 0) ? 1u : 0u;
                            umma(tmem, hi, hi, idesc, acc);
                            if (PREC != TCP_BF16) {
                                const uint64_t lo = desc_sw128(sa + C::LO_OFFSET + kk * 32);
                                umma(tmem, lo, hi, idesc, 1u);
                                umma(tmem, hi, lo, idesc, 1u);
                            }
                        }
                    }
                }
                umma_commit(&sh->empty[st]);
            }
            umma_commit(&sh->done);  // fires once every issued MMA has completed
        }
        __syncwarp();
    }

    // ---------------- epilogue (warps 0-3 own TMEM lanes 0-127)
    double2* o = out + ((int64_t)b * S + s) * K * K;
    bool ok = mbar_wait(&sh->done, 0, abort);
    tc_fence_after();
    __syncthreads();
    ok = ok && !*abort && !sh->bad;
    if (ok && warp < 4) {
        const int m = warp * 32 + lane;  // row of D
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        float v[32], u[32];
        if (KMAX == 32) {
            // the two accumulators (one per sub-tile of every stage)
#pragma unroll
            for (int cb = 0; cb < 2; ++cb) {
                tmem_ld32(trow + cb * 32, v);
                tmem_ld32(trow + 64 + cb * 32, u);
#pragma unroll
                for (int j = 0; j < 32; ++j) fold[m * C::FOLD_LD + cb * 32 + j] = v[j] + u[j];
            }
        } else {
#pragma unroll
            for (int cb = 0; cb < 4; ++cb) {
                tmem_ld32(trow + cb * 32, v);
#pragma unroll
                for (int j = 0; j < 32; ++j) fold[m * C::FOLD_LD + cb * 32 + j] = v[j];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (ok) {
        // R (2 KMAX square) from the fold; complex Gram from R times the per-user factors
        const int P = K * (K + 1) / 2;
        for (int q = tid; q < P; q += TC_THREADS) {
            int i = 0, rl = K, p = q;
            while (p >= rl) { p -= rl; ++i; --rl; }
            const int j = i + p;
            auto R = [&](int r, int c) {  // (X X^T)_rc
                return KMAX == 32 ? fold[r * C::FOLD_LD + c] + fold[(r + 64) * C::FOLD_LD + c] +
                                        fold[(c + 64) * C::FOLD_LD + r]
                                  : fold[r * C::FOLD_LD + c];
            };
            double re = (double)(R(i, j) + R(KMAX + i, KMAX + j));
            double im = (double)(R(i, KMAX + j) - R(KMAX + i, j));
            const double us = sh->fac[i] * sh->fac[j];
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
    __syncthreads();
    if (warp == 8) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
    }
}

template <int KMAX>
static size_t tc_smem_bytes(bool ura = false) {
    return 1024 + GtRing<KMAX>::NRING * GtRing<KMAX>::BYTES + sizeof(TcShared<KMAX>) +
           (ura ? sizeof(UraShared<KMAX>) : 0);
}

using TcKernel = void (*)(Geom, GenParams, const double*, int, int, int64_t, double2*, UraRows);

template <int MODEL, int KMAX>
static TcKernel pick_prec(int prec) {
    return prec == XLMIMO_BF16 ? gram_tc_kernel<MODEL, KMAX, TCP_BF16, false>
         : prec == XLMIMO_F16X3 ? gram_tc_kernel<MODEL, KMAX, TCP_F16X3, false>
                                : gram_tc_kernel<MODEL, KMAX, TCP_BF16X3, false>;
}

template <int KMAX>
static TcKernel pick(int model, int prec) {
    return model == XLMIMO_PNUSW ? pick_prec<XLMIMO_PNUSW, KMAX>(prec)
         : model == XLMIMO_UPW   ? pick_prec<XLMIMO_UPW, KMAX>(prec)
                                 : pick_prec<XLMIMO_FSPL_USW, KMAX>(prec);
}

static bool tc_device(int* dev) {
    int major = 0, minor = 0;
    cudaGetDevice(dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, *dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, *dev);
    return major == 10 && minor == 3;
}

// Launch over B trials of g.N elements in S element chunks (multiples of
// `span`), reducing chunk partials when S > 1.
static int launch_tc_chunks(TcKernel kern, size_t smem, const Geom& g, const GenParams& gp, int span,
                            const double* users, int K, int B, double* gram, const UraRows& ura, cudaStream_t st) {
    int S = choose_split(g.N, B, span, 4);
    int64_t spans = (g.N + span - 1) / span;
    int64_t chunk = ((spans + S - 1) / S) * span;
    S = (int)((g.N + chunk - 1) / chunk);
    double* part = nullptr;
    if (S > 1) {
        int rc = cuda_status(cudaMallocAsync((void**)&part, (size_t)B * S * K * K * sizeof(double2), st),
                             "workspace allocation");
        if (rc) return rc;
    }
    dim3 grid(B, S);
    kern<<<grid, TC_THREADS, smem, st>>>(g, gp, users, K, S, chunk, (double2*)(S == 1 ? gram : part), ura);
    int rc = cuda_status(cudaGetLastError(), "gram_tc launch");
    if (!rc && S > 1) rc = launch_reduce_partials(part, S, K, B, gram, st);
    if (part) cudaFreeAsync(part, st);
    return rc;
}

bool gram_tc_ura_supported(const Geom& g, int64_t ncol, int prec) {
    int dev = 0;
    return prec == XLMIMO_BF16X3 && g.model != XLMIMO_UPW && ncol % URA_SPAN == 0 && tc_device(&dev);
}

int launch_gram_tc_ura(const Geom& g, int64_t ncol, int64_t rows, const double* users, int K, int B, double* gram,
                       cudaStream_t st) {
    int dev = 0;
    if (!tc_device(&dev) || ncol % URA_SPAN != 0 || g.model == XLMIMO_UPW) {
        set_error("the URA mode of the tensor-core Gram needs an sm_103 device, rows of a multiple of %d "
                  "elements and a spherical-wave model", URA_SPAN);
        return XLMIMO_EUNSUPPORTED;
    }
    const bool wide = K > 32;
    const bool pn = g.model == XLMIMO_PNUSW;
    TcKernel kern = wide ? (pn ? gram_tc_kernel<XLMIMO_PNUSW, 64, TCP_BF16X3, true>
                               : gram_tc_kernel<XLMIMO_FSPL_USW, 64, TCP_BF16X3, true>)
                         : (pn ? gram_tc_kernel<XLMIMO_PNUSW, 32, TCP_BF16X3, true>
                               : gram_tc_kernel<XLMIMO_FSPL_USW, 32, TCP_BF16X3, true>);
    const size_t smem = wide ? tc_smem_bytes<64>(true) : tc_smem_bytes<32>(true);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_status(e, "gram_tc attribute");
    Geom row = g, all = g;
    row.N = ncol;                       // element positions within a row
    all.N = ((rows + 1) / 2) * ncol;    // the trial's elements: its row pairs one after another
    UraRows ura{(long long)ncol, (rows & 1) ? 0.0 : 0.5, g.spacing, (int)(rows & 1)};
    return launch_tc_chunks(kern, smem, all, make_gen_params(row), URA_SPAN, users, K, B, gram, ura, st);
}

// ctas_per_sm > 0 caps the kernel's residency by sizing its shared memory, so
// that kernels on other streams can run on the same SMs; 0 leaves the
// residency to the register and shared-memory budget.
int launch_gram_tc(const Geom& g, const double* users, int K, int B, int prec, double* gram, cudaStream_t st,
                   int ctas_per_sm) {
    int dev = 0;
    if (!tc_device(&dev)) {
        set_error("the tensor-core precisions need an sm_103 device (tcgen05)");
        return XLMIMO_EUNSUPPORTED;
    }
    const bool wide = K > 32;
    TcKernel kern = wide ? pick<64>(g.model, prec) : pick<32>(g.model, prec);
    size_t smem = wide ? tc_smem_bytes<64>() : tc_smem_bytes<32>();
    if (ctas_per_sm > 0) {
        int per_sm = 0;
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        size_t want = (size_t)per_sm / (size_t)(ctas_per_sm + 1) + 1024;  // more than 1/(c+1) of the SM
        if (want > smem) smem = want;
    }
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_status(e, "gram_tc attribute");
    return launch_tc_chunks(kern, smem, g, make_gen_params(g), TC_REF_SPAN, users, K, B, gram, UraRows{0, 0.0, 0.0, 0},
                            st);
}

}  // namespace xl
