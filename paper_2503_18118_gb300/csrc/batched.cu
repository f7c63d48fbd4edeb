// Ragged batches: many instances with their own N, K, receiver and noise in
// one persistent tensor-core launch plus ragged receiver / rate launches.
//
// Work items are (instance, element chunk) pairs ordered longest first.
// gram_tc_ragged_kernel runs a fixed number of CTAs per SM; each pulls the
// next item from an atomic counter and runs the same generate -> tcgen05 ->
// fold pipeline as gram_tc_kernel (128-row X_hi / X_lo blocks, so K <= 64),
// keeping its TMEM allocation and mbarrier phases across items.  Items that
// cover a whole instance write its Gram directly; the chunks of a split
// instance write partial Gram matrices that ragged_reduce_kernel sums in
// chunk order.  The receivers run one CTA per instance, launched per user
// count bucket so that shared memory is sized for the bucket.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include <type_traits>

#include "tc_common.cuh"

namespace xl {

struct DevItem {
    int inst, chunk;
    long long n0, n1;
};

constexpr int RG_KMAX = 64;
using RCfg = TcCfg<RG_KMAX>;

struct RgShared {
    uint64_t full[TC_STAGES];
    uint64_t empty[TC_STAGES];
    uint64_t done;
    uint32_t tmem_base;
    int abort;
    int bad;
    int item;
    UserGeo ug[RG_KMAX];
    double fac[RG_KMAX];  // per-user factor of the Gram: G_ij = fac_i fac_j (accumulated sum)
    UserRef ref[2][RG_KMAX];  // phase references of the current and the next span
};

template <int MODEL, int PREC>
__global__ void __launch_bounds__(TC_THREADS, 2)
    gram_tc_ragged_kernel(Geom g, GenParams gp, const DevInst* __restrict__ insts, const DevItem* __restrict__ items,
                          int n_items, int* __restrict__ counter, const double* __restrict__ users,
                          double2* __restrict__ gram, double2* __restrict__ part) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char* stages = base;
    RgShared* sh = reinterpret_cast<RgShared*>(base + TC_STAGES * RCfg::STAGE_BYTES);
    float* fold = reinterpret_cast<float*>(base);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int i = 0; i < TC_STAGES; ++i) {
            mbar_init(&sh->full[i], TC_GEN_THREADS);
            mbar_init(&sh->empty[i], 1);
        }
        mbar_init(&sh->done, 1);
        sh->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh->tmem_base)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh->tmem_base;
    volatile int* abort = &sh->abort;
    long long gs = 0;    // stages issued by this CTA so far (mbarrier phases continue across items)
    int done_count = 0;  // items completed by this CTA

    for (;;) {
        if (tid == 0) sh->item = atomicAdd(counter, 1);
        tc_fence_before();
        __syncthreads();  // previous item's epilogue finished with TMEM and the stage buffers
        tc_fence_after();
        const int w = sh->item;
        if (w >= n_items) break;
        const DevItem itm = items[w];
        const DevInst in = insts[itm.inst];
        const int K = in.k;
        if (tid == 0) sh->bad = 0;
        __syncthreads();
        if (tid < RG_KMAX) {
            double x = 1.0, y = 0.0;
            if (tid < K) {
                x = users[(in.user_off + tid) * 2];
                y = users[(in.user_off + tid) * 2 + 1];
            }
            UserGeo u = make_user_geo(g, x, y);
            if (tid < K && !u.ok) atomicOr(&sh->bad, 1);
            // the BF16 paths generate entries without the amplitude constant and
            // apply it to the Gram in FP64; the FP16 path scales user k's entries by
            // 1/|h_k| at the array centre so that they sit near 1, and divides it out
            double fac = amp_const(g, x, y);
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
        __syncthreads();
        const int64_t nbeg = itm.n0, nend = itm.n1;
        const int nst = (int)((nend - nbeg + TC_T - 1) / TC_T);
        Geom gi = g;
        gi.N = in.n_ant;
        GenParams gpi = gp;
        gpi.nm1 = in.n_ant - 1;

        if (warp < 8) {
            // generators (see gram_tc_kernel): span references made once per
            // CTA by a rotating warp into a double buffer, met at a named
            // barrier that votes on stopping; store offsets computed once; full
            // slices without per-element checks
            constexpr int SPAN_ST = TC_REF_SPAN / TC_T;
            const int nsp = (nst + SPAN_ST - 1) / SPAN_ST;
            auto make_refs = [&](int sp) {
                const long long ncs = (long long)(nbeg + (int64_t)sp * TC_REF_SPAN + TC_REF_SPAN / 2);
                for (int kk = lane; kk < RG_KMAX; kk += 32) sh->ref[sp & 1][kk] = make_user_ref(gpi, sh->ug[kk], ncs);
            };
            if (warp == 0 && nsp > 0) make_refs(0);
            uint32_t soff[2][4];
#pragma unroll
            for (int slot = 0; slot < 2; ++slot)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int f = RG_KMAX * c + lane + 32 * slot;
                    const int rin = f & 7;
                    soff[slot][c] = (uint32_t)((f >> 3) * 1024 + rin * 128 + ((warp ^ rin) << 4));
                }
            // stage bookkeeping incremental and 32-bit (see gram_tc_kernel): ring
            // slot and wrap count continue from the CTA's previous items
            const uint32_t sbase = smem_u32(stages);
            const int last_rem = (int)(nend - nbeg - (int64_t)(nst - 1) * TC_T) - warp * 8;
            int st = (int)(gs % TC_STAGES);
            long long wraps = gs / TC_STAGES;
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
                    mf0 = (float)(warp * 8 - TC_REF_SPAN / 2);
                    if (warp == ((sp + 1) & 7) && sp + 1 < nsp) make_refs(sp + 1);
                } else {
                    mf0 += (float)TC_T;
                }
                const int cur = st;
                const long long wcur = wraps;
                if (++st == TC_STAGES) { st = 0; ++wraps; }
                if (dead) continue;
                if (wcur > 0 && !mbar_wait(&sh->empty[cur], (uint32_t)((wcur - 1) & 1), abort)) {
                    dead = true;
                    continue;
                }
                const int rem = it == nst - 1 ? last_rem : 8;
                const uint32_t sb = sbase + (uint32_t)cur * RCfg::STAGE_BYTES;
#pragma unroll
                for (int slot = 0; slot < 2; ++slot) {
                    const int k = lane + 32 * slot;
                    uint32_t wv[4][4];
                    if (k < K || slot == 0) {
                        const UserGeo& u = sh->ug[k];
                        const PairConst pc =
                            make_pair_const(sh->ref[sp & 1][k], gpi.dprime_f, u.xl2, u.x2x2, k < K ? u.ampc : 0.f);
                        const float base = slice_base(pc, mf0 + 3.5f);  // phase at the slice centre
                        const float dp = pc.dp.x, u0 = mf0 * dp;        // u = m spacing/lambda
                        auto slice = [&](auto partial) {
#pragma unroll
                            for (int i = 0; i < 8; i += 2) {
                                float2 re, im;
                                gen_pair<MODEL, PREC != TCP_F16X3>(pc, make_float2(fmaf((float)i, dp, u0), fmaf((float)(i + 1), dp, u0)),
                                                            make_float2((float)i - 3.5f, (float)i - 2.5f), base, re, im);
                                if (decltype(partial)::value) {
                                    if (i >= rem) { re.x = 0.f; im.x = 0.f; }
                                    if (i + 1 >= rem) { re.y = 0.f; im.y = 0.f; }
                                }
                                split2<PREC>(re.x, re.y, wv[0][i >> 1], wv[2][i >> 1]);
                                split2<PREC>(im.x, im.y, wv[1][i >> 1], wv[3][i >> 1]);
                            }
                        };
                        if (rem >= 8) slice(std::integral_constant<bool, false>());
                        else slice(std::integral_constant<bool, true>());
                    } else {
#pragma unroll
                        for (int c = 0; c < 4; ++c)
#pragma unroll
                            for (int q = 0; q < 4; ++q) wv[c][q] = 0u;
                    }
                    const int ncomp = PREC == TCP_BF16 ? 2 : 4;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        if (c >= ncomp) break;
                        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(sb + soff[slot][c]),
                                     "r"(wv[c][0]), "r"(wv[c][1]), "r"(wv[c][2]), "r"(wv[c][3])
                                     : "memory");
                    }
                }
                fence_async_smem();
                mbar_arrive(&sh->full[cur]);
            }
        } else {
            if (lane == 0) {
                const uint32_t idesc = tc_idesc<PREC>();
                for (int it = 0; it < nst; ++it) {
                    const long long gsi = gs + it;
                    const int st = (int)(gsi % TC_STAGES);
                    if (!mbar_wait(&sh->full[st], (uint32_t)((gsi / TC_STAGES) & 1), abort)) break;
                    tc_fence_after();
                    const uint32_t sa = smem_u32(stages + st * RCfg::STAGE_BYTES);
#pragma unroll
                    for (int kk = 0; kk < TC_T / 16; ++kk) {
                        const uint32_t acc = (it > 0 || kk > 0) ? 1u : 0u;
                        const uint64_t hi = desc_sw128(sa + kk * 32);
                        umma(tmem, hi, hi, idesc, acc);
                        if (PREC != TCP_BF16) {
                            const uint64_t lo = desc_sw128(sa + RCfg::LO_OFFSET + kk * 32);
                            umma(tmem, lo, hi, idesc, 1u);
                            umma(tmem, hi, lo, idesc, 1u);
                        }
                    }
                    umma_commit(&sh->empty[st]);
                }
                umma_commit(&sh->done);
            }
            __syncwarp();
        }
        gs += nst;

        // epilogue
        const bool whole = in.nchunks == 1;
        double2* o = whole ? gram + in.gram_off : part + in.part_off + (long long)itm.chunk * K * K;
        bool ok = mbar_wait(&sh->done, (uint32_t)(done_count & 1), abort);
        ++done_count;
        tc_fence_after();
        __syncthreads();
        ok = ok && !*abort && !sh->bad;
        if (ok && warp < 4) {
            const int m = warp * 32 + lane;
            const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
            float v[32];
#pragma unroll
            for (int cb = 0; cb < 4; ++cb) {
                tmem_ld32(trow + cb * 32, v);
#pragma unroll
                for (int j = 0; j < 32; ++j) fold[m * RCfg::FOLD_LD + cb * 32 + j] = v[j];
            }
        }
        tc_fence_before();
        __syncthreads();
        if (ok) {
            const int P = K * (K + 1) / 2;
            for (int q = tid; q < P; q += TC_THREADS) {
                int i = 0, rl = K, p = q;
                while (p >= rl) { p -= rl; ++i; --rl; }
                const int j = i + p;
                const float* F = fold;
                double re = (double)(F[i * RCfg::FOLD_LD + j] + F[(64 + i) * RCfg::FOLD_LD + 64 + j]);
                double im = (double)(F[i * RCfg::FOLD_LD + 64 + j] - F[(64 + i) * RCfg::FOLD_LD + j]);
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
        const int gave_up = *abort;  // read by every thread between two barriers
        __syncthreads();
        if (gave_up) break;  // a wait gave up: stop pulling work (outstanding MMAs drained at "done")
    }
    __syncthreads();
    if (warp == 8) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
    }
}

// Sum the chunk partials of split instances in chunk order.
__global__ void ragged_reduce_kernel(const DevInst* __restrict__ insts, const int* __restrict__ split_list, int n,
                                     const double2* __restrict__ part, double2* __restrict__ gram) {
    const int inst = split_list[blockIdx.x];
    const DevInst in = insts[inst];
    const int KK = in.k * in.k;
    for (int e = threadIdx.x; e < KK; e += blockDim.x) {
        double re = 0.0, im = 0.0;
        for (int c = 0; c < in.nchunks; ++c) {
            double2 v = part[in.part_off + (long long)c * KK + e];
            re += v.x;
            im += v.y;
        }
        gram[in.gram_off + e] = make_double2(re, im);
    }
}

__global__ void ragged_sumrate_kernel(const DevInst* __restrict__ insts, int n, const double* __restrict__ sinr,
                                      double* __restrict__ rate) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const DevInst in = insts[i];
        double r = 0.0;
        for (int k = 0; k < in.k; ++k) r += log2(1.0 + sinr[in.user_off + k]);
        rate[i] = r;
    }
}

// ---------------------------------------------------------------- plan ----
struct BatchPlan {
    Geom g;
    int prec = XLMIMO_BF16X3;
    int count = 0;
    int64_t users_total = 0;
    std::vector<xlmimo_inst> host;
    DevInst* d_inst = nullptr;
    DevItem* d_items = nullptr;
    int* d_counter = nullptr;
    int* d_lists = nullptr;  // [small bucket | large bucket | split instances]
    double2* d_part = nullptr;
    int n_items = 0, n_small = 0, n_large = 0, n_split = 0;
    int64_t chunk = 0;
    int ctas_per_sm = 2;
    size_t part_bytes = 0;
    int tuned = 0, candidates = 0;
    size_t smem = 0;
};



static void free_tables(BatchPlan* p) {
    cudaFree(p->d_inst);
    cudaFree(p->d_items);
    cudaFree(p->d_counter);
    cudaFree(p->d_lists);
    cudaFree(p->d_part);
    p->d_inst = nullptr;
    p->d_items = nullptr;
    p->d_counter = nullptr;
    p->d_lists = nullptr;
    p->d_part = nullptr;
}

// Host tables for one element chunk: items longest first, split instances'
// partial offsets, receiver buckets.
static int build_tables(BatchPlan* p, int64_t chunk, cudaStream_t st) {
    free_tables(p);
    std::vector<DevInst> di(p->count);
    std::vector<DevItem> items;
    std::vector<int> small, large, split;
    long long part = 0;
    for (int i = 0; i < p->count; ++i) {
        const xlmimo_inst& h = p->host[i];
        DevInst d;
        d.n_ant = h.n_ant;
        d.k = h.k;
        d.scheme = h.scheme;
        d.user_off = h.user_off;
        d.gram_off = h.gram_off;
        d.noise = h.noise;
        const long long nch = (h.n_ant + chunk - 1) / chunk;
        d.nchunks = (int)nch;
        d.part_off = nch > 1 ? part : -1;
        d.pad = 0;
        if (nch > 1) {
            part += nch * (long long)h.k * h.k;
            split.push_back(i);
        }
        for (long long c = 0; c < nch; ++c) {
            DevItem it;
            it.inst = i;
            it.chunk = (int)c;
            it.n0 = c * chunk;
            it.n1 = std::min<long long>(h.n_ant, (c + 1) * chunk);
            items.push_back(it);
        }
        (h.k <= 32 ? small : large).push_back(i);
        di[i] = d;
    }
    // longest (generation work = elements x user slots) first
    std::stable_sort(items.begin(), items.end(), [&](const DevItem& a, const DevItem& b) {
        long long ca = (a.n1 - a.n0) * (p->host[a.inst].k > 32 ? 2 : 1);
        long long cb = (b.n1 - b.n0) * (p->host[b.inst].k > 32 ? 2 : 1);
        return ca > cb;
    });
    p->n_items = (int)items.size();
    p->n_small = (int)small.size();
    p->n_large = (int)large.size();
    p->n_split = (int)split.size();
    p->chunk = chunk;
    p->part_bytes = (size_t)part * sizeof(double2);
    std::vector<int> lists;
    lists.insert(lists.end(), small.begin(), small.end());
    lists.insert(lists.end(), large.begin(), large.end());
    lists.insert(lists.end(), split.begin(), split.end());
    int rc = cuda_status(cudaMalloc((void**)&p->d_inst, sizeof(DevInst) * di.size()), "plan tables");
    if (!rc) rc = cuda_status(cudaMalloc((void**)&p->d_items, sizeof(DevItem) * items.size()), "plan tables");
    if (!rc) rc = cuda_status(cudaMalloc((void**)&p->d_counter, sizeof(int)), "plan tables");
    if (!rc) rc = cuda_status(cudaMalloc((void**)&p->d_lists, sizeof(int) * std::max<size_t>(1, lists.size())), "plan tables");
    if (!rc && part > 0) rc = cuda_status(cudaMalloc((void**)&p->d_part, p->part_bytes), "plan workspace");
    if (!rc) rc = cuda_status(cudaMemcpyAsync(p->d_inst, di.data(), sizeof(DevInst) * di.size(), cudaMemcpyHostToDevice, st), "plan upload");
    if (!rc) rc = cuda_status(cudaMemcpyAsync(p->d_items, items.data(), sizeof(DevItem) * items.size(), cudaMemcpyHostToDevice, st), "plan upload");
    if (!rc && !lists.empty())
        rc = cuda_status(cudaMemcpyAsync(p->d_lists, lists.data(), sizeof(int) * lists.size(), cudaMemcpyHostToDevice, st), "plan upload");
    if (!rc) rc = cuda_status(cudaStreamSynchronize(st), "plan upload");
    return rc;
}

using RgKernel = void (*)(Geom, GenParams, const DevInst*, const DevItem*, int, int*, const double*, double2*, double2*);

template <int MODEL>
static RgKernel rg_pick_prec(int prec) {
    return prec == XLMIMO_BF16 ? gram_tc_ragged_kernel<MODEL, TCP_BF16>
         : prec == XLMIMO_F16X3 ? gram_tc_ragged_kernel<MODEL, TCP_F16X3>
                                : gram_tc_ragged_kernel<MODEL, TCP_BF16X3>;
}

static RgKernel rg_pick(int model, int prec) {
    return model == XLMIMO_PNUSW ? rg_pick_prec<XLMIMO_PNUSW>(prec)
         : model == XLMIMO_UPW   ? rg_pick_prec<XLMIMO_UPW>(prec)
                                 : rg_pick_prec<XLMIMO_FSPL_USW>(prec);
}

// Shared memory for a residency of ctas_per_sm CTAs per SM, and the kernel
// attribute for it (set at plan time, outside any stream capture).
static int prepare_gram(BatchPlan* p) {
    RgKernel kern = rg_pick(p->g.model, p->prec);
    size_t smem = 1024 + TC_STAGES * RCfg::STAGE_BYTES + sizeof(RgShared);
    int dev = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    size_t want = (size_t)per_sm / (size_t)(p->ctas_per_sm + 1) + 1024;
    if (want > smem) smem = want;
    p->smem = smem;
    return cuda_status(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                       "ragged attribute");
}

static int run_gram(BatchPlan* p, const double* users, double* gram, cudaStream_t st) {
    RgKernel kern = rg_pick(p->g.model, p->prec);
    const size_t smem = p->smem;
    int rc = cuda_status(cudaMemsetAsync(p->d_counter, 0, sizeof(int), st), "work counter reset");
    if (rc) return rc;
    int grid = std::min(p->n_items, num_sms() * p->ctas_per_sm);
    if (grid < 1) return XLMIMO_OK;
    kern<<<grid, TC_THREADS, smem, st>>>(p->g, make_gen_params(p->g), p->d_inst, p->d_items, p->n_items, p->d_counter,
                                         users, (double2*)gram, p->d_part);
    rc = cuda_status(cudaGetLastError(), "ragged gram launch");
    if (!rc && p->n_split > 0) {
        ragged_reduce_kernel<<<p->n_split, 256, 0, st>>>(p->d_inst, p->d_lists + p->n_small + p->n_large, p->n_split,
                                                         p->d_part, (double2*)gram);
        rc = cuda_status(cudaGetLastError(), "ragged reduce launch");
    }
    return rc;
}

}  // namespace xl

using namespace xl;

struct xlmimo_batch_plan_st {
    BatchPlan p;
};

extern "C" int xlmimo_batch_plan_create(const xlmimo_array* geo, const xlmimo_inst* insts, int count, int prec,
                                        const double* tune_users, xlmimo_batch_plan* plan, void* stream) {
    clear_error();
    if (!geo || !insts || !plan || count < 1) { set_error("geo, insts and plan must be given and count >= 1"); return XLMIMO_EINVAL; }
    if (prec != XLMIMO_BF16 && prec != XLMIMO_BF16X3 && prec != XLMIMO_F16X3) {
        set_error("batched plans use a tensor-core precision (XLMIMO_BF16, XLMIMO_BF16X3, XLMIMO_F16X3)");
        return XLMIMO_EINVAL;
    }
    xlmimo_array a = *geo;
    a.n_ant = 1;
    Geom g;
    int rc = check_array(&a, &g);
    if (rc) return rc;
    int64_t users_total = 0;
    for (int i = 0; i < count; ++i) {
        const xlmimo_inst& h = insts[i];
        if (h.n_ant < 1 || h.n_ant > (int64_t(1) << 40) || h.k < 1 || h.k > XLMIMO_MAX_USERS || h.scheme < XLMIMO_ZF ||
            h.scheme > XLMIMO_MRC || !(h.noise > 0.0) || h.user_off < 0 || h.gram_off < 0) {
            set_error("instance %d is invalid", i);
            return XLMIMO_EINVAL;
        }
        users_total = std::max<int64_t>(users_total, h.user_off + h.k);
    }
    int dev = 0, major = 0, minor = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3) { set_error("batched plans need an sm_103 device (tcgen05)"); return XLMIMO_EUNSUPPORTED; }
    xlmimo_batch_plan_st* h = new xlmimo_batch_plan_st;
    BatchPlan* p = &h->p;
    p->g = g;
    p->prec = prec;
    p->count = count;
    p->users_total = users_total;
    p->host.assign(insts, insts + count);
    cudaStream_t st = as_stream(stream);
    // element chunk per work item: the tensor cores' FP32 accumulation rounds
    // towards zero, so a chunk's sum loses up to ~chunk x 2^-24 of itself;
    // chunks of a few thousand elements keep that near 1e-5 even when an
    // instance's far elements add many small terms to a large sum
    int64_t best_chunk = 8192;
    int best_ctas = 2;
    if (tune_users) {
        // time the candidate tilings on the given users (Gram phase only)
        int64_t gram_total = 0;
        for (int i = 0; i < count; ++i) gram_total = std::max<int64_t>(gram_total, insts[i].gram_off + (int64_t)insts[i].k * insts[i].k);
        double* scratch = nullptr;
        rc = cuda_status(cudaMalloc((void**)&scratch, (size_t)gram_total * sizeof(double2)), "tuning scratch");
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (!rc) rc = cuda_status(cudaEventCreate(&e0), "tuning event");
        if (!rc) rc = cuda_status(cudaEventCreate(&e1), "tuning event");
        float best = 1e30f;
        const int64_t chunks[3] = {4096, 8192, 16384};
        for (int ci = 0; ci < 3 && !rc; ++ci) {
            rc = build_tables(p, chunks[ci], st);
            for (int cp = 1; cp <= 2 && !rc; ++cp) {
                p->ctas_per_sm = cp;
                rc = prepare_gram(p);
                if (!rc) rc = run_gram(p, tune_users, scratch, st);  // warm
                if (!rc) rc = cuda_status(cudaEventRecord(e0, st), "tuning");
                if (!rc) rc = run_gram(p, tune_users, scratch, st);
                if (!rc) rc = cuda_status(cudaEventRecord(e1, st), "tuning");
                if (!rc) rc = cuda_status(cudaEventSynchronize(e1), "tuning");
                float ms = 0.f;
                if (!rc) cudaEventElapsedTime(&ms, e0, e1);
                if (!rc && ms < best) {
                    best = ms;
                    best_chunk = chunks[ci];
                    best_ctas = cp;
                }
                p->candidates += 1;
            }
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaFree(scratch);
        p->tuned = rc ? 0 : 1;
    }
    if (!rc) {
        p->ctas_per_sm = best_ctas;
        rc = build_tables(p, best_chunk, st);
    }
    if (!rc) rc = prepare_gram(p);
    if (!rc) rc = beamform_ragged_prepare();
    if (rc) {
        free_tables(p);
        delete h;
        return rc;
    }
    *plan = h;
    return XLMIMO_OK;
}

extern "C" int xlmimo_batch_run(xlmimo_batch_plan plan, const double* users, const double* power, int power_mode,
                                double* gram, double* sinr, int32_t* status, double* rate, void* stream) {
    clear_error();
    if (!plan || !users || !power || !gram || !sinr || !status || !rate) {
        set_error("plan and all arrays must be non-NULL");
        return XLMIMO_EINVAL;
    }
    if (power_mode != XLMIMO_POWER_ABS && power_mode != XLMIMO_POWER_RXSNR) { set_error("unknown power mode"); return XLMIMO_EINVAL; }
    BatchPlan* p = &plan->p;
    cudaStream_t st = as_stream(stream);
    int rc = run_gram(p, users, gram, st);
    if (!rc && p->n_small > 0)
        beamform_trial_launch_bucket(p->d_inst, p->d_lists, p->n_small, 32, gram, power, power_mode, sinr, status, st);
    if (!rc && p->n_large > 0)
        beamform_trial_launch_bucket(p->d_inst, p->d_lists + p->n_small, p->n_large, 64, gram, power, power_mode, sinr,
                                     status, st);
    if (!rc) rc = cuda_status(cudaGetLastError(), "ragged receivers");
    if (!rc) {
        int blocks = std::min((p->count + 255) / 256, 16 * num_sms());
        ragged_sumrate_kernel<<<blocks, 256, 0, st>>>(p->d_inst, p->count, sinr, rate);
        rc = cuda_status(cudaGetLastError(), "ragged sumrate");
    }
    return rc;
}

extern "C" int xlmimo_batch_plan_info(xlmimo_batch_plan plan, int64_t* info) {
    clear_error();
    if (!plan || !info) { set_error("plan and info must be non-NULL"); return XLMIMO_EINVAL; }
    const BatchPlan* p = &plan->p;
    info[0] = p->n_items;
    info[1] = p->chunk;
    info[2] = p->ctas_per_sm;
    info[3] = p->n_small;
    info[4] = p->n_large;
    info[5] = (int64_t)p->part_bytes;
    info[6] = p->tuned;
    info[7] = p->candidates;
    return XLMIMO_OK;
}

extern "C" int xlmimo_batch_plan_destroy(xlmimo_batch_plan plan) {
    clear_error();
    if (!plan) return XLMIMO_OK;
    cudaDeviceSynchronize();
    free_tables(&plan->p);
    delete plan;
    return XLMIMO_OK;
}
