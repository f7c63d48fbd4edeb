// Ragged batches: many instances with their own N, K, receiver and noise
// in a few launches: per-user set-up, the tensor-core Gram of every work
// item, the partial-sum reduction of split instances, and the ragged
// receiver / rate launches.
//
// Work items are (instance, element chunk) pairs.  Items of instances with
// K up to the plan's narrow cut-off (at most 32) run the narrow layout of
// gram_engine.cuh (M = 128, N = 64 MMAs, 32 user lanes, three CTAs per SM),
// the others the wide one (M = N = 128, 64 user slots, two CTAs per SM),
// each list ordered longest first so that the block scheduler hands out the
// long items first.  Items share CTAs: a narrow item rides in the spare user
// slots of a wide CTA (64 - K of them, generated as padding otherwise) or
// shares a narrow CTA's 32 lanes with others, when the user counts fit and
// its length lies within PACK_LEN_RATIO of the CTA's longest (the
// accumulator's blocks between members are computed and dropped), since
// channel generation costs per user slot whatever the instance's K.  Every user's position is taken
// relative to its own instance's first element (y + (N - 1) d / 2 for the
// spherical models, the range shifted along the planar wave's direction for
// UPW), so lanes of instances with different N share one array geometry.
// Items that cover a whole instance write its Gram directly; the chunks of a
// split instance write partial Gram matrices that ragged_reduce_kernel sums
// in chunk order.  The receivers run one CTA per instance, launched per user
// count bucket (K up to 16, 32, 40, 48, 56, 64) so that shared memory, and
// with it the CTAs per SM, is sized for the bucket.
#include <limits.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "gram_engine.cuh"

namespace xl {

// A work item (host-side planning).
struct DevItem {
    int inst, chunk;
    long long n0, n1;
};

// A Gram CTA: members [m0, m0 + nm) of the member list, the longest
// member's element count, over which its stages run.
struct DevPack {
    int m0, nm;
    long long len;
};

// One work item inside a CTA: its users occupy user slots lane0 ..
// lane0 + K - 1.
struct DevMember {
    int inst, chunk;
    long long n0, n1;
    int lane0, pad;
};

// An item joins a CTA whose longest item is at most 1/PACK_LEN_RATIO times
// its own length (the slots of the shorter one generate zeros for the rest);
// larger gaps start a CTA of their own.
constexpr double PACK_LEN_RATIO = 0.75;
// A new narrow item is tried against the most recently opened CTAs only.
constexpr int PACK_WINDOW = 64;

// Per-user set-up of a whole ragged batch, once per run (one warp per
// instance), which the Gram CTAs of the instance's items then load.
// iflags[i]: bit 0 an invalid user, bit 1 a user too close for the slice
// expansion.
struct RgUser {
    UserGeo ug;
    double fac;
};

template <int MODEL, int PREC>
__global__ void ragged_user_kernel(Geom g, GenParams gp, const DevInst* __restrict__ insts, int count,
                                   const double* __restrict__ users, RgUser* __restrict__ out, int* __restrict__ iflags) {
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (warp >= count) return;
    const DevInst in = insts[warp];
    int flags = 0;
    // element n of the instance lies at n d - off along the array
    const double off = 0.5 * (double)(in.n_ant - 1) * g.spacing;
    for (int k = lane; k < in.k; k += 32) {
        const double x = users[(in.user_off + k) * 2], y = users[(in.user_off + k) * 2 + 1];
        UserSetup u = user_setup<MODEL, PREC, false>(g, gp, x, y, true);
        if (u.ug.ok) {
            if (MODEL == XLMIMO_UPW) {
                const double r0 = sqrt(x * x + y * y);
                u.ug.r0u = ff_from_double(r0 + off * (y / r0));
            } else {
                u.ug.y = ff_from_double(y + off);
            }
        }
        out[in.user_off + k] = RgUser{u.ug, u.fac};
        flags |= (u.bad ? 1 : 0) | (u.near ? 2 : 0);
    }
    flags = __reduce_or_sync(0xffffffffu, flags);
    if (lane == 0) iflags[warp] = flags;
}

// One CTA of either layout (KMAX user slots: 32 narrow, 64 wide): work items
// side by side in the user slots, each slot over its own item's elements;
// the accumulator is folded once and every member's diagonal block is written
// to its instance's Gram (or chunk partial).  A member with an invalid user
// gets NaN; a member with a user too close for the slice expansion takes the
// whole CTA to the exact per-entry formula.
template <int MODEL, int KMAX, int PREC>
__global__ void __launch_bounds__(TC_THREADS, KMAX == 32 ? 3 : 2)
    gram_tc_packed_kernel(Geom g, GenParams gp, const DevInst* __restrict__ insts, const DevPack* __restrict__ packs,
                          const DevMember* __restrict__ members, const RgUser* __restrict__ users,
                          const int* __restrict__ iflags, double2* __restrict__ gram, double2* __restrict__ part) {
    constexpr int NRING = KMAX == 32 ? 2 : 3;
    using E = GramEngine<MODEL, KMAX, PREC, false, NRING>;
    using SH = EngShared<KMAX, NRING>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    SH* sh = reinterpret_cast<SH*>(base + NRING * E::BYTES);
    float* fold = reinterpret_cast<float*>(base);
    __shared__ long long lane_n0[KMAX];
    __shared__ int lane_len[KMAX];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const DevPack pk = packs[blockIdx.x];
    if (tid == 0) {
        eng_init_barriers(sh);
        int near = 0;
        for (int m = 0; m < pk.nm; ++m) near |= (iflags[members[pk.m0 + m].inst] >> 1) & 1;
        sh->bad = 0;
        sh->near = near;
    }
    if (tid < KMAX) {
        int mi = -1;
        for (int m = 0; m < pk.nm; ++m) {
            const DevMember mb = members[pk.m0 + m];
            if (tid >= mb.lane0 && tid < mb.lane0 + insts[mb.inst].k) mi = m;
        }
        if (mi >= 0) {
            const DevMember mb = members[pk.m0 + mi];
            const RgUser u = users[insts[mb.inst].user_off + (tid - mb.lane0)];
            sh->ug[tid] = u.ug;
            sh->fac[tid] = u.fac;
            lane_n0[tid] = mb.n0;
            lane_len[tid] = (int)(mb.n1 - mb.n0);
        } else {
            // padding user (1, 0), weight 0, over the longest member's range so
            // that its slot takes the same path through each stage as the others
            UserGeo pad = make_user_geo(g, 1.0, 0.0);
            pad.ampc = 0.f;
            sh->ug[tid] = pad;
            sh->fac[tid] = 1.0;
            lane_n0[tid] = 0;
            lane_len[tid] = (int)pk.len;
        }
    }
    __syncthreads();
    if (warp == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh->tmem_base)),
                     "r"(2 * E::WCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh->tmem_base;
    const int nst = E::stages(0, pk.len);
    if (warp < 8) {
        E::template generate<SH, true>(sh, smem_u32(base), tmem, g, gp, 0, pk.len, UraRows{0, 0.0, 0.0, 0}, 0, 0, 0,
                                       !sh->near, lane_n0, lane_len);
    } else {
        if (lane == 0) E::mma(sh, smem_u32(base), tmem, nst, 0, 0);
        __syncwarp();
    }
    bool ok = mbar_wait(&sh->done, 0, &sh->abort);
    tc_fence_before();
    __syncthreads();  // every MMA done and every drain's tcgen05.st complete
    tc_fence_after();
    ok = ok && !*(volatile int*)&sh->abort;
    E::epilogue_fold(fold, tmem, E::drains(nst), ok, warp, lane);
    for (int m = 0; m < pk.nm; ++m) {
        const DevMember mb = members[pk.m0 + m];
        const DevInst in = insts[mb.inst];
        double2* o = in.nchunks == 1 ? gram + in.gram_off : part + in.part_off + (long long)mb.chunk * in.k * in.k;
        E::epilogue_write(sh, fold, in.k, mb.lane0, ok && !(iflags[mb.inst] & 1), o, tid);
    }
    __syncthreads();
    if (warp == 8) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * E::WCOLS) : "memory");
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
// Receiver buckets: instances grouped by user count, each bucket launched with
// shared memory for its largest K ((2 K^2 + K) 16 bytes): K <= 64 alone would
// hold one CTA per SM.
constexpr int RG_BUCKETS[6] = {16, 32, 40, 48, 56, 64};

struct BatchPlan {
    Geom g;
    int prec = XLMIMO_BF16X3;
    int count = 0;
    int64_t users_total = 0;
    std::vector<xlmimo_inst> host;
    DevInst* d_inst = nullptr;
    DevPack* d_packs = nullptr;     // the wide CTAs, then the narrow ones, each longest first
    DevMember* d_members = nullptr; // their work items
    int* d_lists = nullptr;  // [receiver buckets by K (RG_BUCKETS) | split instances]
    double2* d_part = nullptr;
    RgUser* d_users = nullptr;  // per-user set-up, rewritten by every run
    int* d_iflags = nullptr;    // per-instance flags, rewritten by every run
    int n_items = 0, n_wide = 0, n_small = 0, n_large = 0, n_split = 0;  // n_wide: CTAs of the wide tiling
    int n_bucket[6] = {0, 0, 0, 0, 0, 0};  // instances per receiver bucket
    int64_t chunk = 0;
    int narrow_kmax = 32;  // largest K on the narrow tile (0: every item on the wide one)
    int pack = 1;          // narrow items share CTAs (else one per CTA)
    int n_packs = 0;       // narrow CTAs
    int mode = 2;  // 1: the two layouts one after the other; 2: concurrently on two streams
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    size_t part_bytes = 0;
    int tuned = 0, candidates = 0;
    size_t smem = 0;
};



static void release_streams(BatchPlan* p) {
    if (p->side) cudaStreamDestroy(p->side);
    if (p->fork) cudaEventDestroy(p->fork);
    if (p->join) cudaEventDestroy(p->join);
    p->side = nullptr;
    p->fork = p->join = nullptr;
}

static void free_tables(BatchPlan* p) {
    cudaFree(p->d_inst);
    cudaFree(p->d_packs);
    cudaFree(p->d_members);
    cudaFree(p->d_lists);
    cudaFree(p->d_part);
    cudaFree(p->d_users);
    cudaFree(p->d_iflags);
    p->d_inst = nullptr;
    p->d_packs = nullptr;
    p->d_members = nullptr;
    p->d_lists = nullptr;
    p->d_part = nullptr;
    p->d_users = nullptr;
    p->d_iflags = nullptr;
}

// Host tables for one element chunk: items longest first, split instances'
// partial offsets, receiver buckets.
static int build_tables_impl(BatchPlan* p, int64_t chunk, cudaStream_t st) {
    free_tables(p);
    // work items, chunk indices and CTA counts are 32-bit
    long long total_items = 0;
    for (int i = 0; i < p->count; ++i) total_items += (p->host[i].n_ant + chunk - 1) / chunk;
    if (total_items > INT_MAX) {
        set_error("%lld work items at an element chunk of %lld exceed 2^31 - 1: take a longer chunk", total_items,
                  (long long)chunk);
        return XLMIMO_EINVAL;
    }
    std::vector<DevInst> di(p->count);
    std::vector<DevItem> items;
    std::vector<int> small, large, split, buckets[6];
    long long part = 0;
    for (int i = 0; i < p->count; ++i) {
        const xlmimo_inst& h = p->host[i];
        DevInst d;
        d.n_ant = h.n_ant;
        d.k = h.k;
        // the receivers factor in double-float, in FP64 for an ill-conditioned system
        d.scheme = h.scheme | XLMIMO_FACTOR_FF;
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
        int bk = 0;
        while (RG_BUCKETS[bk] < h.k) ++bk;
        buckets[bk].push_back(i);
        di[i] = d;
    }
    // all items longest first, so that a CTA's first member is its longest.
    // An item with K above the narrow cut-off opens a wide CTA (64 user
    // slots); any other item goes to the most recent CTA (of the last
    // PACK_WINDOW: the shortest) with slots to spare and a length within
    // PACK_LEN_RATIO of it, a wide CTA's spare slots first (they are generated
    // as padding anyway), else opens a narrow CTA (32 slots).  Without packing
    // every item opens a CTA of its own kind.
    const int nk = p->narrow_kmax;
    std::stable_sort(items.begin(), items.end(),
                     [&](const DevItem& a, const DevItem& b) { return a.n1 - a.n0 > b.n1 - b.n0; });
    p->n_items = (int)items.size();
    struct Bin {
        std::vector<DevMember> m;
        int used, cap;
        long long len;
    };
    std::vector<Bin> bins;
    for (const DevItem& it : items) {
        const int k = p->host[it.inst].k;
        const long long len = it.n1 - it.n0;
        const bool wide = k > nk;
        int b = -1;
        if (p->pack)
            for (int pass = 0; pass < 2 && b < 0; ++pass)  // wide CTAs first
                for (int c = (int)bins.size() - 1; c >= 0 && c >= (int)bins.size() - PACK_WINDOW; --c) {
                    const Bin& x = bins[c];
                    if ((x.cap == 64) != (pass == 0) || (wide && x.cap != 64)) continue;
                    if (x.used + k <= x.cap && (double)len >= PACK_LEN_RATIO * (double)x.len) {
                        b = c;
                        break;
                    }
                }
        if (b < 0) {
            bins.push_back(Bin{{}, 0, wide ? 64 : 32, len});
            b = (int)bins.size() - 1;
        }
        DevMember m;
        m.inst = it.inst;
        m.chunk = it.chunk;
        m.n0 = it.n0;
        m.n1 = it.n1;
        m.lane0 = bins[b].used;
        m.pad = 0;
        bins[b].m.push_back(m);
        bins[b].used += k;
    }
    // the wide CTAs, then the narrow ones, each in the order opened (longest first)
    std::vector<DevPack> packs;
    std::vector<DevMember> members;
    for (int cap : {64, 32})
        for (const Bin& x : bins)
            if (x.cap == cap) {
                DevPack pk;
                pk.m0 = (int)members.size();
                pk.nm = (int)x.m.size();
                pk.len = x.len;
                packs.push_back(pk);
                members.insert(members.end(), x.m.begin(), x.m.end());
            }
    p->n_wide = (int)std::count_if(bins.begin(), bins.end(), [](const Bin& x) { return x.cap == 64; });
    p->n_packs = (int)packs.size() - p->n_wide;
    p->n_small = (int)small.size();
    p->n_large = (int)large.size();
    p->n_split = (int)split.size();
    p->chunk = chunk;
    p->part_bytes = (size_t)part * sizeof(double2);
    std::vector<int> lists;
    for (int b = 0; b < 6; ++b) {
        // larger K first inside a bucket (longer receivers start early)
        std::stable_sort(buckets[b].begin(), buckets[b].end(),
                         [&](int x, int y) { return p->host[x].k > p->host[y].k; });
        p->n_bucket[b] = (int)buckets[b].size();
        lists.insert(lists.end(), buckets[b].begin(), buckets[b].end());
    }
    lists.insert(lists.end(), split.begin(), split.end());
    int rc = cuda_status(cudaMalloc((void**)&p->d_inst, sizeof(DevInst) * di.size()), "plan tables");
    if (!rc) rc = cuda_status(cudaMalloc((void**)&p->d_packs, sizeof(DevPack) * std::max<size_t>(1, packs.size())), "plan tables");
    if (!rc) rc = cuda_status(cudaMalloc((void**)&p->d_members, sizeof(DevMember) * std::max<size_t>(1, members.size())), "plan tables");
    if (!rc) rc = cuda_status(cudaMalloc((void**)&p->d_users, sizeof(RgUser) * std::max<int64_t>(1, p->users_total)),
                              "plan tables");
    if (!rc) rc = cuda_status(cudaMalloc((void**)&p->d_iflags, sizeof(int) * p->count), "plan tables");
    if (!rc) rc = cuda_status(cudaMalloc((void**)&p->d_lists, sizeof(int) * std::max<size_t>(1, lists.size())), "plan tables");
    if (!rc && part > 0) rc = cuda_status(cudaMalloc((void**)&p->d_part, p->part_bytes), "plan workspace");
    if (!rc) rc = cuda_status(cudaMemcpyAsync(p->d_inst, di.data(), sizeof(DevInst) * di.size(), cudaMemcpyHostToDevice, st), "plan upload");
    if (!rc && !packs.empty())
        rc = cuda_status(cudaMemcpyAsync(p->d_packs, packs.data(), sizeof(DevPack) * packs.size(), cudaMemcpyHostToDevice, st), "plan upload");
    if (!rc && !members.empty())
        rc = cuda_status(cudaMemcpyAsync(p->d_members, members.data(), sizeof(DevMember) * members.size(), cudaMemcpyHostToDevice, st),
                         "plan upload");
    if (!rc && !lists.empty())
        rc = cuda_status(cudaMemcpyAsync(p->d_lists, lists.data(), sizeof(int) * lists.size(), cudaMemcpyHostToDevice, st), "plan upload");
    if (!rc) rc = cuda_status(cudaStreamSynchronize(st), "plan upload");
    return rc;
}

// The host tables are built before any device table is allocated, so a host
// allocation failure leaves the plan without tables (which run refuses) and
// is reported instead of unwinding through the C interface.
static int build_tables(BatchPlan* p, int64_t chunk, cudaStream_t st) {
    try {
        return build_tables_impl(p, chunk, st);
    } catch (const std::bad_alloc&) {
        free_tables(p);
        set_error("plan tables: host memory exhausted");
        return XLMIMO_ENOMEM;
    }
}

using RuKernel = void (*)(Geom, GenParams, const DevInst*, int, const double*, RgUser*, int*);

template <int MODEL>
static RuKernel ru_pick_prec(int prec) {
    return prec == XLMIMO_F16X3 ? ragged_user_kernel<MODEL, TCP_F16X3> : ragged_user_kernel<MODEL, TCP_BF16X3>;
}

static RuKernel ru_pick(int model, int prec) {
    return model == XLMIMO_PNUSW ? ru_pick_prec<XLMIMO_PNUSW>(prec)
         : model == XLMIMO_UPW   ? ru_pick_prec<XLMIMO_UPW>(prec)
                                 : ru_pick_prec<XLMIMO_FSPL_USW>(prec);
}

using RpKernel = void (*)(Geom, GenParams, const DevInst*, const DevPack*, const DevMember*, const RgUser*, const int*,
                          double2*, double2*);

template <int MODEL, int KMAX>
static RpKernel rp_pick_prec(int prec) {
    return prec == XLMIMO_BF16 ? gram_tc_packed_kernel<MODEL, KMAX, TCP_BF16>
         : prec == XLMIMO_F16X3 ? gram_tc_packed_kernel<MODEL, KMAX, TCP_F16X3>
                                : gram_tc_packed_kernel<MODEL, KMAX, TCP_BF16X3>;
}

// the Gram kernel of the narrow (KMAX = 32) or the wide (64) tiling
template <int KMAX>
static RpKernel rp_pick(int model, int prec) {
    return model == XLMIMO_PNUSW ? rp_pick_prec<XLMIMO_PNUSW, KMAX>(prec)
         : model == XLMIMO_UPW   ? rp_pick_prec<XLMIMO_UPW, KMAX>(prec)
                                 : rp_pick_prec<XLMIMO_FSPL_USW, KMAX>(prec);
}

template <int KMAX>
static size_t items_smem() {
    constexpr int NRING = KMAX == 32 ? 2 : 3;
    return 1024 + NRING * GramEngine<XLMIMO_FSPL_USW, KMAX, TCP_BF16X3, false, NRING>::BYTES +
           sizeof(EngShared<KMAX, NRING>);
}

// Kernel attributes and the second stream of the concurrent mode (at plan
// time, outside any stream capture).
static int prepare_gram(BatchPlan* p) {
    int rc = cuda_status(cudaFuncSetAttribute(rp_pick<32>(p->g.model, p->prec),
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)items_smem<32>()),
                         "ragged attribute");
    if (!rc) rc = cuda_status(cudaFuncSetAttribute(rp_pick<64>(p->g.model, p->prec),
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)items_smem<64>()),
                              "ragged attribute");
    if (!rc && !p->side) rc = cuda_status(cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking), "plan stream");
    if (!rc && !p->fork) rc = cuda_status(cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming), "plan event");
    if (!rc && !p->join) rc = cuda_status(cudaEventCreateWithFlags(&p->join, cudaEventDisableTiming), "plan event");
    return rc;
}

// The Gram matrices of a run: per-user set-up, then the wide items (K above
// the narrow cut-off) and the narrow ones, one CTA per item; mode 1 launches the two layouts one
// after the other on `st`, mode 2 the narrow ones on the plan's second stream
// so that the two launches share the GPU (a fork and a join by events).
static int run_gram(BatchPlan* p, const double* users, double* gram, cudaStream_t st) {
    if (p->n_items < 1) return XLMIMO_OK;
    const GenParams gp = make_gen_params(p->g);
    ru_pick(p->g.model, p->prec)<<<(p->count + 7) / 8, 256, 0, st>>>(p->g, gp, p->d_inst, p->count, users, p->d_users,
                                                                      p->d_iflags);
    int rc = cuda_status(cudaGetLastError(), "ragged user set-up launch");
    if (rc) return rc;
    const int n_narrow = p->n_packs;
    cudaStream_t sn = st;
    if (p->mode == 2 && n_narrow > 0 && p->n_wide > 0) {
        rc = cuda_status(cudaEventRecord(p->fork, st), "plan fork");
        if (!rc) rc = cuda_status(cudaStreamWaitEvent(p->side, p->fork, 0), "plan fork");
        if (rc) return rc;
        sn = p->side;
    }
    if (p->n_wide > 0)
        rp_pick<64>(p->g.model, p->prec)<<<p->n_wide, TC_THREADS, items_smem<64>(), st>>>(
            p->g, gp, p->d_inst, p->d_packs, p->d_members, p->d_users, p->d_iflags, (double2*)gram, p->d_part);
    if (n_narrow > 0)
        rp_pick<32>(p->g.model, p->prec)<<<n_narrow, TC_THREADS, items_smem<32>(), sn>>>(
            p->g, gp, p->d_inst, p->d_packs + p->n_wide, p->d_members, p->d_users, p->d_iflags, (double2*)gram,
            p->d_part);
    rc = cuda_status(cudaGetLastError(), "ragged gram launch");
    if (!rc && sn != st) {
        rc = cuda_status(cudaEventRecord(p->join, sn), "plan join");
        if (!rc) rc = cuda_status(cudaStreamWaitEvent(st, p->join, 0), "plan join");
    }
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
    xlmimo_batch_plan_st* h = new (std::nothrow) xlmimo_batch_plan_st;
    if (!h) { set_error("plan: host memory exhausted"); return XLMIMO_ENOMEM; }
    BatchPlan* p = &h->p;
    p->g = g;
    p->prec = prec;
    p->count = count;
    p->users_total = users_total;
    try {
        p->host.assign(insts, insts + count);
    } catch (const std::bad_alloc&) {
        delete h;
        set_error("plan: host memory exhausted");
        return XLMIMO_ENOMEM;
    }
    cudaStream_t st = as_stream(stream);
    // element chunk per work item (the accumulator's periodic drain keeps
    // any chunk length accurate; the chunk trades load balance against
    // partial sums)
    int64_t best_chunk = 8192;
    int best_mode = 2, best_nk = 32, best_pack = 1;
    if (tune_users) {
        // time candidate tilings on the given users (Gram phase only), in two
        // stages: element chunk x launch mode with K <= 32 on the narrow tile
        // and narrow items packed, then, at the best of those, the narrow
        // tile's cut-off (K <= 16 or no instance on it: the wide M = N = 128
        // tile for the rest) and one narrow item per CTA
        int64_t gram_total = 0;
        for (int i = 0; i < count; ++i) gram_total = std::max<int64_t>(gram_total, insts[i].gram_off + (int64_t)insts[i].k * insts[i].k);
        double* scratch = nullptr;
        rc = cuda_status(cudaMalloc((void**)&scratch, (size_t)gram_total * sizeof(double2)), "tuning scratch");
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (!rc) rc = cuda_status(cudaEventCreate(&e0), "tuning event");
        if (!rc) rc = cuda_status(cudaEventCreate(&e1), "tuning event");
        float best = 1e30f;
        auto trial = [&](int64_t chunk, int nk, int md, int pk) {
            p->narrow_kmax = nk;
            p->pack = pk;
            rc = build_tables(p, chunk, st);
            if (!rc) rc = prepare_gram(p);
            p->mode = md;
            if (!rc) rc = run_gram(p, tune_users, scratch, st);  // warm
            if (!rc) rc = cuda_status(cudaEventRecord(e0, st), "tuning");
            if (!rc) rc = run_gram(p, tune_users, scratch, st);
            if (!rc) rc = cuda_status(cudaEventRecord(e1, st), "tuning");
            if (!rc) rc = cuda_status(cudaEventSynchronize(e1), "tuning");
            float ms = 0.f;
            if (!rc) cudaEventElapsedTime(&ms, e0, e1);
            if (!rc && ms < best) {
                best = ms;
                best_chunk = chunk;
                best_mode = md;
                best_nk = nk;
                best_pack = pk;
            }
            p->candidates += 1;
        };
        const int64_t chunks[5] = {4096, 8192, 16384, 32768, 131072};
        for (int ci = 0; ci < 5 && !rc; ++ci)
            for (int md = 1; md <= 2 && !rc; ++md) trial(chunks[ci], 32, md, 1);
        const int64_t c1 = best_chunk;
        const int m1 = best_mode;
        for (int nk : {16, 0})
            if (!rc) trial(c1, nk, m1, 1);
        if (!rc) trial(c1, 32, m1, 0);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaFree(scratch);
        p->tuned = rc ? 0 : 1;
    }
    if (!rc) {
        p->mode = best_mode;
        p->narrow_kmax = best_nk;
        p->pack = best_pack;
        rc = build_tables(p, best_chunk, st);
    }
    if (!rc) rc = prepare_gram(p);
    if (!rc) rc = beamform_ragged_prepare();
    if (rc) {
        free_tables(p);
        release_streams(p);
        delete h;
        return rc;
    }
    *plan = h;
    return XLMIMO_OK;
}

extern "C" int xlmimo_batch_run(xlmimo_batch_plan plan, const double* users, const double* power, int power_mode,
                                double* gram, double* sinr, int32_t* status, double* rate, void* stream) {
    clear_error();
    const bool gram_only = !sinr && !status && !rate;
    if (!plan || !users || !gram || (!gram_only && (!power || !sinr || !status || !rate))) {
        set_error("plan, users and gram must be non-NULL, and power, sinr, status and rate all given or sinr, status "
                  "and rate all NULL");
        return XLMIMO_EINVAL;
    }
    if (power_mode != XLMIMO_POWER_ABS && power_mode != XLMIMO_POWER_RXSNR) { set_error("unknown power mode"); return XLMIMO_EINVAL; }
    BatchPlan* p = &plan->p;
    if (!p->d_inst) { set_error("the plan has no tables: its last xlmimo_batch_plan_set_tiling failed"); return XLMIMO_EINVAL; }
    cudaStream_t st = as_stream(stream);
    int rc = run_gram(p, users, gram, st);
    if (rc || gram_only) return rc;
    for (int b = 0, off = 0; b < 6; off += p->n_bucket[b], ++b)
        if (p->n_bucket[b] > 0)
            beamform_trial_launch_bucket(p->d_inst, p->d_lists + off, p->n_bucket[b], RG_BUCKETS[b], gram, power,
                                         power_mode, sinr, status, st);
    rc = cuda_status(cudaGetLastError(), "ragged receivers");
    if (!rc) {
        int blocks = std::min((p->count + 255) / 256, 16 * num_sms());
        ragged_sumrate_kernel<<<blocks, 256, 0, st>>>(p->d_inst, p->count, sinr, rate);
        rc = cuda_status(cudaGetLastError(), "ragged sumrate");
    }
    return rc;
}

extern "C" int xlmimo_batch_plan_set_tiling(xlmimo_batch_plan plan, int64_t chunk, int mode, int narrow_kmax,
                                            int pack, void* stream) {
    clear_error();
    if (!plan) { set_error("plan must be non-NULL"); return XLMIMO_EINVAL; }
    if (chunk < 128 || chunk % 128 != 0 || chunk > (int64_t(1) << 30) || (mode != 1 && mode != 2) || narrow_kmax < 0 ||
        narrow_kmax > 32 || (pack != 0 && pack != 1)) {
        set_error("tiling: chunk a positive multiple of 128 up to 2^30, mode 1 or 2, narrow cut-off in [0, 32], pack 0 or 1");
        return XLMIMO_EINVAL;
    }
    BatchPlan* p = &plan->p;
    // runs in flight may still read the tables that are rebuilt
    int rc = cuda_status(cudaDeviceSynchronize(), "tiling");
    if (rc) return rc;  // the plan is left as it was
    p->narrow_kmax = narrow_kmax;
    p->pack = pack;
    p->mode = mode;
    p->tuned = 0;
    rc = build_tables(p, chunk, as_stream(stream));
    if (!rc) rc = prepare_gram(p);
    return rc;
}

extern "C" int xlmimo_batch_plan_info(xlmimo_batch_plan plan, int64_t* info) {
    clear_error();
    if (!plan || !info) { set_error("plan and info must be non-NULL"); return XLMIMO_EINVAL; }
    const BatchPlan* p = &plan->p;
    info[0] = p->n_items;
    info[1] = p->chunk;
    info[2] = p->mode;
    info[3] = p->n_small;
    info[4] = p->n_large;
    info[5] = (int64_t)p->part_bytes;
    info[6] = p->tuned;
    info[7] = p->candidates;
    info[8] = p->narrow_kmax;
    info[9] = p->n_wide;
    info[10] = p->pack;
    info[11] = p->n_packs;
    return XLMIMO_OK;
}

extern "C" int xlmimo_batch_plan_destroy(xlmimo_batch_plan plan) {
    clear_error();
    if (!plan) return XLMIMO_OK;
    cudaDeviceSynchronize();
    free_tables(&plan->p);
    release_streams(&plan->p);
    delete plan;
    return XLMIMO_OK;
}
