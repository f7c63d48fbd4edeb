// Ragged batches: many instances with their own N, K, receiver and noise in
// one persistent tensor-core launch plus ragged receiver / rate launches.
//
// Work items are (instance, element chunk) pairs ordered longest first.
// gram_tc_ragged_kernel runs a fixed number of CTAs per SM; each pulls the
// next item from an atomic counter and runs the pipeline of gram_engine.cuh
// on it, in the narrow layout (K <= 32) or the wide one (K <= 64), keeping
// its tensor memory, its ring and its barrier phases across items.  Items
// that cover a whole instance write its Gram directly; the chunks of a split
// instance write partial Gram matrices that ragged_reduce_kernel sums in
// chunk order.  The receivers run one CTA per instance, launched per user
// count bucket so that shared memory is sized for the bucket.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "gram_engine.cuh"

namespace xl {

struct DevItem {
    int inst, chunk;
    long long n0, n1;
};

constexpr int RG_NRING = 3;
using RgShared = EngShared<64, RG_NRING>;

// The current work item as thread 0 claimed it, kept in shared memory so
// that no per-item value occupies registers across the generator loop.
struct RgCur {
    long long n0, n1, n_ant;
    const double* users;  // the instance's users [K][2]
    double2* out;         // its Gram, or this chunk's partial Gram
    int k;
    int valid;
};

// Work items of one layout pulled from `counter` until the list is exhausted
// (E: the layout's engine).  gs / gd / done_count: the CTA's stage, drain and
// item counters, carried across items and lists.  Returns true if a wait
// gave up (the CTA then stops pulling work).
template <class E, class SH>
__device__ __forceinline__ bool ragged_items(SH* sh, RgCur* cur, unsigned char* base, uint32_t tmem, const Geom& g,
                                             const GenParams& gp, const DevInst* __restrict__ insts,
                                             const DevItem* __restrict__ items, int n_items, int* counter,
                                             const double* __restrict__ users, double2* __restrict__ gram,
                                             double2* __restrict__ part, int& gs, int& gd, int& gsp, int& done_count) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int* abort = &sh->abort;
    for (;;) {
        if (tid == 0) {
            const int w = atomicAdd(counter, 1);
            cur->valid = w < n_items;
            if (w < n_items) {
                const DevItem itm = items[w];
                const DevInst in = insts[itm.inst];
                cur->n0 = itm.n0;
                cur->n1 = itm.n1;
                cur->n_ant = in.n_ant;
                cur->users = users + in.user_off * 2;
                cur->out = in.nchunks == 1 ? gram + in.gram_off : part + in.part_off + (long long)itm.chunk * in.k * in.k;
                cur->k = in.k;
            }
            sh->bad = 0;
            sh->near = 0;
        }
        tc_fence_before();
        __syncthreads();  // previous item's epilogue finished with TMEM and the stage buffers
        tc_fence_after();
        if (!cur->valid) return false;
        Geom gi = g;
        gi.N = cur->n_ant;
        GenParams gpi = gp;
        gpi.nm1 = cur->n_ant - 1;
        if (tid < E::KM) E::setup_user(sh, gi, gpi, cur->users, cur->k, tid);
        __syncthreads();
        const int nst = E::stages(cur->n0, cur->n1);
        if (warp < 8) {
            E::generate(sh, smem_u32(base), tmem, gi, gpi, cur->n0, cur->n1, UraRows{0, 0.0, 0.0, 0}, gs, gd, gsp,
                        !sh->near, warp, lane);
        } else {
            if (lane == 0) E::mma(sh, smem_u32(base), tmem, nst, gs, gd);
            __syncwarp();
        }
        gs += nst;
        gd += E::drains(nst);
        gsp += E::spans(nst);
        bool ok = mbar_wait(&sh->done, (uint32_t)(done_count & 1), abort);
        ++done_count;
        tc_fence_before();
        __syncthreads();  // every MMA done and every drain's tcgen05.st complete
        tc_fence_after();
        ok = ok && !*abort && !sh->bad;
        E::epilogue(sh, reinterpret_cast<float*>(base), tmem, cur->k, E::drains(nst), ok, cur->out, tid, warp, lane);
        __syncthreads();
        const int gave_up = *abort;  // read by every thread between two barriers
        __syncthreads();
        if (gave_up) return true;  // outstanding MMAs drained at "done"
    }
}

// Every CTA takes wide items (K > 32, counter[0]) until they are exhausted,
// then narrow ones (counter[1]); both lists are ordered longest first.
template <int MODEL, int PREC>
__global__ void __launch_bounds__(TC_THREADS, 2)
    gram_tc_ragged_kernel(Geom g, GenParams gp, const DevInst* __restrict__ insts, const DevItem* __restrict__ items,
                          int n_wide, int n_narrow, int* __restrict__ counter, const double* __restrict__ users,
                          double2* __restrict__ gram, double2* __restrict__ part) {
    using EN = GramEngine<MODEL, 32, PREC, false, RG_NRING>;  // narrow, K <= 32
    using EW = GramEngine<MODEL, 64, PREC, false, RG_NRING>;  // wide, K <= 64
    static_assert(EN::BYTES == EW::BYTES, "both layouts share the ring");
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    RgShared* sh = reinterpret_cast<RgShared*>(base + RG_NRING * EW::BYTES);
    RgCur* cur = reinterpret_cast<RgCur*>(reinterpret_cast<unsigned char*>(sh) + sizeof(RgShared));

    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) eng_init_barriers(sh);
    __syncthreads();
    if (warp == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh->tmem_base)),
                     "r"(2 * EW::WCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh->tmem_base;
    int gs = 0;          // stages issued by this CTA so far (ring slots and phases run on across items)
    int gd = 0;          // drains so far
    int gsp = 0;         // reference spans so far
    int done_count = 0;  // items completed by this CTA
    if (!ragged_items<EW>(sh, cur, base, tmem, g, gp, insts, items, n_wide, counter, users, gram, part, gs, gd, gsp,
                          done_count))
        ragged_items<EN>(sh, cur, base, tmem, g, gp, insts, items + n_wide, n_narrow, counter + 1, users, gram, part, gs,
                         gd, gsp, done_count);
    __syncthreads();
    if (warp == 8) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * EW::WCOLS) : "memory");
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
    int n_items = 0, n_wide = 0, n_small = 0, n_large = 0, n_split = 0;
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
    // wide items (K > 32) first, then narrow ones, each list longest first
    std::stable_sort(items.begin(), items.end(), [&](const DevItem& a, const DevItem& b) {
        const bool wa = p->host[a.inst].k > 32, wb = p->host[b.inst].k > 32;
        if (wa != wb) return wa;
        return a.n1 - a.n0 > b.n1 - b.n0;
    });
    p->n_items = (int)items.size();
    p->n_wide = (int)std::count_if(items.begin(), items.end(), [&](const DevItem& a) { return p->host[a.inst].k > 32; });
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
    if (!rc) rc = cuda_status(cudaMalloc((void**)&p->d_counter, 2 * sizeof(int)), "plan tables");
    if (!rc) rc = cuda_status(cudaMalloc((void**)&p->d_lists, sizeof(int) * std::max<size_t>(1, lists.size())), "plan tables");
    if (!rc && part > 0) rc = cuda_status(cudaMalloc((void**)&p->d_part, p->part_bytes), "plan workspace");
    if (!rc) rc = cuda_status(cudaMemcpyAsync(p->d_inst, di.data(), sizeof(DevInst) * di.size(), cudaMemcpyHostToDevice, st), "plan upload");
    if (!rc) rc = cuda_status(cudaMemcpyAsync(p->d_items, items.data(), sizeof(DevItem) * items.size(), cudaMemcpyHostToDevice, st), "plan upload");
    if (!rc && !lists.empty())
        rc = cuda_status(cudaMemcpyAsync(p->d_lists, lists.data(), sizeof(int) * lists.size(), cudaMemcpyHostToDevice, st), "plan upload");
    if (!rc) rc = cuda_status(cudaStreamSynchronize(st), "plan upload");
    return rc;
}

using RgKernel = void (*)(Geom, GenParams, const DevInst*, const DevItem*, int, int, int*, const double*, double2*,
                          double2*);

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
    size_t smem = 1024 + RG_NRING * GramEngine<XLMIMO_FSPL_USW, 64, TCP_BF16X3, false, RG_NRING>::BYTES + sizeof(RgShared) +
                  sizeof(RgCur);
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
    int rc = cuda_status(cudaMemsetAsync(p->d_counter, 0, 2 * sizeof(int), st), "work counter reset");
    if (rc) return rc;
    int grid = std::min(p->n_items, num_sms() * p->ctas_per_sm);
    if (grid < 1) return XLMIMO_OK;
    kern<<<grid, TC_THREADS, smem, st>>>(p->g, make_gen_params(p->g), p->d_inst, p->d_items, p->n_wide,
                                         p->n_items - p->n_wide, p->d_counter, users, (double2*)gram, p->d_part);
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
    // element chunk per work item (the accumulator's periodic drain keeps
    // any chunk length accurate; the chunk trades load balance against
    // partial sums)
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
        const int64_t chunks[5] = {4096, 8192, 16384, 32768, 131072};
        for (int ci = 0; ci < 5 && !rc; ++ci) {
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
    const bool gram_only = !sinr && !status && !rate;
    if (!plan || !users || !gram || (!gram_only && (!power || !sinr || !status || !rate))) {
        set_error("plan, users and gram must be non-NULL, and power, sinr, status and rate all given or sinr, status "
                  "and rate all NULL");
        return XLMIMO_EINVAL;
    }
    if (power_mode != XLMIMO_POWER_ABS && power_mode != XLMIMO_POWER_RXSNR) { set_error("unknown power mode"); return XLMIMO_EINVAL; }
    BatchPlan* p = &plan->p;
    cudaStream_t st = as_stream(stream);
    int rc = run_gram(p, users, gram, st);
    if (rc || gram_only) return rc;
    if (p->n_small > 0)
        beamform_trial_launch_bucket(p->d_inst, p->d_lists, p->n_small, 32, gram, power, power_mode, sinr, status, st);
    if (p->n_large > 0)
        beamform_trial_launch_bucket(p->d_inst, p->d_lists + p->n_small, p->n_large, 64, gram, power, power_mode, sinr,
                                     status, st);
    rc = cuda_status(cudaGetLastError(), "ragged receivers");
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
