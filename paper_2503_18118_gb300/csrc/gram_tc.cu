// Exact Gram matrices of a batch of trials on the tensor cores: one CTA per
// (trial, element chunk) running the pipeline of gram_engine.cuh (narrow
// layout for K <= 32 at three CTAs per SM, wide layout for K <= 64 at two).
// Chunks are reduced in FP64 in chunk order when a small batch splits the
// elements to fill the GPU.
#include "gram_engine.cuh"

namespace xl {

template <int KMAX>
struct GtCfg {
    static constexpr int NRING = KMAX == 32 ? 2 : 3;  // what three (two) CTAs per SM leave of shared memory
};

template <int MODEL, int KMAX, int PREC, bool URA>
__global__ void __launch_bounds__(TC_THREADS, KMAX == 32 ? 3 : 2)
    gram_tc_kernel(Geom g, GenParams gp, const double* __restrict__ users, int K, int S, int64_t chunk,
                   double2* __restrict__ out, UraRows ura) {
    static_assert(!URA || PREC == TCP_BF16X3, "the URA mode generates weighted entries for the BF16 hi/lo split");
    constexpr int NRING = GtCfg<KMAX>::NRING;
    using E = GramEngine<MODEL, KMAX, PREC, URA, NRING>;
    using SH = EngShared<KMAX, NRING>;
    extern __shared__ unsigned char smem_raw[];
    // stages must be 1024-byte aligned for the 128-byte swizzle
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    SH* sh = reinterpret_cast<SH*>(base + NRING * E::BYTES);
    float* fold = reinterpret_cast<float*>(base);  // epilogue reuses the stages

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int b = blockIdx.x, s = blockIdx.y;
    if (tid == 0) {
        eng_init_barriers(sh);
        sh->bad = 0;
        sh->near = 0;
    }
    __syncthreads();
    if (warp == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh->tmem_base)),
                     "r"(2 * E::WCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid < KMAX) E::setup_user(sh, g, gp, users + (int64_t)b * K * 2, K, tid);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh->tmem_base;

    const int64_t nbeg = (int64_t)s * chunk;
    const int64_t nend = min(g.N, nbeg + chunk);
    const int nst = E::stages(nbeg, nend);
    if (warp < 8) {
        E::generate(sh, smem_u32(base), tmem, g, gp, nbeg, nend, ura, 0, 0, 0, !sh->near);
    } else {
        if (lane == 0) E::mma(sh, smem_u32(base), tmem, nst, 0, 0);
        __syncwarp();
    }
    bool ok = mbar_wait(&sh->done, 0, &sh->abort);
    tc_fence_before();
    __syncthreads();  // every MMA done and every drain's tcgen05.st complete
    tc_fence_after();
    ok = ok && !*(volatile int*)&sh->abort && !sh->bad;
    E::epilogue(sh, fold, tmem, K, E::drains(nst), ok, out + ((int64_t)b * S + s) * K * K, tid, warp, lane);
    __syncthreads();
    if (warp == 8) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * E::WCOLS) : "memory");
    }
}

template <int KMAX>
static size_t tc_smem_bytes() {
    constexpr int NRING = GtCfg<KMAX>::NRING;
    return 1024 + NRING * GramEngine<XLMIMO_FSPL_USW, KMAX, TCP_BF16X3, false, NRING>::BYTES +
           sizeof(EngShared<KMAX, NRING>);
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
// `span`), reducing chunk partials when S > 1.  The engine counts a chunk's
// 64-element stages in 32 bits, so a chunk holds at most ~2^36 elements: an
// array longer than that is split whatever the batch size.
static int launch_tc_chunks(TcKernel kern, size_t smem, const Geom& g, const GenParams& gp, int span,
                            const double* users, int K, int B, double* gram, const UraRows& ura, cudaStream_t st) {
    constexpr int64_t MAX_CHUNK = int64_t(1) << 36;
    int S = choose_split(g.N, B, span, 4);
    const int64_t min_s = (g.N + MAX_CHUNK - 1) / MAX_CHUNK;
    if (S < min_s) S = (int)min_s;
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
    const size_t smem = wide ? tc_smem_bytes<64>() : tc_smem_bytes<32>();
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
