// xlmimo_channel_gram_noalloc: the exact Gram without any device allocation.
//
// Some callers cannot allocate device memory while they run: a host
// application that reserves the GPU's memory up front for its own pool and
// forbids allocations after start-up, or a latency-critical loop that cannot
// accept cudaMalloc/cudaFree (which may block or synchronise the device).
// For them the element-split partial sums live in the fixed array below,
// allocated once when the library's module is loaded on a device and kept
// until the process exits.
#include <mutex>
#include <vector>

#include "common.cuh"

namespace xl {

int launch_gram_into_scratch(const Geom& g, const double* users, int K, int B, int prec, double* gram,
                             double* scratch, size_t scratch_bytes, cudaStream_t st);

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(XLMIMO_NOALLOC_SCRATCH_MIB) << 20;

static __device__ __align__(256) double2 g_noalloc_scratch[NOALLOC_SCRATCH_BYTES / sizeof(double2)];

// Device address of the scratch array on the current device, looked up once
// per device (the host-side name of the array is only a stand-in and must
// never be passed to a kernel).
static int scratch_address(double** out) {
    static std::mutex mu;
    static std::vector<double*> addr;
    int dev = 0;
    int rc = cuda_status(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(mu);
    if ((int)addr.size() <= dev) addr.resize(dev + 1, nullptr);
    if (!addr[dev]) {
        void* p = nullptr;
        rc = cuda_status(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress(noalloc scratch)");
        if (rc) return rc;
        addr[dev] = static_cast<double*>(p);
    }
    *out = addr[dev];
    return XLMIMO_OK;
}

}  // namespace xl

using namespace xl;

extern "C" int xlmimo_channel_gram_noalloc(const xlmimo_array* arr, const double* users, int K, int B, int prec,
                                           double* gram, void* stream) {
    clear_error();
    Geom g;
    int rc = check_array(arr, &g);
    if (rc) return rc;
    if (K < 1 || K > XLMIMO_MAX_USERS) { set_error("K must be in [1, %d], got %d", XLMIMO_MAX_USERS, K); return XLMIMO_EINVAL; }
    if (B < 0) { set_error("B must be >= 0, got %d", B); return XLMIMO_EINVAL; }
    if (prec != XLMIMO_F64 && prec != XLMIMO_F32) {
        set_error("xlmimo_channel_gram_noalloc supports XLMIMO_F64 and XLMIMO_F32 only");
        return (prec >= XLMIMO_BF16 && prec <= XLMIMO_F16X3) ? XLMIMO_EUNSUPPORTED : XLMIMO_EINVAL;
    }
    if (B == 0) return XLMIMO_OK;
    if (!users || !gram) { set_error("users and gram must be non-NULL"); return XLMIMO_EINVAL; }
    double* scratch = nullptr;
    rc = scratch_address(&scratch);
    if (rc) return rc;
    return launch_gram_into_scratch(g, users, K, B, prec, gram, scratch, NOALLOC_SCRATCH_BYTES, as_stream(stream));
}
