// Measured pipe throughput for the roofline of the channel generator: many
// independent dependency chains of one operation per thread, every SM full,
// timed with CUDA events on the caller's stream.  The paper has no
// counterpart; this measures the device the kernels run on.
#include <math.h>

#include "common.cuh"

namespace xl {

constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_THREADS = 256;
constexpr int PROBE_BLOCKS_PER_SM = 8;

template <int PIPE>
__global__ void __launch_bounds__(PROBE_THREADS) pipe_probe_kernel(float* __restrict__ sink, int iters) {
    float a[PROBE_CHAINS];
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) a[i] = 0.5f + 1e-3f * (float)(threadIdx.x & 63) + 0.1f * (float)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < PROBE_CHAINS; ++i) {
            if (PIPE == XLMIMO_PIPE_SINCOS) a[i] = (i & 1) ? __cosf(a[i]) : __sinf(a[i]);
            else if (PIPE == XLMIMO_PIPE_RSQRT) a[i] = rsqrtf(a[i]);
            else a[i] = fmaf(a[i], 0.999f, 1e-3f);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) s += a[i];
    if (s == 12345.678f) sink[blockIdx.x] = s;  // keeps the chains alive; never true in practice
}

// The sink is never written (the chains never reach the sentinel); a module
// array serves as a valid address, so the probe allocates nothing.
static __device__ float probe_sink[1];

}  // namespace xl

using namespace xl;

extern "C" int xlmimo_measure_pipe(int pipe, double* out, void* stream) {
    clear_error();
    if (!out) { set_error("out must be non-NULL"); return XLMIMO_EINVAL; }
    if (pipe < XLMIMO_PIPE_SINCOS || pipe > XLMIMO_PIPE_FFMA) { set_error("unknown pipe %d", pipe); return XLMIMO_EINVAL; }
    cudaStream_t st = as_stream(stream);
    const int blocks = num_sms() * PROBE_BLOCKS_PER_SM;
    const int iters = pipe == XLMIMO_PIPE_FFMA ? 1 << 17 : 1 << 14;
    auto launch = [&](float* sink) {
        if (pipe == XLMIMO_PIPE_SINCOS) pipe_probe_kernel<XLMIMO_PIPE_SINCOS><<<blocks, PROBE_THREADS, 0, st>>>(sink, iters);
        else if (pipe == XLMIMO_PIPE_RSQRT) pipe_probe_kernel<XLMIMO_PIPE_RSQRT><<<blocks, PROBE_THREADS, 0, st>>>(sink, iters);
        else pipe_probe_kernel<XLMIMO_PIPE_FFMA><<<blocks, PROBE_THREADS, 0, st>>>(sink, iters);
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = cuda_status(cudaEventCreate(&e0), "probe event");
    if (!rc) rc = cuda_status(cudaEventCreate(&e1), "probe event");
    float* sink = nullptr;
    if (!rc) rc = cuda_status(cudaGetSymbolAddress((void**)&sink, probe_sink), "probe sink");
    if (!rc) {
        launch(sink);  // warm-up
        rc = cuda_status(cudaGetLastError(), "probe launch");
    }
    float best = 1e30f;
    for (int r = 0; r < 3 && !rc; ++r) {
        cudaEventRecord(e0, st);
        launch(sink);
        cudaEventRecord(e1, st);
        rc = cuda_status(cudaEventSynchronize(e1), "probe sync");
        float ms = 0.f;
        if (!rc) rc = cuda_status(cudaEventElapsedTime(&ms, e0, e1), "probe time");
        if (!rc && ms < best) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc) return rc;
    const double ops = (double)blocks * PROBE_THREADS * (double)iters * PROBE_CHAINS;
    out[0] = ops / (best * 1e-3);
    out[1] = best;
    return XLMIMO_OK;
}
