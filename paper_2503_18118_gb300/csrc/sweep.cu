// Capacity-saturation sweep (Sec. IV-C and V-C): for each array size, the
// exact and the closed-form Gram matrices of the same trials, ZF / MMSE
// rates of the exact receiver and of the receiver built from the closed
// form (modified ZF, judged on the exact channel), and the capacity, at
// every SNR.  Host loop over sizes; every trial-level step is a kernel.
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace xl {

int launch_stats_strided(const double* x, int B, int stride, double* out, cudaStream_t st);

__global__ void fill_kernel(double* __restrict__ x, int64_t n, double v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = v;
}

// Per-trial max_ij |A_ij - G_ij| / sqrt(G_ii G_jj).
__global__ void normwise_err_kernel(const double2* __restrict__ A, const double2* __restrict__ G, int K, int B,
                                    double* __restrict__ err) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < B; b += (int64_t)gridDim.x * blockDim.x) {
        const double2* a = A + b * K * K;
        const double2* g = G + b * K * K;
        double m = 0.0;
        for (int i = 0; i < K; ++i)
            for (int j = 0; j < K; ++j) {
                double dx = a[i * K + j].x - g[i * K + j].x, dy = a[i * K + j].y - g[i * K + j].y;
                double v = sqrt(dx * dx + dy * dy) / sqrt(g[i * K + i].x * g[j * K + j].x);
                m = fmax(m, v);
            }
        err[b] = m;
    }
}

__global__ void max_kernel(const double* __restrict__ x, int n, double* __restrict__ out) {
    __shared__ double sh[256];
    double m = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += 256) m = fmax(m, x[i]);
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

static int sweep_impl(const xlmimo_sweep_cfg* c, xlmimo_sweep_result* r, cudaStream_t st) {
    const int K = c->K, B = c->B, NS = c->snr_count;
    const size_t KK = (size_t)K * K;
    double *g_ex = nullptr, *g_cf = nullptr, *pw = nullptr, *nz = nullptr, *sinr = nullptr, *rate = nullptr,
           *cap = nullptr, *tmp = nullptr, *acc = nullptr, *sat = nullptr;
    int* status = nullptr;
    const int nacc = 3 * (4 * NS) + 3 * NS + 1 + 3 * 3;  // stats triplets; only means are reported
    size_t bytes = (2 * KK * 2 + 2 * (size_t)K + 5) * B * sizeof(double);
    int rc = cuda_status(cudaMallocAsync((void**)&g_ex, bytes, st), "sweep workspace");
    if (rc) return rc;
    g_cf = g_ex + 2 * KK * B;
    pw = g_cf + 2 * KK * B;
    sinr = pw + (size_t)K * B;
    nz = sinr + (size_t)K * B;
    rate = nz + B;
    cap = rate + B;
    tmp = cap + B;
    rc = cuda_status(cudaMallocAsync((void**)&acc, nacc * sizeof(double) + B * 3 * sizeof(double), st), "sweep acc");
    if (rc) { cudaFreeAsync(g_ex, st); return rc; }
    sat = acc + nacc;
    rc = cuda_status(cudaMallocAsync((void**)&status, B * sizeof(int), st), "sweep status");
    if (rc) { cudaFreeAsync(g_ex, st); cudaFreeAsync(acc, st); return rc; }

    int threads = 256, blocks = 4 * num_sms();
    fill_kernel<<<blocks, threads, 0, st>>>(nz, B, 1.0);

    // per-trial saturation interval (independent of N)
    if (!rc) rc = launch_saturation(c->users, K, B, c->t, c->spacing, sat, st);
    for (int q = 0; q < 3 && !rc; ++q) rc = launch_stats_strided(sat + q, B, 3, acc + nacc - 9 + 3 * q, st);
    std::vector<double> host(nacc);
    if (!rc) {
        rc = cuda_status(cudaMemcpyAsync(host.data(), acc, nacc * sizeof(double), cudaMemcpyDeviceToHost, st), "copy");
        if (!rc) rc = cuda_status(cudaStreamSynchronize(st), "sweep sync");
        if (!rc)
            for (int q = 0; q < 3; ++q) r->sat_mean[q] = host[nacc - 9 + 3 * q];
    }

    for (int ni = 0; ni < c->n_count && !rc; ++ni) {
        Geom g;
        g.N = c->n_list[ni];
        g.lambda = c->wavelength;
        g.inv_lambda = 1.0 / c->wavelength;
        g.spacing = c->spacing;
        g.beta0 = c->beta0;
        g.model = c->model;
        switch (c->prec) {
            case XLMIMO_F64: rc = launch_gram_f64(g, c->users, K, B, g_ex, st); break;
            case XLMIMO_F32: rc = launch_gram_f32(g, c->users, K, B, g_ex, st); break;
            default: rc = launch_gram_tc(g, c->users, K, B, c->prec, g_ex, st); break;
        }
        if (!rc) rc = launch_closed_form(g, c->users, K, B, g_cf, st);
        if (!rc) {
            const int blocks = (int)std::min<int64_t>(((int64_t)B + 255) / 256, 16LL * num_sms());
            normwise_err_kernel<<<blocks, 256, 0, st>>>((const double2*)g_cf, (const double2*)g_ex, K, B, tmp);
            max_kernel<<<1, 256, 0, st>>>(tmp, B, acc + 3 * (4 * NS) + 3 * NS);
            rc = cuda_status(cudaGetLastError(), "sweep err");
        }
        // N-independent power from the large-N limit of ||h||^2 at (ref_x, 0)
        double glim;
        if (c->model == XLMIMO_PNUSW)
            glim = 2.0 * c->beta0 / (c->spacing * c->ref_x);
        else if (c->model == XLMIMO_FSPL_USW)
            glim = 3.14159265358979323846 * (c->wavelength / (4.0 * 3.14159265358979323846)) *
                   (c->wavelength / (4.0 * 3.14159265358979323846)) / (c->spacing * c->ref_x);
        else
            glim = c->beta0 * (double)c->n_list[c->n_count - 1] / (c->ref_x * c->ref_x);
        for (int si = 0; si < NS && !rc; ++si) {
            double p = pow(10.0, c->snr_db[si] / 10.0) / glim;
            fill_kernel<<<blocks, threads, 0, st>>>(pw, (int64_t)K * B, p);
            int slot = 0;
            for (int path = 0; path < 2 && !rc; ++path)
                for (int sch = 0; sch < 2 && !rc; ++sch) {
                    const double* gf = path == 0 ? g_ex : g_cf;
                    const double* gt = path == 0 ? nullptr : g_ex;
                    int scheme = sch == 0 ? XLMIMO_ZF : XLMIMO_MMSE;
                    double* capp = (path == 0 && sch == 1) ? cap : nullptr;
                    rc = launch_beamform(gf, gt, pw, nz, K, B, scheme, XLMIMO_POWER_ABS, sinr, status, capp, st);
                    slot = (path * 2 + sch) * NS + si;
                    if (!rc) rc = launch_sumrate(sinr, K, B, rate, acc + 3 * slot, st);
                }
            if (!rc) rc = launch_stats_strided(cap, B, 1, acc + 3 * (4 * NS) + 3 * si, st);
        }
        if (!rc) {
            rc = cuda_status(cudaMemcpyAsync(host.data(), acc, nacc * sizeof(double), cudaMemcpyDeviceToHost, st),
                             "copy");
            if (!rc) rc = cuda_status(cudaStreamSynchronize(st), "sweep sync");
        }
        if (!rc) {
            for (int path = 0; path < 2; ++path)
                for (int sch = 0; sch < 2; ++sch)
                    for (int si = 0; si < NS; ++si)
                        r->rate[((size_t)ni * 4 + path * 2 + sch) * NS + si] = host[3 * ((path * 2 + sch) * NS + si)];
            for (int si = 0; si < NS; ++si) r->capacity[(size_t)ni * NS + si] = host[3 * (4 * NS) + 3 * si];
            r->gram_err[ni] = host[3 * (4 * NS) + 3 * NS];
        }
    }
    cudaFreeAsync(g_ex, st);
    cudaFreeAsync(acc, st);
    cudaFreeAsync(status, st);
    int rc2 = cuda_status(cudaStreamSynchronize(st), "sweep free");
    return rc ? rc : rc2;
}

}  // namespace xl

using namespace xl;

extern "C" int xlmimo_capacity_sweep(const xlmimo_sweep_cfg* c, xlmimo_sweep_result* r, void* stream) {
    clear_error();
    if (!c || !r) { set_error("cfg and result must be non-NULL"); return XLMIMO_EINVAL; }
    if (c->K < 1 || c->K > XLMIMO_MAX_USERS || c->B < 1) { set_error("K must be in [1, 64] and B >= 1"); return XLMIMO_EINVAL; }
    if (c->n_count < 1 || c->snr_count < 1 || !c->n_list || !c->snr_db || !c->users) {
        set_error("n_list, snr_db and users must be given");
        return XLMIMO_EINVAL;
    }
    if (!r->rate || !r->capacity || !r->gram_err) { set_error("result arrays must be non-NULL"); return XLMIMO_EINVAL; }
    if (!(c->wavelength > 0.0) || !(c->spacing > 0.0) || !(c->beta0 > 0.0) || !(c->ref_x > 0.0) ||
        !(c->t > 0.0 && c->t < 1.0)) {
        set_error("wavelength, spacing, beta0, ref_x must be > 0 and t in (0, 1)");
        return XLMIMO_EINVAL;
    }
    if (c->model < XLMIMO_PNUSW || c->model > XLMIMO_UPW) { set_error("unknown model"); return XLMIMO_EINVAL; }
    if (c->prec < XLMIMO_F64 || c->prec > XLMIMO_F16X3) {
        set_error("unknown precision");
        return XLMIMO_EINVAL;
    }
    for (int i = 0; i < c->n_count; ++i)
        if (c->n_list[i] < 1) { set_error("n_list entries must be >= 1"); return XLMIMO_EINVAL; }
    return sweep_impl(c, r, as_stream(stream));
}
