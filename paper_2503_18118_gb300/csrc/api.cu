// C-ABI entry points of libxlmimo: argument validation, error plumbing and
// dispatch to the kernel launchers.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "common.cuh"

namespace xl {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = 0; }

int cuda_status(cudaError_t e, const char* where) {
    if (e == cudaSuccess) return XLMIMO_OK;
    set_error("%s: %s", where, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? XLMIMO_ENOMEM : XLMIMO_ECUDA;
}

int num_sms() {
    static std::mutex mu;
    static std::vector<int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    std::lock_guard<std::mutex> lk(mu);
    if ((int)cache.size() <= dev) cache.resize(dev + 1, 0);
    if (!cache[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
        cache[dev] = v;
    }
    return cache[dev];
}

int check_array(const xlmimo_array* arr, Geom* g) {
    if (!arr) { set_error("array descriptor is NULL"); return XLMIMO_EINVAL; }
    if (arr->n_ant < 1 || arr->n_ant > (int64_t(1) << 40)) {
        set_error("n_ant must be in [1, 2^40], got %lld", (long long)arr->n_ant);
        return XLMIMO_EINVAL;
    }
    if (!(arr->wavelength > 0.0) || !isfinite(arr->wavelength)) { set_error("wavelength must be > 0"); return XLMIMO_EINVAL; }
    if (!(arr->spacing > 0.0) || !isfinite(arr->spacing)) { set_error("spacing must be > 0"); return XLMIMO_EINVAL; }
    if (!(arr->beta0 > 0.0) || !isfinite(arr->beta0)) { set_error("beta0 must be > 0"); return XLMIMO_EINVAL; }
    if (arr->model < XLMIMO_PNUSW || arr->model > XLMIMO_UPW) { set_error("unknown channel model %d", arr->model); return XLMIMO_EINVAL; }
    if (arr->reserved != 0) { set_error("reserved field must be 0"); return XLMIMO_EINVAL; }
    g->N = arr->n_ant;
    g->lambda = arr->wavelength;
    g->inv_lambda = 1.0 / arr->wavelength;
    g->spacing = arr->spacing;
    g->beta0 = arr->beta0;
    g->model = arr->model;
    return XLMIMO_OK;
}

int choose_split(int64_t N, int B, int tile, int ctas_per_sm_hint) {
    int64_t tiles = (N + tile - 1) / tile;
    int64_t want = (int64_t)num_sms() * ctas_per_sm_hint;
    if (B >= want) return 1;
    int64_t s = (want + B - 1) / B;
    int64_t max_s = tiles / 2;  // keep at least two tiles per chunk
    if (s > max_s) s = max_s;
    if (s < 1) s = 1;
    if (s > 4096) s = 4096;
    return (int)s;
}

__global__ void reduce_partials_kernel(const double2* __restrict__ part, int S, int K, int B,
                                       double2* __restrict__ gram) {
    int64_t kk = (int64_t)K * K;
    int64_t total = (int64_t)B * kk;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t b = e / kk, ij = e - b * kk;
        const double2* p = part + b * S * kk + ij;
        double re = 0.0, im = 0.0;
        for (int s = 0; s < S; ++s) {
            double2 v = p[(int64_t)s * kk];
            re += v.x;
            im += v.y;
        }
        gram[e] = make_double2(re, im);
    }
}

int launch_reduce_partials(const double* partial, int S, int K, int B, double* gram, cudaStream_t st) {
    int64_t total = (int64_t)B * K * K;
    int threads = 256;
    int64_t blocks = (total + threads - 1) / threads;
    if (blocks > 8LL * num_sms()) blocks = 8LL * num_sms();
    if (blocks < 1) blocks = 1;
    reduce_partials_kernel<<<(unsigned)blocks, threads, 0, st>>>((const double2*)partial, S, K, B, (double2*)gram);
    return cuda_status(cudaGetLastError(), "reduce_partials launch");
}

}  // namespace xl

using namespace xl;

static int check_kb(int K, int B) {
    if (K < 1 || K > XLMIMO_MAX_USERS) { set_error("K must be in [1, %d], got %d", XLMIMO_MAX_USERS, K); return XLMIMO_EINVAL; }
    if (B < 0) { set_error("B must be >= 0, got %d", B); return XLMIMO_EINVAL; }
    return XLMIMO_OK;
}

extern "C" {

int xlmimo_version(void) { return (1 << 16) | 0; }

const char* xlmimo_last_error(void) { return g_err; }

int xlmimo_channel_gram(const xlmimo_array* arr, const double* users, int K, int B, int prec,
                        double* gram, void* stream) {
    clear_error();
    Geom g;
    int rc = check_array(arr, &g);
    if (rc) return rc;
    if ((rc = check_kb(K, B))) return rc;
    if (B == 0) return XLMIMO_OK;
    if (!users || !gram) { set_error("users and gram must be non-NULL"); return XLMIMO_EINVAL; }
    switch (prec) {
        case XLMIMO_F64: return launch_gram_f64(g, users, K, B, gram, as_stream(stream));
        case XLMIMO_F32: return launch_gram_f32(g, users, K, B, gram, as_stream(stream));
        case XLMIMO_BF16:
        case XLMIMO_BF16X3:
        case XLMIMO_F16X3: return launch_gram_tc(g, users, K, B, prec, gram, as_stream(stream));
        default: set_error("unknown precision %d", prec); return XLMIMO_EINVAL;
    }
}

int xlmimo_channel_gram_ura(const xlmimo_array* arr, int64_t rows, const double* users, int K, int B, int prec,
                            double* gram, void* stream) {
    clear_error();
    Geom g;
    int rc = check_array(arr, &g);
    if (rc) return rc;
    if ((rc = check_kb(K, B))) return rc;
    if (rows < 1 || rows > XLMIMO_MAX_URA_ROWS || rows > ((int64_t)1 << 40) / arr->n_ant) {
        set_error("rows must be in [1, %d] with n_ant * rows <= 2^40, got %lld", XLMIMO_MAX_URA_ROWS,
                  (long long)rows);
        return XLMIMO_EINVAL;
    }
    if (prec < XLMIMO_F64 || prec > XLMIMO_F16X3) { set_error("unknown precision %d", prec); return XLMIMO_EINVAL; }
    if (B == 0) return XLMIMO_OK;
    if (!users || !gram) { set_error("users and gram must be non-NULL"); return XLMIMO_EINVAL; }
    return launch_gram_ura(g, rows, users, K, B, prec, gram, as_stream(stream));
}

int xlmimo_corr_closed_form(const xlmimo_array* arr, const double* users, int K, int B, double* gram,
                            void* stream) {
    clear_error();
    Geom g;
    int rc = check_array(arr, &g);
    if (rc) return rc;
    if ((rc = check_kb(K, B))) return rc;
    if (B == 0) return XLMIMO_OK;
    if (!users || !gram) { set_error("users and gram must be non-NULL"); return XLMIMO_EINVAL; }
    return launch_closed_form(g, users, K, B, gram, as_stream(stream));
}

int xlmimo_corr_closed_form_aperture(const xlmimo_array* arr, const double* users, int K, int B, int mode,
                                     double* gram, void* stream) {
    clear_error();
    Geom g;
    int rc = check_array(arr, &g);
    if (rc) return rc;
    if ((rc = check_kb(K, B))) return rc;
    if (mode < XLMIMO_APERTURE_NONE || mode > XLMIMO_APERTURE_FRESNEL) {
        set_error("unknown aperture mode %d", mode);
        return XLMIMO_EINVAL;
    }
    if (B == 0) return XLMIMO_OK;
    if (!users || !gram) { set_error("users and gram must be non-NULL"); return XLMIMO_EINVAL; }
    rc = launch_closed_form(g, users, K, B, gram, as_stream(stream));
    if (!rc) rc = launch_aperture_apply(g, mode, users, K, B, gram, as_stream(stream));
    return rc;
}

int xlmimo_beamform(const double* gram_filter, const double* gram_true, const double* power,
                    const double* noise, int K, int B, int scheme, int power_mode, double* sinr,
                    int* trial_status, double* capacity, void* stream) {
    clear_error();
    int rc = check_kb(K, B);
    if (rc) return rc;
    const int base = scheme & ~(XLMIMO_MISMATCH_FP32 | XLMIMO_FACTOR_FF);
    if (base < XLMIMO_ZF || base > XLMIMO_ZF_DL) { set_error("unknown scheme %d", scheme); return XLMIMO_EINVAL; }
    if (power_mode != XLMIMO_POWER_ABS && power_mode != XLMIMO_POWER_RXSNR) {
        set_error("unknown power mode %d", power_mode);
        return XLMIMO_EINVAL;
    }
    if (B == 0) return XLMIMO_OK;
    if (!gram_filter || !power || !noise || !sinr || !trial_status) {
        set_error("gram_filter, power, noise, sinr and trial_status must be non-NULL");
        return XLMIMO_EINVAL;
    }
    return launch_beamform(gram_filter, gram_true, power, noise, K, B, scheme, power_mode, sinr, trial_status,
                           capacity, as_stream(stream));
}

int xlmimo_sumrate(const double* sinr, int K, int B, double* rate, double* stats, void* stream) {
    clear_error();
    int rc = check_kb(K, B);
    if (rc) return rc;
    if (B == 0) {
        if (stats) {
            double z[3] = {0.0, 0.0, 0.0};
            return cuda_status(cudaMemcpyAsync(stats, z, sizeof(z), cudaMemcpyHostToDevice, as_stream(stream)),
                               "sumrate stats");
        }
        return XLMIMO_OK;
    }
    if (!sinr || !rate) { set_error("sinr and rate must be non-NULL"); return XLMIMO_EINVAL; }
    return launch_sumrate(sinr, K, B, rate, stats, as_stream(stream));
}

int xlmimo_saturation(const double* users, int K, int B, double t, double spacing, double* sat, void* stream) {
    clear_error();
    int rc = check_kb(K, B);
    if (rc) return rc;
    if (!(t > 0.0 && t < 1.0)) { set_error("t must be in (0, 1)"); return XLMIMO_EINVAL; }
    if (!(spacing > 0.0) || !isfinite(spacing)) { set_error("spacing must be > 0"); return XLMIMO_EINVAL; }
    if (B == 0) return XLMIMO_OK;
    if (!users || !sat) { set_error("users and sat must be non-NULL"); return XLMIMO_EINVAL; }
    return launch_saturation(users, K, B, t, spacing, sat, as_stream(stream));
}

int xlmimo_saturation_analytic(const xlmimo_user_dist* d, int K, double t, double spacing, double* out,
                               void* stream) {
    clear_error();
    if (!d || !out) { set_error("dist and out must be non-NULL"); return XLMIMO_EINVAL; }
    if (K < 1 || K > 100000000) { set_error("K must be in [1, 1e8]"); return XLMIMO_EINVAL; }
    if (!(t > 0.0 && t < 1.0)) { set_error("t must be in (0, 1)"); return XLMIMO_EINVAL; }
    if (!(spacing > 0.0)) { set_error("spacing must be > 0"); return XLMIMO_EINVAL; }
    if (d->reserved != 0 || (d->kind != XLMIMO_DIST_RECT && d->kind != XLMIMO_DIST_POLAR)) {
        set_error("bad distribution descriptor");
        return XLMIMO_EINVAL;
    }
    if (!(d->a0 > 0.0 && d->a1 > d->a0 && d->b1 > d->b0) || !isfinite(d->a1) || !isfinite(d->b0) ||
        !isfinite(d->b1)) {
        set_error("distribution ranges must satisfy 0 < a0 < a1, b0 < b1");
        return XLMIMO_EINVAL;
    }
    if (d->kind == XLMIMO_DIST_POLAR && (d->b0 < -1.5707963267948966 || d->b1 > 1.5707963267948966)) {
        set_error("polar angles must lie in [-pi/2, pi/2]");
        return XLMIMO_EINVAL;
    }
    return saturation_analytic(d, K, t, spacing, out, as_stream(stream));
}

}  // extern "C"
