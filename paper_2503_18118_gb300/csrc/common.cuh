// Internal helpers shared by the CUDA translation units of libxlmimo.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "xlmimo.h"

namespace xl {

// Thread-local message behind xlmimo_last_error().
void set_error(const char* fmt, ...);
void clear_error();

int num_sms();

// Translate a CUDA error into XLMIMO_ECUDA with a message.
int cuda_status(cudaError_t e, const char* where);

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Geometry shared by the channel generators.
struct Geom {
    int64_t N;
    double lambda, inv_lambda, spacing, beta0;
    int model;
};

int check_array(const xlmimo_array* arr, Geom* g);

// Host launchers implemented in the .cu files (validated arguments only).
int launch_gram_f64(const Geom& g, const double* users, int K, int B, double* gram, cudaStream_t st);
int launch_gram_f32(const Geom& g, const double* users, int K, int B, double* gram, cudaStream_t st);
int launch_gram_tc(const Geom& g, const double* users, int K, int B, int prec, double* gram, cudaStream_t st,
                   int ctas_per_sm = 0);
// URA of `rows` rows of g.N elements (rows >= 1): the tensor-core Gram's URA
// mode where it applies, else per-row-pair ULA Grams.
int launch_gram_ura(const Geom& g, int64_t rows, const double* users, int K, int B, int prec, double* gram,
                    cudaStream_t st);
// URA mode of the tensor-core Gram (BF16 hi/lo, spherical-wave models, rows of
// ncol elements, ncol a multiple of 128, on an sm_103 device): all row pairs
// of a trial accumulated in one pass.
bool gram_tc_ura_supported(const Geom& g, int64_t ncol, int prec);
int launch_gram_tc_ura(const Geom& g, int64_t ncol, int64_t rows, const double* users, int K, int B, double* gram,
                       cudaStream_t st);
// threads per block: 256 alone; 64 lets a block (at most 48 registers a thread) fit
// beside three tensor-core Gram CTAs on an SM, so that it runs during the Gram.
int launch_closed_form(const Geom& g, const double* users, int K, int B, double* gram, cudaStream_t st,
                       int threads = 256);
// Finite-aperture factor (APERTURE_* of aperture.cuh) applied in place to the
// off-diagonal entries of closed-form Grams.
int launch_aperture_apply(const Geom& g, int mode, const double* users, int K, int B, double* gram, cudaStream_t st);
// The same factor written only below the diagonal, conj(G~_ij F_ij), leaving
// G~_ij above it (the surrogate's base).
int launch_aperture_base(const Geom& g, int mode, const double* users, int K, int B, double* gram, cudaStream_t st);
// Row r and column c of the q-th entry of a lower triangle stored row by
// row (c <= r), without FP64 arithmetic.
__device__ __forceinline__ void tri_index(int q, int* r, int* c) {
    int rr = (int)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);
    while ((rr + 1) * (rr + 2) / 2 <= q) ++rr;
    while (rr * (rr + 1) / 2 > q) --rr;
    *r = rr;
    *c = q - rr * (rr + 1) / 2;
}

// rate (nullable): per-trial sum rate, computed by the receiver kernel itself.
int launch_beamform(const double* gf, const double* gt, const double* power, const double* noise, int K,
                    int B, int scheme, int power_mode, double* sinr, int* status, double* cap,
                    cudaStream_t st, double* rate = nullptr);
int launch_sumrate(const double* sinr, int K, int B, double* rate, double* stats, cudaStream_t st);
int launch_saturation(const double* users, int K, int B, double t, double spacing, double* sat,
                      cudaStream_t st);
int saturation_analytic(const xlmimo_user_dist* d, int K, double t, double spacing, double* out,
                        cudaStream_t st);

// One instance of a ragged batch, device copy (see xlmimo_inst).
struct DevInst {
    long long n_ant;
    int k, scheme;
    long long user_off, gram_off;
    double noise;
    long long part_off;  // first complex entry of its chunk partials (-1: single work item)
    int nchunks, pad;
};

// Receivers of the instances list[0..n) of a ragged batch (matched, on their
// exact Gram), shared memory sized for kmax users.
void beamform_trial_launch_bucket(const DevInst* insts, const int* list, int n, int kmax, const double* gram,
                                  const double* power, int power_mode, double* sinr, int* status, cudaStream_t st);
int beamform_ragged_prepare();  // one-time kernel attribute, outside any stream capture

// Split of the element range when the batch alone cannot fill the GPU.
// Returns the number of contiguous element chunks per trial (>= 1); each chunk
// is a whole number of `tile` elements except the last.
int choose_split(int64_t N, int B, int tile, int ctas_per_sm_hint);

// Deterministic sum of S partial Gram matrices [B][S][K][K] (complex double)
// into gram [B][K][K], in increasing chunk order.
int launch_reduce_partials(const double* partial, int S, int K, int B, double* gram, cudaStream_t st);

}  // namespace xl

// ---- device helpers -------------------------------------------------------

#define XL_DEV __device__ __forceinline__

namespace xl {

XL_DEV double element_y(int64_t n, int64_t N, double spacing) {
    return ((double)n - 0.5 * (double)(N - 1)) * spacing;
}

XL_DEV bool user_ok(double x, double y) { return x > 0.0 && isfinite(x) && isfinite(y); }

}  // namespace xl
