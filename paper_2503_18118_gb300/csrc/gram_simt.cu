// Exact Gram matrices H^H H on the SIMT pipes (Sec. III inner products,
// Sec. V-B "the most time-consuming process").
//
//   gram_f64_kernel  FP64 generation (per-element FP64 distance and phase) and
//                    FP64 accumulation: the plain FP64 GPU baseline.
//   gram_f32_kernel  FP32 generation with an FP64 phase reference every
//                    REF_SPAN elements (chan_gen.cuh), FP32 accumulation in
//                    4x4 complex register blocks over the upper triangle.
//
// One CTA per (trial, element chunk).  Each CTA walks its chunk in tiles:
// all threads generate the tile's K x T channel entries into shared memory,
// then accumulate conj(h_i) h_j for the pairs they own.  Chunks > 1 only when
// the batch is too small to fill the GPU; their partial Gram matrices are
// summed in a fixed order by reduce_partials_kernel.
#include <math.h>

#include "chan_gen.cuh"
#include "common.cuh"

namespace xl {

// ---------------------------------------------------------------- FP64 ----
constexpr int F64_T = 32;
constexpr int F64_THREADS = 256;
constexpr int F64_MAXQ = (XLMIMO_MAX_USERS * (XLMIMO_MAX_USERS + 1) / 2 + F64_THREADS - 1) / F64_THREADS;

__device__ __forceinline__ double2 gen_entry_f64(const Geom& g, int64_t n, double x, double y, double r0u,
                                                 double su) {
    double yn = element_y(n, g.N, g.spacing);
    double q, amp;
    if (g.model == XLMIMO_UPW) {
        q = (r0u - yn * su) * g.inv_lambda;
        amp = sqrt(g.beta0) / r0u;
    } else {
        double dy = yn - y;
        double r = sqrt(fma(dy, dy, x * x));
        q = r * g.inv_lambda;
        amp = (g.model == XLMIMO_PNUSW) ? sqrt(g.beta0) * sqrt(x / r) / r
                                        : g.lambda / (4.0 * 3.14159265358979323846 * r);
    }
    double f = q - rint(q);
    double s, c;
    sincospi(2.0 * f, &s, &c);
    return make_double2(amp * c, -amp * s);
}

__global__ void __launch_bounds__(F64_THREADS) gram_f64_kernel(Geom g, const double* __restrict__ users, int K,
                                                              int S, int64_t chunk, double2* __restrict__ out) {
    __shared__ double ux[XLMIMO_MAX_USERS], uy[XLMIMO_MAX_USERS], ur0[XLMIMO_MAX_USERS], us[XLMIMO_MAX_USERS];
    __shared__ double2 H[F64_T * XLMIMO_MAX_USERS];
    __shared__ unsigned char pi_[XLMIMO_MAX_USERS * (XLMIMO_MAX_USERS + 1) / 2];
    __shared__ unsigned char pj_[XLMIMO_MAX_USERS * (XLMIMO_MAX_USERS + 1) / 2];
    __shared__ int bad;
    const int tid = threadIdx.x;
    const int b = blockIdx.x, s = blockIdx.y;
    if (tid == 0) bad = 0;
    __syncthreads();
    if (tid < K) {
        double x = users[((int64_t)b * K + tid) * 2], y = users[((int64_t)b * K + tid) * 2 + 1];
        ux[tid] = x;
        uy[tid] = y;
        ur0[tid] = sqrt(x * x + y * y);
        us[tid] = y / ur0[tid];
        if (!user_ok(x, y)) atomicOr(&bad, 1);
    }
    const int P = K * (K + 1) / 2;
    if (tid == 0) {
        int p = 0;
        for (int i = 0; i < K; ++i)
            for (int j = i; j < K; ++j) { pi_[p] = (unsigned char)i; pj_[p] = (unsigned char)j; ++p; }
    }
    __syncthreads();
    double2* o = out + ((int64_t)b * S + s) * K * K;
    if (bad) {
        for (int e = tid; e < K * K; e += F64_THREADS) o[e] = make_double2(nan(""), nan(""));
        return;
    }
    double2 acc[F64_MAXQ];
#pragma unroll
    for (int q = 0; q < F64_MAXQ; ++q) acc[q] = make_double2(0.0, 0.0);
    const int64_t nb = (int64_t)s * chunk;
    const int64_t ne = min(g.N, nb + chunk);
    for (int64_t n0 = nb; n0 < ne; n0 += F64_T) {
        __syncthreads();
        for (int e = tid; e < F64_T * K; e += F64_THREADS) {
            int t = e / K, k = e - t * K;
            int64_t n = n0 + t;
            H[e] = (n < ne) ? gen_entry_f64(g, n, ux[k], uy[k], ur0[k], us[k]) : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < F64_MAXQ; ++q) {
            int p = tid + q * F64_THREADS;
            if (p < P) {
                int i = pi_[p], j = pj_[p];
                double re = acc[q].x, im = acc[q].y;
                for (int t = 0; t < F64_T; ++t) {
                    double2 a = H[t * K + i], c = H[t * K + j];
                    re = fma(a.x, c.x, fma(a.y, c.y, re));
                    im = fma(a.x, c.y, fma(-a.y, c.x, im));
                }
                acc[q] = make_double2(re, im);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < F64_MAXQ; ++q) {
        int p = tid + q * F64_THREADS;
        if (p < P) {
            int i = pi_[p], j = pj_[p];
            if (i == j) {
                o[i * K + i] = make_double2(acc[q].x, 0.0);
            } else {
                o[i * K + j] = acc[q];
                o[j * K + i] = make_double2(acc[q].x, -acc[q].y);
            }
        }
    }
}

// ---------------------------------------------------------------- FP32 ----
// Tile layout in shared memory: row t (one element) holds the K users'
// entries in 4-user blocks of 6 complex slots (4 used), so the 16-byte loads
// of up to eight different blocks of one row hit distinct banks.
//
// Pair mapping.  The upper triangle of 4x4 complex blocks (nblk blocks) is
// accumulated by (block, sub-stream) threads; sub-stream s owns elements
// [s*tps, (s+1)*tps) of every tile.
//   mode 1 (nb == 8, K = 29..32, 36 blocks, 8 sub-streams, 9 warps): warp w < 8
//     is sub-stream w with lane = block 0..31, so each of its loads reads one
//     row; warp 8 takes blocks 32..35 of all eight sub-streams.
//   mode 0 (other K): thread -> (tid % nblk, tid / nblk).
constexpr int F32_T = 64;          // elements per tile
constexpr int F32_MAXTHREADS = 288;
constexpr int F32_BLK = 6;         // complex slots per 4-user block in a tile row

struct F32Plan {
    int nb;      // 4-user blocks per side
    int nblk;    // upper-triangle blocks
    int ssub;    // element sub-streams per tile
    int tps;     // elements per sub-stream per tile
    int mode;
    int threads;
    int ks;      // row stride of the shared tile, in complex entries
    int kp;      // users rounded up to a power of two (generation lanes per element)
    int gen_threads;
    size_t smem;
};

static F32Plan plan_f32(int K) {
    F32Plan p;
    p.nb = (K + 3) / 4;
    p.nblk = p.nb * (p.nb + 1) / 2;
    if (p.nb == 8) {
        p.mode = 1;
        p.ssub = 8;
        p.threads = 288;
    } else {
        p.mode = 0;
        p.ssub = 16;
        while (p.ssub > 1 && p.nblk * p.ssub > F32_MAXTHREADS) p.ssub >>= 1;
        p.threads = ((p.nblk * p.ssub + 31) / 32) * 32;
    }
    p.tps = F32_T / p.ssub;
    p.ks = F32_BLK * p.nb;
    p.kp = 1;
    while (p.kp < K) p.kp <<= 1;
    int warps = p.threads / 32, gw = 1;
    while (gw * 2 <= warps && gw * 2 <= 8) gw *= 2;
    p.gen_threads = 32 * gw;
    if (p.gen_threads < p.kp) p.gen_threads = p.kp;  // K > 32 needs two warps (always available)
    size_t tile = (size_t)F32_T * p.ks * sizeof(float2);
    size_t red = (size_t)p.nblk * p.ssub * 16 * sizeof(float2);
    size_t big = tile > red ? tile : red;
    p.smem = big + XLMIMO_MAX_USERS * sizeof(UserGeo) + p.nblk * 2;
    return p;
}

__global__ void __launch_bounds__(F32_MAXTHREADS, 3) gram_f32_kernel(Geom g, GenParams gp,
                                                                 const double* __restrict__ users, int K, F32Plan pl,
                                                                 int S, int64_t chunk, double2* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int nb = pl.nb, nblk = pl.nblk, ssub = pl.ssub, tps = pl.tps, ks = pl.ks;
    size_t tile_bytes = (size_t)F32_T * ks * sizeof(float2);
    size_t red_bytes = (size_t)nblk * ssub * 16 * sizeof(float2);
    size_t big = tile_bytes > red_bytes ? tile_bytes : red_bytes;
    float2* H = reinterpret_cast<float2*>(smem);
    float2* red = reinterpret_cast<float2*>(smem);
    UserGeo* ug = reinterpret_cast<UserGeo*>(smem + big);
    unsigned char* bi = reinterpret_cast<unsigned char*>(ug + XLMIMO_MAX_USERS);
    unsigned char* bj = bi + nblk;
    __shared__ int bad;

    const int tid = threadIdx.x;
    const int b = blockIdx.x, s = blockIdx.y;
    if (tid == 0) {
        bad = 0;
        int q = 0;
        for (int jb = 0; jb < nb; ++jb)
            for (int ib = 0; ib <= jb; ++ib) { bi[q] = (unsigned char)ib; bj[q] = (unsigned char)jb; ++q; }
    }
    __syncthreads();
    if (tid < K) {
        double x = users[((int64_t)b * K + tid) * 2], y = users[((int64_t)b * K + tid) * 2 + 1];
        UserGeo u = make_user_geo(g, x, y);
        if (!u.ok) atomicOr(&bad, 1);
        ug[tid] = u;
    }
    __syncthreads();
    double2* o = out + ((int64_t)b * S + s) * K * K;
    if (bad) {
        for (int e = tid; e < K * K; e += blockDim.x) o[e] = make_double2(nan(""), nan(""));
        return;
    }
    // pair mapping
    int blk, sub;
    bool active;
    if (pl.mode == 1) {
        const int w = tid >> 5, l = tid & 31;
        if (w < 8) { blk = l; sub = w; } else { blk = 32 + (l & 3); sub = l >> 2; }
        active = true;
    } else {
        active = tid < nblk * ssub;
        blk = active ? tid % nblk : 0;
        sub = active ? tid / nblk : 0;
    }
    const int ib = bi[blk], jb = bj[blk];
    // generation mapping: thread -> fixed user, strided elements
    const bool gen = tid < pl.gen_threads;
    const int kmask = pl.kp - 1;
    int lk = 0;
    while ((1 << lk) < pl.kp) ++lk;
    const int gk = tid & kmask;                  // user of this generating thread
    const int gt0 = tid >> lk;                   // first element of this thread in a tile
    const int gts = pl.gen_threads >> lk;        // element stride
    const bool gen_user = gen && gk < K;
    float xl2 = 0.f, x2x2 = 0.f, ampc = 0.f;
    if (gen_user) { xl2 = ug[gk].xl2; x2x2 = ug[gk].x2x2; ampc = ug[gk].ampc; }
    const int slot = (gk >> 2) * F32_BLK + (gk & 3);
    UserRef ref = {0.f, 0.f, 0.f, 0.f, 1.f};

    float ar[16], ai[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) { ar[e] = 0.f; ai[e] = 0.f; }

    const int64_t nbeg = (int64_t)s * chunk;
    const int64_t nend = min(g.N, nbeg + chunk);
    int64_t nc = 0;
    for (int64_t n0 = nbeg; n0 < nend; n0 += F32_T) {
        if (((n0 - nbeg) % REF_SPAN) == 0) {
            nc = n0 + REF_SPAN / 2;
            if (gen_user) ref = make_user_ref(gp, ug[gk], (long long)nc);
        }
        __syncthreads();  // previous tile consumed
        if (gen && gk < pl.kp) {
            for (int t = gt0; t < F32_T; t += gts) {
                int64_t n = n0 + t;
                float2 h = make_float2(0.f, 0.f);
                if (gen_user && n < nend) h = gen_entry_f32(gp.model, gp.dprime_f, xl2, x2x2, ampc, ref, (float)(int)(n - nc));
                if (gk < 4 * nb) H[t * ks + slot] = h;
            }
        }
        __syncthreads();
        if (active) {
            const float2* rowp = H + (sub * tps) * ks;
            for (int tt = 0; tt < tps; ++tt, rowp += ks) {
                float4 a01 = *reinterpret_cast<const float4*>(rowp + F32_BLK * ib);
                float4 a23 = *reinterpret_cast<const float4*>(rowp + F32_BLK * ib + 2);
                float4 c01 = *reinterpret_cast<const float4*>(rowp + F32_BLK * jb);
                float4 c23 = *reinterpret_cast<const float4*>(rowp + F32_BLK * jb + 2);
                float are[4] = {a01.x, a01.z, a23.x, a23.z}, aim[4] = {a01.y, a01.w, a23.y, a23.w};
                float cre[4] = {c01.x, c01.z, c23.x, c23.z}, cim[4] = {c01.y, c01.w, c23.y, c23.w};
#pragma unroll
                for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                        // conj(a) * c
                        ar[ii * 4 + jj] = fmaf(are[ii], cre[jj], fmaf(aim[ii], cim[jj], ar[ii * 4 + jj]));
                        ai[ii * 4 + jj] = fmaf(are[ii], cim[jj], fmaf(-aim[ii], cre[jj], ai[ii * 4 + jj]));
                    }
            }
        }
    }
    __syncthreads();
    // deterministic reduction over the element sub-streams
    if (active) {
#pragma unroll
        for (int e = 0; e < 16; ++e) red[((int64_t)blk * 16 + e) * ssub + sub] = make_float2(ar[e], ai[e]);
    }
    __syncthreads();
    for (int w = tid; w < nblk * 16; w += blockDim.x) {
        int q = w / 16, e = w - q * 16;
        float re = 0.f, im = 0.f;
        for (int u = 0; u < ssub; ++u) {
            float2 v = red[(int64_t)w * ssub + u];
            re += v.x;
            im += v.y;
        }
        int i = 4 * bi[q] + e / 4, j = 4 * bj[q] + (e & 3);
        if (i < K && j < K && i <= j) {
            if (i == j) {
                o[i * K + i] = make_double2((double)re, 0.0);
            } else {
                o[i * K + j] = make_double2((double)re, (double)im);
                o[j * K + i] = make_double2((double)re, -(double)im);
            }
        }
    }
}

// ---------------------------------------------------------------- host ----
static int run_split(int S, int K, int B, double* gram, double** part, cudaStream_t st) {
    *part = nullptr;
    if (S == 1) return XLMIMO_OK;
    size_t bytes = (size_t)B * S * K * K * sizeof(double2);
    return cuda_status(cudaMallocAsync((void**)part, bytes, st), "workspace allocation");
}

int launch_gram_f64(const Geom& g, const double* users, int K, int B, double* gram, cudaStream_t st) {
    int S = choose_split(g.N, B, F64_T, 4);
    int64_t tiles = (g.N + F64_T - 1) / F64_T;
    int64_t chunk = ((tiles + S - 1) / S) * F64_T;
    S = (int)((g.N + chunk - 1) / chunk);
    double* part = nullptr;
    int rc = run_split(S, K, B, gram, &part, st);
    if (rc) return rc;
    dim3 grid(B, S);
    gram_f64_kernel<<<grid, F64_THREADS, 0, st>>>(g, users, K, S, chunk, (double2*)(S == 1 ? gram : part));
    rc = cuda_status(cudaGetLastError(), "gram_f64 launch");
    if (!rc && S > 1) rc = launch_reduce_partials(part, S, K, B, gram, st);
    if (part) cudaFreeAsync(part, st);
    return rc;
}

int launch_gram_f32(const Geom& g, const double* users, int K, int B, double* gram, cudaStream_t st) {
    F32Plan p = plan_f32(K);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(gram_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        attr_set = true;
    }
    int S = choose_split(g.N, B, REF_SPAN, 4);
    int64_t spans = (g.N + REF_SPAN - 1) / REF_SPAN;
    int64_t chunk = ((spans + S - 1) / S) * REF_SPAN;
    S = (int)((g.N + chunk - 1) / chunk);
    double* part = nullptr;
    int rc = run_split(S, K, B, gram, &part, st);
    if (rc) return rc;
    dim3 grid(B, S);
    gram_f32_kernel<<<grid, p.threads, p.smem, st>>>(g, make_gen_params(g), users, K, p, S, chunk,
                                                     (double2*)(S == 1 ? gram : part));
    rc = cuda_status(cudaGetLastError(), "gram_f32 launch");
    if (!rc && S > 1) rc = launch_reduce_partials(part, S, K, B, gram, st);
    if (part) cudaFreeAsync(part, st);
    return rc;
}

}  // namespace xl

namespace xl {

// Same element split and kernels as launch_gram_f64 / launch_gram_f32, with
// the partial Gram matrices written to caller-provided device scratch instead
// of stream-ordered allocations.  Rejects the call (nothing enqueued) when the
// split needs more than scratch_bytes.
int launch_gram_into_scratch(const Geom& g, const double* users, int K, int B, int prec, double* gram,
                             double* scratch, size_t scratch_bytes, cudaStream_t st) {
    int tile = prec == XLMIMO_F64 ? F64_T : REF_SPAN;
    int S = choose_split(g.N, B, tile, 4);
    int64_t tiles = (g.N + tile - 1) / tile;
    int64_t chunk = ((tiles + S - 1) / S) * tile;
    S = (int)((g.N + chunk - 1) / chunk);
    size_t need = S > 1 ? (size_t)B * S * K * K * sizeof(double2) : 0;
    if (need > scratch_bytes) {
        set_error("this batch splits each trial into %d element chunks and needs %zu bytes of scratch; the static "
                  "scratch holds %zu bytes (use fewer trials per call, or xlmimo_channel_gram)",
                  S, need, scratch_bytes);
        return XLMIMO_EINVAL;
    }
    double2* out = (double2*)(S == 1 ? gram : scratch);
    dim3 grid(B, S);
    if (prec == XLMIMO_F64) {
        gram_f64_kernel<<<grid, F64_THREADS, 0, st>>>(g, users, K, S, chunk, out);
    } else {
        F32Plan p = plan_f32(K);
        cudaError_t e = cudaFuncSetAttribute(gram_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        if (e != cudaSuccess) return cuda_status(e, "gram_f32 attribute");
        gram_f32_kernel<<<grid, p.threads, p.smem, st>>>(g, make_gen_params(g), users, K, p, S, chunk, out);
    }
    int rc = cuda_status(cudaGetLastError(), "gram launch");
    if (!rc && S > 1) rc = launch_reduce_partials(scratch, S, K, B, gram, st);
    return rc;
}

}  // namespace xl
