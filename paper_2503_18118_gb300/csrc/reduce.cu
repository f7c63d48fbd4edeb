// Rate / capacity reductions and the capacity-saturation point.
//
//   sumrate_kernel      R_b = sum_k log2(1 + SINR_bk) (Sec. V-C rates).
//   stats_kernel        mean and sum of squared deviations over the batch,
//                       one CTA, fixed-order tree: deterministic.
//   saturation_kernel   per-trial interval of Eqs. (15)-(16).
//   quad_kernel         E[max_k z_k] = z_hi - int F(z)^K dz (Appendix B,
//                       integrated by parts), composite Gauss-Legendre.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace xl {

// One warp per trial (lane = user), summed by a fixed shuffle tree, so the
// FP64 logarithms of a trial run side by side rather than one after another.
__global__ void sumrate_kernel(const double* __restrict__ sinr, int K, int B, double* __restrict__ rate) {
    const int lane = threadIdx.x & 31;
    const int64_t wpb = blockDim.x >> 5;
    for (int64_t b = blockIdx.x * wpb + (threadIdx.x >> 5); b < B; b += (int64_t)gridDim.x * wpb) {
        double r = 0.0;
        for (int k = lane; k < K; k += 32) r += log2(1.0 + sinr[b * K + k]);
        for (int off = 16; off > 0; off >>= 1) r += __shfl_xor_sync(0xffffffffu, r, off);
        if (lane == 0) rate[b] = r;
    }
}

constexpr int STATS_THREADS = 1024;

__device__ double block_sum(double v, double* sh) {
    const int tid = threadIdx.x;
    sh[tid] = v;
    __syncthreads();
    for (int s = STATS_THREADS / 2; s > 0; s >>= 1) {
        if (tid < s) sh[tid] += sh[tid + s];
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(STATS_THREADS) stats_kernel(const double* __restrict__ x, int B,
                                                              double* __restrict__ stats) {
    __shared__ double sh[STATS_THREADS];
    double s = 0.0;
    for (int64_t b = threadIdx.x; b < B; b += STATS_THREADS) s += x[b];
    double mean = block_sum(s, sh) / (double)B;
    double q = 0.0;
    for (int64_t b = threadIdx.x; b < B; b += STATS_THREADS) {
        double d = x[b] - mean;
        q += d * d;
    }
    double m2 = block_sum(q, sh);
    if (threadIdx.x == 0) {
        stats[0] = mean;
        stats[1] = m2;
        stats[2] = (double)B;
    }
}

__global__ void __launch_bounds__(STATS_THREADS) stats_strided_kernel(const double* __restrict__ x, int B,
                                                                      int stride, double* __restrict__ stats) {
    __shared__ double sh[STATS_THREADS];
    double s = 0.0;
    for (int64_t b = threadIdx.x; b < B; b += STATS_THREADS) s += x[b * stride];
    double mean = block_sum(s, sh) / (double)B;
    double q = 0.0;
    for (int64_t b = threadIdx.x; b < B; b += STATS_THREADS) {
        double d = x[b * stride] - mean;
        q += d * d;
    }
    double m2 = block_sum(q, sh);
    if (threadIdx.x == 0) {
        stats[0] = mean;
        stats[1] = m2;
        stats[2] = (double)B;
    }
}

int launch_stats_strided(const double* x, int B, int stride, double* out, cudaStream_t st) {
    stats_strided_kernel<<<1, STATS_THREADS, 0, st>>>(x, B, stride, out);
    return cuda_status(cudaGetLastError(), "stats launch");
}

int launch_sumrate(const double* sinr, int K, int B, double* rate, double* stats, cudaStream_t st) {
    const int threads = 256, wpb = threads / 32;
    const int blocks = (int)std::min<int64_t>(((int64_t)B + wpb - 1) / wpb, 16LL * num_sms());
    sumrate_kernel<<<blocks, threads, 0, st>>>(sinr, K, B, rate);
    int rc = cuda_status(cudaGetLastError(), "sumrate launch");
    if (rc || !stats) return rc;
    stats_kernel<<<1, STATS_THREADS, 0, st>>>(rate, B, stats);
    return cuda_status(cudaGetLastError(), "stats launch");
}

__global__ void saturation_kernel(const double* __restrict__ users, int K, int B, double a, double spacing,
                                  double* __restrict__ sat) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < B; b += (int64_t)gridDim.x * blockDim.x) {
        double up = -INFINITY, dn = INFINITY;
        for (int k = 0; k < K; ++k) {
            double x = users[((int64_t)b * K + k) * 2], y = users[((int64_t)b * K + k) * 2 + 1];
            up = fmax(up, fma(a, x, y));
            dn = fmin(dn, fma(-a, x, y));
        }
        sat[(int64_t)b * 3] = up;
        sat[(int64_t)b * 3 + 1] = dn;
        sat[(int64_t)b * 3 + 2] = ceil((up - dn) / spacing);
    }
}

int launch_saturation(const double* users, int K, int B, double t, double spacing, double* sat, cudaStream_t st) {
    double a = t / sqrt(1.0 - t * t);
    int threads = 256;
    const int blocks = (int)std::min<int64_t>(((int64_t)B + threads - 1) / threads, 16LL * num_sms());
    saturation_kernel<<<blocks, threads, 0, st>>>(users, K, B, a, spacing, sat);
    return cuda_status(cudaGetLastError(), "saturation launch");
}

// ---------------------------------------------------------------------------
// Ergodic saturation point.  z = a x + y for one user, a = t / sqrt(1 - t^2).
//
// RECT (x ~ U[x0, x1], y ~ U[y0, y1]): z is the sum of two independent
// uniforms of widths wa = a (x1 - x0) and wb = y1 - y0, so its CDF is the
// integral of a trapezoidal density; with lo = a x0 + y0, s = min(wa, wb),
// l = max(wa, wb), u = z - lo:
//   F = u^2 / (2 wa wb)                     for 0 <= u < s
//     = (2u - s) / (2 l)                     for s <= u < l
//     = 1 - (wa + wb - u)^2 / (2 wa wb)      for l <= u < wa + wb.
// POLAR (r ~ U[r0, r1], theta ~ U[th0, th1]): z = r c(theta) with
// c(theta) = a cos theta + sin theta = rho sin(theta + phi) > 0 on the range,
// rho = sqrt(1 + a^2), phi = atan(a).  Conditioning on theta,
// P(z <= v | theta) = clamp((v / c(theta) - r0) / (r1 - r0), 0, 1), and
// int d theta / c(theta) = log(tan((theta + phi) / 2)) / rho, so F(v) is a sum
// of closed-form pieces between the angles where v / c(theta) crosses r0 or r1.
// ---------------------------------------------------------------------------
struct DistDev {
    int kind;
    double a;            // slope t / sqrt(1 - t^2)
    double p0, p1, q0, q1;  // RECT: x0, x1, y0, y1 (y possibly reflected); POLAR: r0, r1, th0, th1
    double rho, phi;
};

__device__ double cdf_rect(const DistDev& d, double z) {
    double wa = d.a * (d.p1 - d.p0), wb = d.q1 - d.q0;
    double s = fmin(wa, wb), l = fmax(wa, wb);
    double u = z - (d.a * d.p0 + d.q0);
    if (u <= 0.0) return 0.0;
    if (u >= wa + wb) return 1.0;
    if (u < s) return u * u / (2.0 * wa * wb);
    if (u < l) return (2.0 * u - s) / (2.0 * l);
    double w = wa + wb - u;
    return 1.0 - w * w / (2.0 * wa * wb);
}

__device__ double polar_prim(const DistDev& d, double th) {  // int d theta / c(theta)
    return log(tan(0.5 * (th + d.phi))) / d.rho;
}

__device__ double cdf_polar(const DistDev& d, double v) {
    if (v <= 0.0) return 0.0;
    // break angles where v / c(theta) = r0 or r1, i.e. sin(theta + phi) = v / (r rho)
    double pts[6];
    int np = 0;
    pts[np++] = d.q0;
    double rr[2] = {d.p0, d.p1};
    for (int k = 0; k < 2; ++k) {
        double w = v / (rr[k] * d.rho);
        if (w < 1.0) {
            double base = asin(w);
            double c1 = base - d.phi, c2 = 3.14159265358979323846 - base - d.phi;
            if (c1 > d.q0 && c1 < d.q1) pts[np++] = c1;
            if (c2 > d.q0 && c2 < d.q1) pts[np++] = c2;
        }
    }
    pts[np++] = d.q1;
    // sort (at most 6 entries)
    for (int i = 1; i < np; ++i)
        for (int j = i; j > 0 && pts[j] < pts[j - 1]; --j) { double t = pts[j]; pts[j] = pts[j - 1]; pts[j - 1] = t; }
    double dr = d.p1 - d.p0, acc = 0.0;
    for (int i = 0; i + 1 < np; ++i) {
        double lo = pts[i], hi = pts[i + 1];
        if (hi <= lo) continue;
        double mid = 0.5 * (lo + hi);
        double rz = v / (d.a * cos(mid) + sin(mid));  // r at which z = v for this angle
        if (rz >= d.p1) acc += hi - lo;
        else if (rz > d.p0) acc += (v * (polar_prim(d, hi) - polar_prim(d, lo)) - d.p0 * (hi - lo)) / dr;
    }
    return acc / (d.q1 - d.q0);
}

__device__ double cdf_any(const DistDev& d, double z) {
    double F = d.kind == XLMIMO_DIST_RECT ? cdf_rect(d, z) : cdf_polar(d, z);
    return fmin(1.0, fmax(0.0, F));
}

constexpr int GL_N = 16;
__constant__ double c_gl_x[GL_N], c_gl_w[GL_N];

// One thread per (panel, node); panel sums reduced per block then by a second pass.
__global__ void quad_kernel(DistDev d, int K, const double* __restrict__ edges, int npanel,
                            double* __restrict__ panel_sum) {
    int gid = blockIdx.x * blockDim.x + threadIdx.x;
    int panel = gid / GL_N, node = gid - panel * GL_N;
    double v = 0.0;
    if (panel < npanel) {
        double lo = edges[panel], hi = edges[panel + 1];
        double h = 0.5 * (hi - lo);
        double z = lo + h * (1.0 + c_gl_x[node]);
        double F = cdf_any(d, z);
        v = h * c_gl_w[node] * pow(F, (double)K);
    }
    // GL_N consecutive lanes form a panel: fixed-order shuffle tree
    for (int off = GL_N / 2; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off, GL_N);
    if (node == 0 && panel < npanel) panel_sum[panel] = v;
}

__global__ void ordered_sum_kernel(const double* __restrict__ x, int n, double* __restrict__ out) {
    __shared__ double sh[STATS_THREADS];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += STATS_THREADS) s += x[i];
    double r = block_sum(s, sh);
    if (threadIdx.x == 0) *out = r;
}

// Gauss-Legendre nodes on [-1, 1] by Newton iteration on P_n (textbook recurrence).
static void gauss_legendre(int n, double* x, double* w) {
    for (int i = 0; i < n; ++i) {
        double z = cos(3.14159265358979323846 * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// Support [z_lo, z_hi] and the kink abscissae of F for one orientation.
static void support_and_kinks(const DistDev& d, std::vector<double>& ks, double* zlo, double* zhi) {
    if (d.kind == XLMIMO_DIST_RECT) {
        double wa = d.a * (d.p1 - d.p0), wb = d.q1 - d.q0;
        double lo = d.a * d.p0 + d.q0;
        *zlo = lo;
        *zhi = lo + wa + wb;
        ks = {lo + fmin(wa, wb), lo + fmax(wa, wb)};
        return;
    }
    // c(theta) extremes on [q0, q1]: end points and the interior maximum at theta = pi/2 - phi
    double cands[3] = {d.q0, d.q1, 1.5707963267948966 - d.phi};
    double cmin = 1e300, cmax = -1e300;
    std::vector<double> cs;
    for (int i = 0; i < 3; ++i) {
        double th = cands[i];
        if (i == 2 && !(th > d.q0 && th < d.q1)) continue;
        double c = d.a * cos(th) + sin(th);
        cs.push_back(c);
        cmin = fmin(cmin, c);
        cmax = fmax(cmax, c);
    }
    *zlo = d.p0 * cmin;
    *zhi = d.p1 * cmax;
    ks.clear();
    for (double c : cs) {
        ks.push_back(d.p0 * c);
        ks.push_back(d.p1 * c);
    }
}

static int expected_max(const DistDev& d, int K, double* result, cudaStream_t st) {
    std::vector<double> ks;
    double zlo, zhi;
    support_and_kinks(d, ks, &zlo, &zhi);
    std::vector<double> br = {zlo, zhi};
    for (double k : ks)
        if (k > zlo && k < zhi) br.push_back(k);
    std::sort(br.begin(), br.end());
    // each segment split into equal panels; F^K steepens near z_hi for large K,
    // so the panels are graded towards the upper end
    const int per_seg = 512;
    std::vector<double> edges;
    for (size_t s = 0; s + 1 < br.size(); ++s) {
        double a = br[s], b = br[s + 1];
        if (!(b > a)) continue;
        for (int i = 0; i < per_seg; ++i) {
            double u = (double)i / per_seg;
            double g = 1.0 - (1.0 - u) * (1.0 - u);  // denser near b
            edges.push_back(a + (b - a) * g);
        }
    }
    edges.push_back(br.back());
    int npanel = (int)edges.size() - 1;
    double *d_edges = nullptr, *d_panel = nullptr, *d_out = nullptr;
    int rc = cuda_status(cudaMallocAsync((void**)&d_edges, edges.size() * sizeof(double), st), "quad alloc");
    if (rc) return rc;
    rc = cuda_status(cudaMallocAsync((void**)&d_panel, (npanel + 1) * sizeof(double), st), "quad alloc");
    if (rc) { cudaFreeAsync(d_edges, st); return rc; }
    d_out = d_panel + npanel;
    cudaMemcpyAsync(d_edges, edges.data(), edges.size() * sizeof(double), cudaMemcpyHostToDevice, st);
    int threads = 256;
    int blocks = (npanel * GL_N + threads - 1) / threads;
    quad_kernel<<<blocks, threads, 0, st>>>(d, K, d_edges, npanel, d_panel);
    rc = cuda_status(cudaGetLastError(), "quad launch");
    if (!rc) {
        ordered_sum_kernel<<<1, STATS_THREADS, 0, st>>>(d_panel, npanel, d_out);
        rc = cuda_status(cudaGetLastError(), "quad sum launch");
    }
    double integral = 0.0;
    if (!rc) rc = cuda_status(cudaMemcpyAsync(&integral, d_out, sizeof(double), cudaMemcpyDeviceToHost, st), "quad copy");
    cudaFreeAsync(d_edges, st);
    cudaFreeAsync(d_panel, st);
    if (!rc) rc = cuda_status(cudaStreamSynchronize(st), "quad sync");
    *result = zhi - integral;
    return rc;
}

int saturation_analytic(const xlmimo_user_dist* dist, int K, double t, double spacing, double* out,
                        cudaStream_t st) {
    static bool gl_ready = false;
    static double gx[GL_N], gw[GL_N];
    if (!gl_ready) {
        gauss_legendre(GL_N, gx, gw);
        gl_ready = true;
    }
    int rc = cuda_status(cudaMemcpyToSymbolAsync(c_gl_x, gx, sizeof(gx), 0, cudaMemcpyHostToDevice, st), "gl nodes");
    if (!rc) rc = cuda_status(cudaMemcpyToSymbolAsync(c_gl_w, gw, sizeof(gw), 0, cudaMemcpyHostToDevice, st), "gl w");
    if (rc) return rc;
    DistDev up{};
    up.kind = dist->kind;
    up.a = t / sqrt(1.0 - t * t);
    up.rho = sqrt(1.0 + up.a * up.a);
    up.phi = atan(up.a);
    up.p0 = dist->a0;
    up.p1 = dist->a1;
    up.q0 = dist->b0;
    up.q1 = dist->b1;
    if (up.kind == XLMIMO_DIST_POLAR) {
        // c(theta) > 0 needed on both orientations
        double lo = fmin(up.q0, -up.q1), hi = fmax(up.q1, -up.q0);
        if (!(lo + up.phi > 0.0 && hi + up.phi < 3.14159265358979323846)) {
            set_error("polar angle range makes a t/sqrt(1-t^2) cos(theta) +- sin(theta) non-positive");
            return XLMIMO_EINVAL;
        }
    }
    // y_down = -max_k (a x_k - y_k): the same problem with y (or theta) reflected
    DistDev dn = up;
    dn.q0 = -up.q1;
    dn.q1 = -up.q0;
    double e_up = 0.0, e_dn = 0.0;
    rc = expected_max(up, K, &e_up, st);
    if (!rc) rc = expected_max(dn, K, &e_dn, st);
    if (rc) return rc;
    e_dn = -e_dn;
    out[0] = e_up;
    out[1] = e_dn;
    out[2] = (e_up - e_dn) / spacing;
    out[3] = ceil(out[2]);
    // the quadrature carries the ratio to ~1e-9 relative; within 1e-6 of an
    // integer m (relative) its ceiling is not decided, and both m and m + 1
    // are reported
    const double m = rint(out[2]);
    const bool near = fabs(out[2] - m) <= XLMIMO_SAT_NEAR_REL * fmax(1.0, fabs(out[2]));
    out[4] = near ? 1.0 : 0.0;
    out[5] = near ? (out[3] == m ? m + 1.0 : m) : out[3];
    return XLMIMO_OK;
}

}  // namespace xl
