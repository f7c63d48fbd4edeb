/*
 * xlmimo.h -- C interface of the GB300 (sm_103a) Monte-Carlo engine for
 * near-field XL-MIMO multiuser beamforming (Cui, Park, Alouini, "Channel
 * Capacity Saturation Point and Beamforming Acceleration for Near-Field
 * XL-MIMO Multiuser Communications").
 *
 * Problem statement (Sec. II): an uplink with one base station whose
 * uniform linear array of N elements lies on the y axis, centred at the
 * origin, element n = 0..N-1 at y_n = (n - (N-1)/2) * spacing (Sec. II-A);
 * K single-antenna users at (x_k, y_k), x_k > 0; carrier wavelength lambda;
 * transmit power p_k per user (E[x x^H] = P I in Eq. 1, generalised to
 * diag(p)); white noise of power sigma^2 per element (Eq. 1).
 *
 * Conventions for every call:
 *   - All array arguments are DEVICE pointers owned by the caller unless a
 *     comment says "host".  The library never frees caller memory.
 *   - Every call is asynchronous on `stream` (a cudaStream_t; NULL = the
 *     legacy default stream) and makes no implicit device synchronisation,
 *     except those documented as synchronous.
 *   - Returns an xlmimo_status.  XLMIMO_EINVAL is returned before any work is
 *     enqueued; the reason is in xlmimo_last_error() (thread-local).
 *     XLMIMO_ECUDA reports a CUDA launch or runtime error.  No C++ exception
 *     crosses this interface.
 *   - B == 0 is a valid empty batch: nothing is enqueued, XLMIMO_OK (except
 *     that xlmimo_sumrate writes the empty batch's statistics {0, 0, 0} to a
 *     given `stats`).
 *   - Complex numbers are interleaved (re, im) doubles.  A Gram matrix batch
 *     is [B][K][K] complex, row-major, G[b][i][j] = h_i^H h_j (conjugate on
 *     the row user, as rho_ij of Sec. III), both triangles written.
 *   - User positions are [B][K][2] doubles (x, y) in metres.  A trial with a
 *     user at x <= 0 or a non-finite coordinate gets a NaN Gram matrix.
 *   - K is limited to 1..XLMIMO_MAX_USERS.
 */
#ifndef XLMIMO_H
#define XLMIMO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define XLMIMO_MAX_USERS 64

typedef enum {
    XLMIMO_OK = 0,
    XLMIMO_EINVAL = 1,       /* bad argument; nothing enqueued */
    XLMIMO_ECUDA = 2,        /* CUDA runtime or launch error */
    XLMIMO_ENOMEM = 3,       /* device workspace allocation failed */
    XLMIMO_ESINGULAR = 4,    /* per-trial status: receiver matrix singular */
    XLMIMO_ETIMEOUT = 5,     /* a bounded device-side wait gave up */
    XLMIMO_EUNSUPPORTED = 6  /* valid request this build or device cannot serve */
} xlmimo_status;

/* Channel models.
 *   XLMIMO_PNUSW    Eq. (3): h_k(n) = sqrt(beta0) e^{-j 2 pi r/lambda} / r * sqrt(x_k / r)
 *   XLMIMO_FSPL_USW free-space spherical wave: h_k(n) = lambda / (4 pi r) e^{-j 2 pi r/lambda}
 *   XLMIMO_UPW      planar wave (the far-field model compared in Sec. V-A):
 *                   h_k(n) = sqrt(beta0) / r_k e^{-j 2 pi (r_k - y_n sin theta_k) / lambda}
 *   with r = sqrt(x_k^2 + (y_n - y_k)^2), r_k = sqrt(x_k^2 + y_k^2),
 *   sin theta_k = y_k / r_k. */
typedef enum { XLMIMO_PNUSW = 0, XLMIMO_FSPL_USW = 1, XLMIMO_UPW = 2 } xlmimo_model;

/* Arithmetic of the exact Gram accumulation.  Accuracy is stated normwise,
 * max_ij |dG_ij| / sqrt(G_ii G_jj) against the FP64 definition, as measured
 * and as the tests bound it; it does not grow with N.
 *   XLMIMO_F64    FP64 generation and FP64 accumulation (SIMT): 1e-12, or the
 *                 FP64 rounding of the phase 2 pi r / lambda where larger.
 *   XLMIMO_F32    FP32 generation with a double-float phase reference every 128
 *                 elements, FP32 accumulation (SIMT): ~5e-7 (bound 1e-5).
 *   XLMIMO_BF16   FP32 generation (reference every 256 elements, then a local
 *                 expansion per 8 elements); each entry rounded to one BF16
 *                 number; tensor cores (tcgen05) with FP32 accumulation in
 *                 TMEM, added into a running total every 64 accumulations:
 *                 ~3e-3 (bound 1e-2).
 *   XLMIMO_BF16X3 as XLMIMO_BF16 with each entry split h = hi + lo into two BF16
 *                 parts and the products hi*hi + hi*lo + lo*hi accumulated:
 *                 ~5e-6 (bound 2e-5).
 *   XLMIMO_F16X3  as XLMIMO_BF16X3 in FP16, after scaling user k's entries by
 *                 1/|h_k| at the array centre (undone in FP64): ~3e-6 (bound
 *                 2e-5; limited by the FP32 generation and the tensor cores'
 *                 FP32 accumulation, which rounds towards zero).
 * The tensor-core precisions need an sm_103 device. */
typedef enum {
    XLMIMO_F64 = 0,
    XLMIMO_F32 = 1,
    XLMIMO_BF16 = 2,
    XLMIMO_BF16X3 = 3,
    XLMIMO_F16X3 = 4
} xlmimo_prec;

/* Aperture-aware closed form (not the paper's; NEXT item of the paper's
 * modified ZF): the stationary-phase off-diagonal of Eq. (6) (and its
 * free-space analogue) assumes the stationary point of the pair phase lies
 * inside an unbounded aperture.  The point is where the line through the
 * two users meets the array axis, y* = y_i - x_i (y_j - y_i)/(x_j - x_i).
 *   XLMIMO_APERTURE_MASK     drop the term when |y*| > N spacing / 2;
 *   XLMIMO_APERTURE_FRESNEL  multiply it by the finite-aperture factor of the
 *       quadratic phase, F = [(C(u_hi) - C(u_lo)) + j s (S(u_hi) - S(u_lo))]
 *       / (1 + j s), u = (edge - y*) sqrt(|phi''|/pi), s = sign(phi''),
 *       phi'' = (2 pi/lambda)(x_i^2/r_i^3 - x_j^2/r_j^3) at y*, C, S the
 *       Fresnel integrals; an edge beyond |u| = 2 counts at its limit 1/2
 *       (the quadratic model's oscillating tail has the wrong phase there).
 * The diagonal is the closed form's. */
typedef enum { XLMIMO_APERTURE_NONE = 0, XLMIMO_APERTURE_MASK = 1, XLMIMO_APERTURE_FRESNEL = 2 } xlmimo_aperture;

/* Linear receivers (Sec. V): ZF (Eq. 21), MMSE, MRC; and ZF precoding on
 * the downlink, which the paper leaves to the reader (Sec. II). */
typedef enum { XLMIMO_ZF = 0, XLMIMO_MMSE = 1, XLMIMO_MRC = 2, XLMIMO_ZF_DL = 3 } xlmimo_scheme;
/* OR-ed into the scheme of xlmimo_beamform: the mismatched SINR from the
 * FP32 correction (see xlmimo_beamform).  No effect on matched receivers. */
#define XLMIMO_MISMATCH_FP32 0x100
/* OR-ed into the scheme of a matched receiver (gram_true NULL or equal to
 * gram_filter): its Cholesky factorisation in double-float on the FP32 pipe
 * (~2^-48 relative), in FP64 when a pivot falls below 2^-16 of its diagonal
 * entry (an ill-conditioned system: closely spaced users), the rule that the
 * mismatched filter always follows.  Ignored where the capacity is asked for
 * (its log-determinant comes from FP64 pivots).  The ragged batch's receivers
 * take it. */
#define XLMIMO_FACTOR_FF 0x200

/* How beamform() reads `power`:
 *   XLMIMO_POWER_ABS    power[b][k] is the transmit power p_k.
 *   XLMIMO_POWER_RXSNR  power[b][k] is user k's received SNR on its own,
 *                       p_k G_kk / sigma^2 with G the TRUE Gram matrix, so
 *                       p_k = power[b][k] * sigma^2 / G_kk. */
typedef enum { XLMIMO_POWER_ABS = 0, XLMIMO_POWER_RXSNR = 1 } xlmimo_power_mode;

/* Array geometry and channel model (Sec. II-A, II-B). */
typedef struct {
    int64_t n_ant;      /* 1 <= N <= 2^40 */
    double wavelength;  /* lambda > 0 [m] */
    double spacing;     /* element spacing > 0 [m]; the paper uses lambda / 2 */
    double beta0;       /* channel gain constant of PNUSW / UPW (the paper sets 1) */
    int32_t model;      /* xlmimo_model */
    int32_t reserved;   /* must be 0 */
} xlmimo_array;

/* Exact Gram matrices H^H H of B independent trials (Sec. III: received
 * power P_i = P ||h_i||^2 on the diagonal, h_i^H h_j off it; Sec. V-B: the
 * inner products that dominate ZF).  The channel entries are generated on
 * the fly from the geometry and never stored.
 *   users : [B][K][2] doubles (device)
 *   gram  : [B][K][K] complex doubles (device, written)
 *   prec  : xlmimo_prec
 * Needs device workspace only when the element range is split, the partial
 * sums then reduced in a fixed order: when B is too small to fill the GPU,
 * and on the tensor cores for arrays longer than 2^36 elements; that
 * workspace (B x chunks x K x K complex doubles) is stream-ordered memory of
 * the current device. */
int xlmimo_channel_gram(const xlmimo_array* arr, const double* users, int K, int B, int prec,
                        double* gram, void* stream);

/* Exact Gram matrices of a uniform rectangular array (URA), the planar array
 * the paper names as an extension in the footnote of Sec. II: `rows` rows of
 * arr->n_ant elements on the square lattice of arr->spacing in the y-z plane,
 * element (q, n) at (0, y_n, z_q), z_q = (q - (rows-1)/2) spacing, y_n as for
 * the ULA; users in the plane z = 0.  The channel models of xlmimo_model with
 * the 3-D distance r = sqrt(x^2 + (y_n-y)^2 + z_q^2) (PNUSW keeps the
 * projection sqrt(x / r) on the array normal; UPW is the planar wave of a user
 * at elevation 0).  rows = 1 is xlmimo_channel_gram.
 *   rows  : 1..XLMIMO_MAX_URA_ROWS, n_ant * rows <= 2^40
 *   users : [B][K][2] doubles (device, caller-owned), (x, y) as for the ULA
 *   prec  : xlmimo_prec, accuracy class as for the ULA
 *   gram  : [B][K][K] complex doubles (device, caller-owned, written),
 *           G[b][i][j] = h_i^H h_j over all rows * n_ant elements
 * Computed per row pair: rows at +-z_q see the users alike, and row q sees
 * them as the ULA sees users moved to x' = sqrt(x^2 + z_q^2).  At
 * XLMIMO_BF16X3 with n_ant a multiple of 128 up to 1024 (PNUSW, free space)
 * the tensor-core Gram accumulates all ceil(rows/2) row pairs of a trial in
 * one pass; otherwise ceil(rows/2) ULA Grams are summed with the weights of
 * the amplitude (one for UPW) in stream-ordered device workspace (up to
 * 1 GiB, or one trial's ceil(rows/2) K x K Grams if larger).  Asynchronous on
 * `stream`.  A trial with an invalid user (x <= 0 or not finite) gets NaN.
 * Errors: XLMIMO_EINVAL (arguments), XLMIMO_ENOMEM, XLMIMO_EUNSUPPORTED
 * (tensor-core precisions off sm_103), XLMIMO_ECUDA. */
#define XLMIMO_MAX_URA_ROWS 1048576
int xlmimo_channel_gram_ura(const xlmimo_array* arr, int64_t rows, const double* users, int K, int B, int prec,
                            double* gram, void* stream);

/* Size of the fixed device scratch used by xlmimo_channel_gram_noalloc, in MiB. */
#define XLMIMO_NOALLOC_SCRATCH_MIB 16

/* xlmimo_channel_gram without any device memory allocation.  The paper has
 * no counterpart: this serves callers that cannot allocate device memory
 * while they run -- for example an application that reserves the GPU's
 * memory for its own pool at start-up and forbids later allocations, or a
 * latency-critical loop that cannot accept cudaMalloc / cudaFree, which may
 * block or synchronise the device.  Arguments, results and precisions
 * (XLMIMO_F64 and XLMIMO_F32; the tensor-core precisions return
 * XLMIMO_EUNSUPPORTED) are
 * those of xlmimo_channel_gram, with the same element split and the same
 * summation order.
 * When the batch is too small to fill the GPU, the partial Gram matrices of
 * the element chunks go to a fixed device array of XLMIMO_NOALLOC_SCRATCH_MIB
 * MiB that every GPU which loads this library holds until the process exits.
 * A call whose split needs more than that (B x chunks x K x K x 16 bytes) is
 * rejected with XLMIMO_EINVAL and a message saying how much it needed;
 * nothing is enqueued.  Every call shares the array and it keeps the last
 * call's contents; nothing in it needs to start at zero, because each chunk's
 * partial is written in full before it is summed.  Calls that overlap on the
 * GPU (on different streams, or from different host threads) race on it:
 * serialise them.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) once for that device; make that first call
 * before any stream capture.  No cudaMalloc, cudaFree or allocating library
 * routine is called. */
int xlmimo_channel_gram_noalloc(const xlmimo_array* arr, const double* users, int K, int B, int prec,
                                double* gram, void* stream);

/* Closed-form Gram matrices of "modified ZF" (Sec. V-B): diagonal P_i / P
 * from Eq. (4), off-diagonal rho_ij sqrt(P_i P_j) / P with rho_ij from
 * Eq. (6) (SPM correlation).  Written for the PNUSW model exactly as the
 * paper gives it (element spacing generalised: 2/lambda -> 1/spacing,
 * M lambda -> 2 N spacing).  For XLMIMO_FSPL_USW the same derivation
 * (Riemann integral, stationary phase) is applied to the amplitude
 * lambda / (4 pi r): diagonal (lambda/4pi)^2 (atan((D/2-y)/x) + atan((D/2+y)/x)) / (spacing x),
 * off-diagonal (lambda/4pi)^2 / spacing * sqrt(lambda / (d x_i x_j)) e^{j sgn(x_i-x_j)(2 pi d/lambda - pi/4)},
 * D = N spacing, d = |user_i - user_j|.  For XLMIMO_UPW the exact
 * Dirichlet-kernel form is written.  O(K^2) per trial, FP64.
 *   users : [B][K][2] doubles (device);  gram : [B][K][K] complex doubles (device, written) */
int xlmimo_corr_closed_form(const xlmimo_array* arr, const double* users, int K, int B,
                            double* gram, void* stream);

/* xlmimo_corr_closed_form followed by the finite-aperture correction `mode`
 * (xlmimo_aperture) of every off-diagonal entry; same layout. */
int xlmimo_corr_closed_form_aperture(const xlmimo_array* arr, const double* users, int K, int B, int mode,
                                     double* gram, void* stream);

/* Per-user SINR of a linear receiver built from gram_filter and applied to
 * the channel whose Gram matrix is gram_true (Sec. V; with gram_filter the
 * closed form this is "modified ZF").  A receiver W^H = M H^H gives
 *   SINR_k = p_k |(M G)_kk|^2 / (sum_{j!=k} p_j |(M G)_kj|^2 + sigma^2 (M G M^H)_kk)
 * with M = Gf^{-1} (ZF), (Gf + sigma^2 diag(p)^{-1})^{-1} (MMSE), I (MRC).
 * When gram_true is NULL (or equal to gram_filter) the matched forms are
 * used: ZF p_k / (sigma^2 [G^{-1}]_kk), MMSE p_k / (sigma^2 [Z^{-1}]_kk) - 1
 * with Z = G + sigma^2 diag(p)^{-1}, MRC p_k G_kk^2 / (sum_{j!=k} p_j |G_kj|^2 + sigma^2 G_kk).
 * XLMIMO_ZF_DL (downlink ZF precoding, total power P_T = sum_k p_k): the
 * precoder W = beta H M, M = Gf^{-1}, beta^2 = P_T / tr(M G M^H), gives user k
 *   SINR_k = beta^2 |(M G)_kk|^2 / (beta^2 sum_{j!=k} |(M G)_jk|^2 + sigma^2),
 * matched: P_T / (sigma^2 tr(G^{-1})) for every user.
 * Solves use an FP64 Cholesky factorisation in shared memory, except for
 * the filter of a mismatched receiver, factored in double-float (FP32 pairs,
 * ~2^-48) unless a pivot falls below 2^-16 of its diagonal entry
 * (ill-conditioned: FP64); a matrix that is not numerically positive
 * definite falls back to LU with partial pivoting.  Mismatched SINRs: by
 * default (M G) is formed in double-float (~1e-7 relative or better on the
 * tested cases); with scheme | XLMIMO_MISMATCH_FP32 only the correction
 * B = M (G - Gf) - M diag(sigma^2/p) of M G = I + B is formed, in FP32 (MRC:
 * B = G): |dB_kj| <= (K + 2) 2^-24 (|M| |G - Gf|)_kj + 3 2^-24 |M_kj| sigma^2/p_j
 * + 2^-24 |B_kj|, tens of times cheaper; ~1e-8 relative where the filter's
 * Gram is accurate (the closed form at large N), up to ~1e-4 on the sum rate
 * where interference dominates (the closed form at small N).
 *   gram_filter, gram_true : [B][K][K] complex doubles (device; gram_true may be NULL)
 *   power  : [B][K] doubles (device), read per power_mode
 *   noise  : [B] doubles (device), sigma^2 > 0 per trial
 *   sinr   : [B][K] doubles (device, written)
 *   trial_status : [B] ints (device, written): 0 ok, 1 Cholesky failed and LU
 *            was used, 4 (XLMIMO_ESINGULAR) singular: that trial's SINRs are 0
 *   capacity : [B] doubles (device, written) or NULL:
 *            log2 det(I + sigma^{-2} diag(p)^{1/2} G diag(p)^{1/2}) with G the
 *            true Gram matrix (Eq. 9 with per-user powers). */
int xlmimo_beamform(const double* gram_filter, const double* gram_true, const double* power,
                    const double* noise, int K, int B, int scheme, int power_mode, double* sinr,
                    int* trial_status, double* capacity, void* stream);

/* Sum rate R_b = sum_k log2(1 + SINR_bk) of every trial, and the batch
 * statistics {mean, M2 = sum_b (R_b - mean)^2, count} reduced in a fixed
 * order (deterministic).
 *   sinr : [B][K] doubles (device);  rate : [B] doubles (device, written)
 *   stats : 3 doubles (device, written) or NULL */
int xlmimo_sumrate(const double* sinr, int K, int B, double* rate, double* stats, void* stream);

/* Per-trial power-saturation interval (Sec. IV-A, Eqs. 13-16):
 *   y_up = max_k x_k t / sqrt(1-t^2) + y_k,  y_down = min_k -x_k t / sqrt(1-t^2) + y_k
 * and n_sat = ceil((y_up - y_down) / spacing), the element count spanning it.
 *   users : [B][K][2] doubles (device);  0 < t < 1;  spacing > 0
 *   sat   : [B][3] doubles (device, written) {y_up, y_down, n_sat} */
int xlmimo_saturation(const double* users, int K, int B, double t, double spacing, double* sat,
                      void* stream);

/* User distributions for the ergodic saturation point. */
typedef enum { XLMIMO_DIST_RECT = 0, XLMIMO_DIST_POLAR = 1 } xlmimo_dist_kind;

typedef struct {
    int32_t kind;       /* xlmimo_dist_kind */
    int32_t reserved;   /* must be 0 */
    double a0, a1;      /* RECT: x in [a0, a1] (0 < a0 < a1);  POLAR: r in [a0, a1] (0 < a0 < a1) */
    double b0, b1;      /* RECT: y in [b0, b1];  POLAR: theta in [b0, b1] radians from broadside,
                           with a t/sqrt(1-t^2) cos(theta) + |sin(theta)| > 0 on the range */
} xlmimo_user_dist;

/* Ergodic saturation interval and antenna count (Sec. IV-B and Appendix B):
 * E[y_up] = int y d(F_z(y)^K) with F_z the CDF of z = x t/sqrt(1-t^2) + y for
 * one user, and E[y_down] = -E[max_k(x_k t/sqrt(1-t^2) - y_k)]; for the
 * rectangle these equal Eqs. (17)-(18).  Evaluated on the device in FP64 by
 * composite Gauss-Legendre quadrature of the closed-form CDF.
 * SYNCHRONOUS: returns host results.
 *   out : 6 doubles (host, written)
 *         {E[y_up], E[y_down], v = (E[y_up]-E[y_down])/spacing, ceil(v), near, other}
 *   The quadrature carries v to ~1e-9 relative.  When v lies within
 *   XLMIMO_SAT_NEAR_REL * max(1, v) of an integer m, the ceiling is not
 *   decided by the computation: near = 1 and {ceil(v), other} = {m, m + 1},
 *   both candidates.  Otherwise near = 0 and other = ceil(v). */
#define XLMIMO_SAT_NEAR_REL 1e-6
int xlmimo_saturation_analytic(const xlmimo_user_dist* dist, int K, double t, double spacing,
                               double* out, void* stream);

/* Appendix A: the influence of the off-diagonal Gram entries on the capacity.
 * For each trial b, with R the users' correlation matrix (r_ij = h_i^H h_j /
 * (|h_i| |h_j|), h_k the exact channel of user k on the array) and every user
 * at receive SNR `snr` (linear; a_i = snr is the i-th diagonal element of
 * (P/sigma_n^2) H^H H):
 *   out[4b + 0] = log2 det R              (-(1/K) of it is Fig. 5's -E_K[log2 lambda^R])
 *   out[4b + 1] = log2 det(I + snr R)     (the capacity C)
 *   out[4b + 2] = K log2(1 + snr)         (log2 U, Hadamard's upper bound)
 *   out[4b + 3] = log2 det R + log2 U     (log2 L, the Schur-Horn lower bound)
 * K is 1..XLMIMO_MAX_BOUNDS_USERS (Fig. 5 reaches K = 1000); users[b][k][2]
 * positions on the device as for xlmimo_channel_gram; out on the device.
 * Channels are generated in FP32 (span-referenced phase) and stored as a BF16
 * split h = h_hi + h_lo; the real Gram of [Re H; Im H] runs on the tensor
 * cores as hi*hi + lo*hi + hi*lo with FP32 totals (each product within
 * 3 * 2^-16 of |h_i,n||h_j,n|, ~1e-6 relative per correlation entry in
 * practice); the blocked Cholesky factorisations of R and I + snr R run in
 * FP64 on their diagonal blocks and in double-float (FP32 pairs, ~2^-48) on
 * their panels and trailing updates.  A trial whose R is not numerically
 * positive definite (coincident users) gets NaN.
 * Asynchronous on `stream`; allocates 8*B*Kp*Np + 16*B*Kp^2 + 32*B*Kp^2 + 16*B
 * bytes (Kp = K rounded up to 64, Np = n_ant rounded up to 64) of
 * stream-ordered workspace and frees it.
 * XLMIMO_EINVAL for K out of range, snr < 0 or NULL pointers. */
#define XLMIMO_MAX_BOUNDS_USERS 1024
int xlmimo_capacity_bounds(const xlmimo_array* arr, const double* users, int K, int B, double snr,
                           double* out, void* stream);

/* xlmimo_capacity_bounds with the device time of each of its phases, for
 * measurement: phase_ms[5] (host, written) = {channels, tensor-core Gram,
 * correlation matrices, Cholesky factorisations, bounds} in milliseconds,
 * from CUDA events recorded on `stream` between the phases.  Same inputs,
 * outputs, workspace and errors as xlmimo_capacity_bounds, plus
 * XLMIMO_EINVAL for a NULL phase_ms.  SYNCHRONOUS: returns once the work is
 * done. */
int xlmimo_capacity_bounds_timed(const xlmimo_array* arr, const double* users, int K, int B, double snr,
                                 double* out, float* phase_ms, void* stream);

/* Capacity-saturation sweep (Sec. IV-C, Fig. 3; Sec. V-C, Fig. 4): for each
 * array size in n_list, over the same B trials of users, the exact Gram (at
 * `prec`) and the closed-form Gram, ZF and MMSE sum rates (exact receiver,
 * and the receiver from the closed form judged on the exact channel) and
 * the capacity, at every SNR.  The transmit power is the same for every
 * N: p = snr * sigma^2 / g_lim, g_lim the large-N limit of ||h||^2 for a
 * reference user at (ref_x, 0) (Eq. 5 for PNUSW; pi (lambda/4pi)^2 / (spacing ref_x)
 * for the free-space model; for UPW N-proportional, so the reference
 * array size n_list[last] is used), sigma^2 = 1.
 * SYNCHRONOUS: returns host results.  Allocates its device buffers with
 * stream-ordered allocation and frees them before returning. */
typedef struct {
    double wavelength, spacing, beta0;
    int32_t model;        /* xlmimo_model */
    int32_t prec;         /* xlmimo_prec of the exact Gram */
    int32_t n_count;      /* number of array sizes */
    int32_t snr_count;    /* number of SNR points */
    const int64_t* n_list;   /* host [n_count] */
    const double* snr_db;    /* host [snr_count] */
    const double* users;     /* device [B][K][2] */
    int32_t K, B;
    double t;             /* saturation threshold for the per-trial interval */
    double ref_x;         /* reference user distance for the power normalisation */
} xlmimo_sweep_cfg;

typedef struct {
    /* all host arrays, caller-allocated, written by the call */
    double* rate;         /* [n_count][2 path: exact, closed][2 scheme: ZF, MMSE][snr_count] trial means */
    double* capacity;     /* [n_count][snr_count] trial means of log2 det (Eq. 9) */
    double* gram_err;     /* [n_count] max over trials and entries of |G~ - G|_ij / sqrt(G_ii G_jj) */
    double sat_mean[3];   /* trial means of {y_up, y_down, n_sat} (Eqs. 15-16) */
} xlmimo_sweep_result;

int xlmimo_capacity_sweep(const xlmimo_sweep_cfg* cfg, xlmimo_sweep_result* res, void* stream);

/* One Monte-Carlo step over a batch of trials: the whole path of Secs. II-V
 * in one call.  For every trial: exact Gram (channel generated on the fly,
 * at `prec`), receiver `scheme` on it with SINR, status and capacity, sum
 * rate; the closed-form Gram of modified ZF (Sec. V-B) and the receiver
 * `cf_scheme` built from it and judged on the exact channel, with its sum
 * rate; and the per-trial saturation interval (Eqs. 15-16).
 * The batch is cut into `chunks` pieces that flow through three streams: the
 * Gram kernels run on `stream` while the receivers of the previous piece run
 * on two streams owned by the library (one pair per device, created on first
 * use): the exact receivers on one, the closed-form ones beside them on the
 * other, so the generation/tensor-core work and the FP64 solves overlap.  The
 * call returns once everything is enqueued; all work is ordered before any
 * later work on `stream`.  Concurrent calls on different streams of one
 * device share the library's streams and are serialised on them.  Batch statistics {mean, M2, count} of both rates are
 * reduced over the whole batch in a fixed order.  With an exact Gram below
 * FP64 (prec != XLMIMO_F64) the closed-form receiver takes
 * XLMIMO_MISMATCH_FP32, whose error lies far below that Gram's own. */
typedef struct {
    xlmimo_array arr;         /* array geometry and channel model */
    int32_t prec;             /* xlmimo_prec of the exact Gram */
    int32_t scheme;           /* xlmimo_scheme on the exact Gram */
    int32_t cf_scheme;        /* xlmimo_scheme built from the closed form; -1 skips the closed-form path */
    int32_t power_mode;       /* xlmimo_power_mode */
    int32_t K, B;
    int32_t chunks;           /* pipeline pieces, 1..64; 0 chooses automatically */
    int32_t reserved;         /* must be 0 */
    double t;                 /* saturation threshold in (0, 1); 0 skips the saturation interval */
    const double* users;      /* device [B][K][2] */
    const double* power;      /* device [B][K] */
    const double* noise;      /* device [B] */
    double* gram;             /* device [B][K][K] complex, written */
    double* gram_cf;          /* device [B][K][K] complex, written (NULL if cf_scheme < 0) */
    double* sinr;             /* device [B][K], written */
    double* sinr_cf;          /* device [B][K], written (NULL if cf_scheme < 0) */
    int32_t* status;          /* device [B], written */
    int32_t* status_cf;       /* device [B], written (NULL if cf_scheme < 0) */
    double* capacity;         /* device [B], written, or NULL */
    double* rate;             /* device [B], written */
    double* rate_cf;          /* device [B], written (NULL if cf_scheme < 0) */
    double* stats;            /* device [3], written, or NULL */
    double* stats_cf;         /* device [3], written, or NULL */
    double* sat;              /* device [B][3], written (NULL if t == 0) */
} xlmimo_mc_batch;

int xlmimo_mc_step(const xlmimo_mc_batch* job, void* stream);

/* ---- Ragged batches --------------------------------------------------------
 * Many independent instances with their own array size, user count,
 * receiver and noise, evaluated together: exact Gram (tensor cores), receiver
 * SINR and sum rate per instance.  A plan fixes the instance list once
 * (host side: work items ordered longest first, instances grouped by user
 * count, device tables and workspace allocated, tile shapes optionally
 * chosen by timing candidates on sample inputs); running a plan only
 * enqueues kernels -- no allocation, no synchronisation -- so it may be
 * captured in a CUDA graph and replayed.  The paper's problem is one
 * instance; batching many is this library's Monte-Carlo engine. */
typedef struct {
    int64_t n_ant;     /* N of this instance, 1 .. 2^40 */
    int32_t k;         /* users, 1 .. XLMIMO_MAX_USERS */
    int32_t scheme;    /* xlmimo_scheme of its receiver (matched, on the exact Gram) */
    int64_t user_off;  /* first user of the instance in the packed users / power / sinr arrays */
    int64_t gram_off;  /* first complex entry of its K x K Gram in the packed Gram array */
    double noise;      /* sigma^2 > 0 */
} xlmimo_inst;

typedef struct xlmimo_batch_plan_st* xlmimo_batch_plan;

/* Build a plan for `count` instances (host array `insts`) sharing the
 * wavelength, spacing, beta0 and model of *geo (geo->n_ant is ignored).
 * prec: XLMIMO_BF16, XLMIMO_BF16X3 or XLMIMO_F16X3.  Work items (instance,
 * element chunk) run one per CTA of the tensor-core Gram kernel, in one of two
 * tilings: the narrow one (M = 128, N = 64 MMAs over 32 user lanes, three CTAs
 * per SM) for instances with K up to the plan's narrow cut-off, the wide one
 * (M = N = 128 MMAs over 64 user slots, two CTAs per SM) for the others.
 * With packing, narrow work items ride in the spare user slots of wide CTAs
 * or share a narrow CTA's 32, when the user counts fit and the lengths are
 * within 3/4 of the CTA's longest.  If
 * tune_users (device, packed [sum K][2]) is non-NULL the plan times
 * candidates on those users (Gram phase only) and keeps the fastest: element
 * chunks of 4096, 8192, 16384, 32768 and 131072 elements x the two launch
 * modes with cut-off 32 and packing, then cut-offs 16 and 0 (every instance
 * on the wide tiling) and no packing at the best of those; otherwise it takes
 * 8192 elements, launch mode 2, cut-off 32 and packing.  The accumulator's periodic drain keeps every chunk
 * length accurate, so the chunk trades load balance against partial sums.
 * SYNCHRONOUS on `stream`. */
int xlmimo_batch_plan_create(const xlmimo_array* geo, const xlmimo_inst* insts, int count, int prec,
                             const double* tune_users, xlmimo_batch_plan* plan, void* stream);

/* Run a plan: users [sum K][2], power [sum K] (read per power_mode) in;
 * gram (packed complex, at each gram_off), sinr [sum K], status [count],
 * rate [count] out (all device).  Asynchronous on `stream`; capturable.
 * With sinr, status and rate all NULL (power then unused) only the Gram
 * matrices are computed. */
int xlmimo_batch_run(xlmimo_batch_plan plan, const double* users, const double* power, int power_mode,
                     double* gram, double* sinr, int32_t* status, double* rate, void* stream);

/* Pin a plan's tiling, overriding the tuner: element chunk per work item (a
 * positive multiple of 128 up to 2^30), launch mode (1 or 2, as in
 * xlmimo_batch_plan_info), narrow cut-off (0 to 32: instances with K up to it
 * on the narrow tiling, the others on the wide one) and pack (1: items share
 * CTAs, 0: one per CTA).  Waits for the device to finish pending work
 * (runs may still read the plan's tables), then rebuilds the tables;
 * SYNCHRONOUS on `stream`.  The plan then reports tuned = 0.  If the wait
 * fails the plan is left as it was; if the rebuild fails (XLMIMO_ENOMEM, ...)
 * the plan keeps no tables and xlmimo_batch_run refuses it (XLMIMO_EINVAL)
 * until a later call succeeds. */
int xlmimo_batch_plan_set_tiling(xlmimo_batch_plan plan, int64_t chunk, int mode, int narrow_kmax, int pack,
                                 void* stream);

/* Plan facts (host, written; XLMIMO_PLAN_INFO_LEN entries): {work items,
 * element chunk per item, launch mode (1: the narrow and the wide items
 * launched one after the other, 2: both launches at once on two streams),
 * instances with K <= 32, instances with K > 32, workspace bytes, tuned
 * (0/1), candidates timed, narrow cut-off (largest K on the narrow tiling),
 * CTAs of the wide tiling, packing (0/1), CTAs of the narrow tiling}. */
#define XLMIMO_PLAN_INFO_LEN 12
int xlmimo_batch_plan_info(xlmimo_batch_plan plan, int64_t* info);

int xlmimo_batch_plan_destroy(xlmimo_batch_plan plan);

/* ---- Learned correlation surrogate ------------------------------------------
 * Not part of the paper.  A multilayer perceptron corrects the closed-form
 * correlation of modified ZF (Sec. V-B, Eqs. 4 and 6, and its free-space
 * analogue): for a user pair i < j it predicts t_ij from the pair's geometry,
 * and the surrogate Gram is G~_ij (F_ij + t_ij) off the diagonal (its
 * conjugate mirrored below), the closed-form G~_ii on it, F_ij the
 * finite-aperture factor `base` (xlmimo_aperture; XLMIMO_APERTURE_NONE: F = 1).
 * It is trained on targets t_ij = G_ij / G~_ij - F_ij from the exact Gram:
 * the ratio removes the fast 2 pi d / lambda phase that the closed form
 * already carries, so what is left is a smooth function of the geometry
 * (with base NONE: about 0 where the stationary point of the phase lies
 * inside the aperture, about -1 where it lies outside and the exact entry is
 * small; with MASK or FRESNEL that step is taken analytically).
 *
 * Architecture: XLMIMO_MLP_IN features -> XLMIMO_MLP_HIDDEN hidden layers of
 * XLMIMO_MLP_WIDTH units with SiLU, silu(z) = z / (1 + e^-z) -> XLMIMO_MLP_OUT
 * outputs (Re t, Im t).  Parameters: one FP32 buffer of XLMIMO_MLP_PARAMS
 * floats, layer by layer, each layer's W [in][out] (row-major) followed by
 * its bias [out].
 * Features of a pair (r the user's distance to the array centre, theta its
 * angle from broadside, atan2(y, x)):
 *   ((ln(r_i/lambda) - 7.5)/2, theta_i/(pi/3), (ln(r_j/lambda) - 7.5)/2,
 *    theta_j/(pi/3), (log2 N - 14)/4, (spacing/lambda - 1/2) * 4)
 * Pair rows: trial-major, then i, then j (i < j): B * K(K-1)/2 rows.
 * Numerics (training and inference alike): the first (6 -> 256) and last
 * (256 -> 2) layers in FP32; the three 256 x 256 layers multiply BF16-rounded
 * (round to nearest even) inputs by BF16-rounded weights with FP32
 * accumulation.  Gradients pass through the rounding unchanged.  Training
 * runs the three 256 x 256 layers on the tensor cores (forward, input and
 * weight gradients; the FP32 gradient enters as a BF16 hi/lo pair, within
 * 2^-16 of each FP32 product) and the other two on FP32 SIMT.  Inference
 * runs every layer but the last on the tensor cores (the first with a BF16
 * hi/lo split of features and weights, which keeps it to ~2^-16 of FP32) and
 * evaluates SiLU as z/2 (1 + tanh(z/2)) with the FP32 hardware tanh
 * approximation (relative error ~2^-11, below the BF16 rounding that follows). */
#define XLMIMO_MLP_IN 6
#define XLMIMO_MLP_WIDTH 256
#define XLMIMO_MLP_HIDDEN 4
#define XLMIMO_MLP_OUT 2
#define XLMIMO_MLP_PARAMS 199682
/* floats per row of the forward cache: pre-activation z and activation h of
 * every hidden layer, stored as [layer][z | h][M][256] */
#define XLMIMO_MLP_CACHE_PER_ROW (2 * XLMIMO_MLP_HIDDEN * XLMIMO_MLP_WIDTH)
/* bytes of the packed inference image written by xlmimo_mlp_pack */
#define XLMIMO_MLP_PACKED_BYTES 432384

/* Features (and optionally targets and weights) of every pair of every trial.
 * users [B][K][2], K >= 2.  feat [B*P][6] out, P = K(K-1)/2.  If gram (exact)
 * and gram_cf (closed form, xlmimo_corr_closed_form) are both non-NULL,
 * target [B*P][2] gets (Re, Im) of G_ij / G~_ij - F_ij, F the factor `base`
 * (xlmimo_aperture); if weight is non-NULL it gets
 * |G~_ij|^2 / (G~_ii G~_jj) (needs gram_cf).  Features are computed in FP32
 * from the FP64 positions, targets and weights in FP64; all outputs FP32. */
int xlmimo_pair_features(const xlmimo_array* arr, const double* users, int K, int B, int base, const double* gram,
                         const double* gram_cf, float* feat, float* target, float* weight, void* stream);

/* Forward pass over M rows: x [M][6] -> out [M][2].  cache is NULL or
 * [M * XLMIMO_MLP_CACHE_PER_ROW] floats (needed by xlmimo_mlp_backward).
 * Allocates 786,432 bytes of stream-ordered workspace (the packed weights of
 * the 256 x 256 layers), plus 2 * M * 256 floats when cache is NULL. */
int xlmimo_mlp_forward(const float* params, const float* x, int M, float* out, float* cache, void* stream);

/* Loss 0.5/M * sum_m w_m |out_m - target_m|^2 into *loss (device float) and
 * its gradient dout [M][2].  weight NULL means w = 1. */
int xlmimo_mlp_loss(const float* out, const float* target, const float* weight, int M, float* dout, float* loss,
                    void* stream);

/* Floats of device workspace xlmimo_mlp_backward and xlmimo_mlp_train_step
 * need for M rows (the buffer 16-byte aligned). */
int64_t xlmimo_mlp_work_floats(int M);

/* Backward pass: grad [XLMIMO_MLP_PARAMS] (overwritten) of the loss whose
 * output gradient is dout [M][2], from the forward cache of the same x. */
int xlmimo_mlp_backward(const float* params, const float* x, const float* cache, const float* dout, int M,
                        float* grad, float* work, void* stream);

/* One Adam step (Kingma and Ba) on params with moments m, v (all
 * [XLMIMO_MLP_PARAMS], updated in place): m = b1 m + (1-b1) g,
 * v = b2 v + (1-b2) g^2, p -= lr * (m/(1-b1^step)) / (sqrt(v/(1-b2^step)) + eps).
 * step >= 1. */
int xlmimo_mlp_adam(float* params, float* m, float* v, const float* grad, int64_t step, double lr, double beta1,
                    double beta2, double eps, void* stream);

/* Forward, loss, backward and Adam on one batch, in that order (out [M][2],
 * cache, work as above; loss may be NULL). */
int xlmimo_mlp_train_step(float* params, float* m, float* v, float* grad, int64_t step, double lr, const float* x,
                          const float* target, const float* weight, int M, float* out, float* cache, float* work,
                          float* loss, void* stream);

/* BF16 inference image of params (packed: XLMIMO_MLP_PACKED_BYTES, 16-byte
 * aligned) for xlmimo_surrogate_gram. */
int xlmimo_mlp_pack(const float* params, void* packed, void* stream);

/* Surrogate Gram [B][K][K]: the closed form of xlmimo_corr_closed_form with
 * every off-diagonal entry multiplied by F_ij + t_ij, F the factor `base`
 * (the one the network was trained with), t from the network in `packed`.
 * One fused tensor-core launch evaluates the network on all pairs.  A bounded
 * device-side wait that gives up leaves NaN in its pairs. */
int xlmimo_surrogate_gram(const xlmimo_array* arr, const double* users, int K, int B, int base, const void* packed,
                          double* gram, void* stream);

/* Measured throughput of one pipe of the device, for the roofline of the
 * channel generator (the paper has no counterpart).  Runs independent
 * dependency chains of one operation on every SM (8 blocks of 256 threads
 * per SM, 8 chains per thread) and times the best of three launches with
 * CUDA events on `stream`.  SYNCHRONOUS.  Pipes:
 *   XLMIMO_PIPE_SINCOS  alternating sin.approx / cos.approx (MUFU)
 *   XLMIMO_PIPE_RSQRT   rsqrt.approx (MUFU)
 *   XLMIMO_PIPE_FFMA    scalar FP32 FMA
 *   out : 2 doubles (host, written) {operations per second, best launch ms}
 * The caller samples the SM clock around the call if it needs it. */
typedef enum { XLMIMO_PIPE_SINCOS = 0, XLMIMO_PIPE_RSQRT = 1, XLMIMO_PIPE_FFMA = 2 } xlmimo_pipe;
int xlmimo_measure_pipe(int pipe, double* out, void* stream);

/* Message of the last error on this host thread ("" if none). */
const char* xlmimo_last_error(void);

/* Interface version, (major << 16) | minor. */
int xlmimo_version(void);

/* Releases what the library keeps between calls: the streams and events that
 * xlmimo_mc_step creates on first use on each device (work already enqueued
 * there completes first).  The library stays usable; the next call creates
 * them again.  Must not run concurrently with another library call.  The
 * scratch of xlmimo_channel_gram_noalloc is part of the library's module
 * and lives as long as the CUDA context.  Returns XLMIMO_OK, or
 * XLMIMO_ECUDA if a device could not be selected or synchronised. */
int xlmimo_shutdown(void);

#ifdef __cplusplus
}
#endif

#endif /* XLMIMO_H */
