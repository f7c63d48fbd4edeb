// xlmimo_mc_step: one Monte-Carlo step over a batch, pipelined over
// streams.  The receivers compute their sum rates themselves; the exact
// (matched, one shared-memory buffer) and the closed-form (modified ZF)
// receivers run as two launches on two library streams at once, so that the
// first one's FP64 factorisations and the second one's FP32 work share every
// SM (measured: two streams 7.29 ms per headline step, the two launches on one
// stream 7.31 ms, both receivers in one interleaved launch 7.37 ms).  The
// exact-Gram kernels (channel generation on the FP32 and MUFU pipes,
// contraction on the tensor cores) and the receivers (FP64 pipe) use disjoint
// execution units, so piece c's Gram on the caller's stream runs next to
// piece c-1's receivers on a library stream; events order each piece's
// receivers after its Gram and the caller's stream after everything.
#include <mutex>
#include <vector>

#include "common.cuh"

namespace xl {

int launch_stats_strided(const double* x, int B, int stride, double* out, cudaStream_t st);

constexpr int PIPE_MAX_CHUNKS = 64;

struct PipeState {
    cudaStream_t side = nullptr;
    cudaStream_t side2 = nullptr;  // the closed-form receivers
    cudaEvent_t gram_done[PIPE_MAX_CHUNKS] = {};
    cudaEvent_t cf_fork[PIPE_MAX_CHUNKS] = {}, cf_join[PIPE_MAX_CHUNKS] = {};
    cudaEvent_t inputs_ready = nullptr;
    cudaEvent_t side_done = nullptr;
    bool ready = false;
};

static std::mutex g_pipe_mu;
static std::vector<PipeState> g_pipe;

// Destroy what a PipeState holds (null handles are skipped) and reset it.
static void release_pipe(PipeState& p) {
    for (int i = 0; i < PIPE_MAX_CHUNKS; ++i) {
        if (p.gram_done[i]) cudaEventDestroy(p.gram_done[i]);
        if (p.cf_fork[i]) cudaEventDestroy(p.cf_fork[i]);
        if (p.cf_join[i]) cudaEventDestroy(p.cf_join[i]);
    }
    if (p.inputs_ready) cudaEventDestroy(p.inputs_ready);
    if (p.side_done) cudaEventDestroy(p.side_done);
    if (p.side) cudaStreamDestroy(p.side);
    if (p.side2) cudaStreamDestroy(p.side2);
    p = PipeState{};
}

static int pipe_state(PipeState** out) {
    int dev = 0;
    int rc = cuda_status(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc) return rc;
    if ((int)g_pipe.size() <= dev) g_pipe.resize(dev + 1);
    PipeState& p = g_pipe[dev];
    if (!p.ready) {
        // highest priority: the closed form launched on it during the Gram kernel
        // gets the leftover space on every SM instead of waiting for the Gram's
        // last wave
        int least = 0, greatest = 0;
        rc = cuda_status(cudaDeviceGetStreamPriorityRange(&least, &greatest), "stream priorities");
        if (!rc) rc = cuda_status(cudaStreamCreateWithPriority(&p.side, cudaStreamNonBlocking, greatest), "side stream");
        if (!rc) rc = cuda_status(cudaStreamCreateWithPriority(&p.side2, cudaStreamNonBlocking, greatest), "side stream");
        for (int i = 0; !rc && i < PIPE_MAX_CHUNKS; ++i) {
            rc = cuda_status(cudaEventCreateWithFlags(&p.gram_done[i], cudaEventDisableTiming), "pipeline event");
            if (!rc) rc = cuda_status(cudaEventCreateWithFlags(&p.cf_fork[i], cudaEventDisableTiming), "pipeline event");
            if (!rc) rc = cuda_status(cudaEventCreateWithFlags(&p.cf_join[i], cudaEventDisableTiming), "pipeline event");
        }
        if (!rc) rc = cuda_status(cudaEventCreateWithFlags(&p.side_done, cudaEventDisableTiming), "pipeline event");
        if (!rc) rc = cuda_status(cudaEventCreateWithFlags(&p.inputs_ready, cudaEventDisableTiming), "pipeline event");
        if (rc) {
            release_pipe(p);  // nothing half-made is kept; the next call starts afresh
            return rc;
        }
        p.ready = true;
    }
    *out = &p;
    return XLMIMO_OK;
}

static int launch_gram_prec(const Geom& g, const double* users, int K, int B, int prec, double* gram, cudaStream_t st,
                            bool leave_room) {
    switch (prec) {
        case XLMIMO_F64: return launch_gram_f64(g, users, K, B, gram, st);
        case XLMIMO_F32: return launch_gram_f32(g, users, K, B, gram, st);
        default: return launch_gram_tc(g, users, K, B, prec, gram, st, leave_room ? 2 : 0);
    }
}

static int check_job(const xlmimo_mc_batch* j) {
    if (!j) { set_error("job is NULL"); return XLMIMO_EINVAL; }
    if (j->K < 1 || j->K > XLMIMO_MAX_USERS || j->B < 0) { set_error("K must be in [1, 64] and B >= 0"); return XLMIMO_EINVAL; }
    if (j->prec < XLMIMO_F64 || j->prec > XLMIMO_F16X3) { set_error("unknown precision"); return XLMIMO_EINVAL; }
    if (j->scheme < XLMIMO_ZF || j->scheme > XLMIMO_ZF_DL) { set_error("unknown scheme"); return XLMIMO_EINVAL; }
    if (j->cf_scheme > XLMIMO_ZF_DL || j->cf_scheme < -1) { set_error("unknown closed-form scheme"); return XLMIMO_EINVAL; }
    if (j->power_mode != XLMIMO_POWER_ABS && j->power_mode != XLMIMO_POWER_RXSNR) { set_error("unknown power mode"); return XLMIMO_EINVAL; }
    if (j->chunks < 0 || j->chunks > PIPE_MAX_CHUNKS || j->reserved != 0) { set_error("chunks must be in [0, 64], reserved 0"); return XLMIMO_EINVAL; }
    if (!(j->t == 0.0 || (j->t > 0.0 && j->t < 1.0))) { set_error("t must be 0 or in (0, 1)"); return XLMIMO_EINVAL; }
    if (j->B == 0) return XLMIMO_OK;
    if (!j->users || !j->power || !j->noise || !j->gram || !j->sinr || !j->status || !j->rate) {
        set_error("users, power, noise, gram, sinr, status and rate must be non-NULL");
        return XLMIMO_EINVAL;
    }
    if (j->cf_scheme >= 0 && (!j->gram_cf || !j->sinr_cf || !j->status_cf || !j->rate_cf)) {
        set_error("the closed-form path needs gram_cf, sinr_cf, status_cf and rate_cf");
        return XLMIMO_EINVAL;
    }
    if (j->t > 0.0 && !j->sat) { set_error("sat must be non-NULL when t > 0"); return XLMIMO_EINVAL; }
    return XLMIMO_OK;
}

}  // namespace xl

using namespace xl;

extern "C" int xlmimo_mc_step(const xlmimo_mc_batch* j, void* stream) {
    clear_error();
    int rc = check_job(j);
    if (rc) return rc;
    Geom g;
    if ((rc = check_array(&j->arr, &g))) return rc;
    if (j->B == 0) return XLMIMO_OK;
    const int K = j->K, B = j->B;
    int C = j->chunks;
    // measured at 1e4 headline trials: one piece 7.27 ms, 2 / 4 pieces 7.32 / 7.54 ms (the Gram
    // kernel fills every SM, so a piece's receivers only take SMs as the next Gram's CTAs finish;
    // with the interleaved receivers of an earlier build: 9.33 / 9.41 / 9.64 ms, and 10.19 /
    // 10.47 ms when the Gram kernel left room for the receivers by running 2 CTAs/SM)
    if (C == 0) C = 1;
    if (C > B) C = B;
    cudaStream_t s0 = as_stream(stream);
    std::lock_guard<std::mutex> lk(g_pipe_mu);
    PipeState* ps = nullptr;
    if ((rc = pipe_state(&ps))) return rc;
    cudaStream_t s1 = ps->side;
    const size_t KK = (size_t)K * K;
    // the side stream starts once the caller's inputs are ready
    rc = cuda_status(cudaEventRecord(ps->inputs_ready, s0), "event record");
    if (!rc) rc = cuda_status(cudaStreamWaitEvent(s1, ps->inputs_ready, 0), "stream wait");
    for (int c = 0; c < C && !rc; ++c) {
        const int b0 = (int)((int64_t)B * c / C), b1 = (int)((int64_t)B * (c + 1) / C);
        const int nb = b1 - b0;
        if (nb <= 0) continue;
        const double* u = j->users + (size_t)b0 * K * 2;
        double* gm = j->gram + (size_t)b0 * KK * 2;
        double* gc = j->cf_scheme >= 0 ? j->gram_cf + (size_t)b0 * KK * 2 : nullptr;
        rc = launch_gram_prec(g, u, K, nb, j->prec, gm, s0, false);
        // the closed form and the saturation interval need only the positions:
        // they run on the side stream during the Gram kernel, in blocks small
        // enough to fit beside its CTAs
        if (!rc && gc) rc = launch_closed_form(g, u, K, nb, gc, s1, 64);
        if (!rc && j->t > 0.0) rc = launch_saturation(u, K, nb, j->t, g.spacing, j->sat + (size_t)b0 * 3, s1);
        if (!rc) rc = cuda_status(cudaEventRecord(ps->gram_done[c], s0), "event record");
        if (!rc) rc = cuda_status(cudaStreamWaitEvent(s1, ps->gram_done[c], 0), "stream wait");
        if (rc) break;
        const double* pw = j->power + (size_t)b0 * K;
        const double* nz = j->noise + b0;
        double* sinr = j->sinr + (size_t)b0 * K;
        double* cap = j->capacity ? j->capacity + b0 : nullptr;
        if (gc) {
            // the closed-form receivers on the second library stream, forked
            // after the Gram and the closed form and joined before the stats;
            // below the FP64 Gram the mismatched SINR takes the FP32
            // correction: its error stays far under the exact Gram's own
            const int cfs = j->cf_scheme | (j->prec != XLMIMO_F64 ? XLMIMO_MISMATCH_FP32 : 0);
            cudaStream_t s2 = ps->side2;
            rc = cuda_status(cudaEventRecord(ps->cf_fork[c], s1), "event record");
            if (!rc) rc = cuda_status(cudaStreamWaitEvent(s2, ps->cf_fork[c], 0), "stream wait");
            if (!rc)
                rc = launch_beamform(gc, gm, pw, nz, K, nb, cfs, j->power_mode, j->sinr_cf + (size_t)b0 * K,
                                     j->status_cf + b0, nullptr, s2, j->rate_cf + b0);
            if (!rc)
                rc = launch_beamform(gm, nullptr, pw, nz, K, nb, j->scheme, j->power_mode, sinr, j->status + b0, cap, s1,
                                     j->rate + b0);
            // joined even after an error once the fork was recorded, so that
            // nothing on the second stream outlives the step
            const int rj = cuda_status(cudaEventRecord(ps->cf_join[c], s2), "event record");
            const int rw = rj ? rj : cuda_status(cudaStreamWaitEvent(s1, ps->cf_join[c], 0), "stream wait");
            if (!rc) rc = rw;
        } else {
            rc = launch_beamform(gm, nullptr, pw, nz, K, nb, j->scheme, j->power_mode, sinr, j->status + b0, cap, s1,
                                 j->rate + b0);
        }
    }
    if (!rc && j->stats) rc = launch_stats_strided(j->rate, B, 1, j->stats, s1);
    if (!rc && j->stats_cf && j->cf_scheme >= 0) rc = launch_stats_strided(j->rate_cf, B, 1, j->stats_cf, s1);
    // the caller's stream waits for the side stream even after an error, so
    // nothing enqueued above can outlive the caller's view of the step
    int rc2 = cuda_status(cudaEventRecord(ps->side_done, s1), "event record");
    if (!rc2) rc2 = cuda_status(cudaStreamWaitEvent(s0, ps->side_done, 0), "stream wait");
    return rc ? rc : rc2;
}

// Release the pipeline's per-device stream and events (created by the first
// xlmimo_mc_step on a device); work already enqueued on the side stream
// completes first.  The next xlmimo_mc_step creates them again.
extern "C" int xlmimo_shutdown(void) {
    clear_error();
    std::lock_guard<std::mutex> lk(g_pipe_mu);
    int caller = -1, rc = XLMIMO_OK;
    for (int dev = 0; dev < (int)g_pipe.size(); ++dev) {
        PipeState& p = g_pipe[dev];
        if (!p.ready) continue;
        if (caller < 0 && (rc = cuda_status(cudaGetDevice(&caller), "cudaGetDevice"))) return rc;
        int r = cuda_status(cudaSetDevice(dev), "cudaSetDevice");
        if (!r) r = cuda_status(cudaStreamSynchronize(p.side), "side stream synchronize");
        if (!r) r = cuda_status(cudaStreamSynchronize(p.side2), "side stream synchronize");
        release_pipe(p);
        if (!rc) rc = r;
    }
    if (caller >= 0) {
        int r = cuda_status(cudaSetDevice(caller), "cudaSetDevice");
        if (!rc) rc = r;
    }
    return rc;
}
