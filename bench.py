"""Monte-Carlo beamforming throughput on GB300.

One step = the whole hot path over one batch of trials of the headline
workload (100 GHz ULA, N = 16384 elements, K = 32 users at r in [3, 30] m,
theta in [-60, 60] deg, free-space spherical-wave channel, MMSE at 10 dB
per-user received SNR with FP64 Cholesky, 10^4 trials):
  exact Gram (generated channel, no HBM channel matrix) -> MMSE SINR and
  capacity -> sum rate; closed-form Gram -> modified ZF judged on the exact
  channel -> sum rate; per-trial saturation interval.
Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2503_18118_gb300 import inputs  # noqa: E402

PATHS = {"f64": 0, "f32": 1, "bf16x3": 3}
KERNEL_OF_PATH = {"f64": "gram_f64_kernel", "f32": "gram_f32_kernel", "bf16x3": "gram_tc_kernel"}
SRC_OF_PATH = {"f64": "gram_simt.cu", "f32": "gram_simt.cu", "bf16x3": "gram_tc.cu"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--path", default="auto", choices=["auto", "f64", "f32", "bf16x3"])
    ap.add_argument("--trials", type=int, default=None)
    ap.add_argument("--chunks", type=int, default=0, help="pipeline pieces per step (0 = library default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-baseline", action="store_true")
    ap.add_argument("--source-hash", metavar="KERNEL", choices=sorted(PROFILE_SOURCES),
                    help="print the source hash a profile summary records, and exit")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the precision table, the ragged batch, the sweep and the surrogate")
    ap.add_argument("--only", choices=["ragged", "appendix_a", "sweep", "surrogate", "ura"],
                    help="run one extra section alone (no headline step) and print its JSON; for profiling")
    ap.add_argument("--ragged-count", type=int, default=1 << 14, help="instances of the ragged section")
    ap.add_argument("--no-ragged-tune", action="store_true", help="ragged section with the default tiling (no autotune)")
    ap.add_argument("--ref-seconds", type=float, default=90.0,
                    help="--impl reference: seconds of oracle work the warm-up and timed steps share")
    ap.add_argument("--surrogate-train-steps", type=int, default=None,
                    help="Adam steps of the surrogate section (default: the workload's 8000)")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------- oracle (CPU) -----
def oracle_pipeline(oracle, wl, users):
    """The same per-trial work as one GPU step, on the CPU oracle."""
    B = users.shape[0]
    G = oracle.gram(wl.model, wl.n_ant, wl.wavelength, wl.spacing, 1.0, users)
    s, _, cap = oracle.beamform(G, wl.power(B), wl.noise(B), oracle.MMSE, oracle.POWER_RXSNR, want_capacity=True)
    r, _ = oracle.sumrate(s)
    Gc = oracle.closed_form(wl.model, wl.n_ant, wl.wavelength, wl.spacing, 1.0, users)
    sm, _, _ = oracle.beamform(Gc, wl.power(B), wl.noise(B), oracle.ZF, oracle.POWER_RXSNR, gram_true=G)
    rm, _ = oracle.sumrate(sm)
    oracle.saturation(users, 0.9, wl.spacing)
    return r, cap, rm


def cpu_trials_per_s(oracle, wl, budget_s=12.0, max_trials=4096):
    """Oracle timed on a bounded sample: calibrate on 16 trials, then run a
    sample sized to about budget_s seconds."""
    users = wl.users(max_trials)
    t0 = time.perf_counter()
    oracle_pipeline(oracle, wl, users[:16])
    t16 = time.perf_counter() - t0
    n = int(min(max_trials, max(16, budget_s / max(t16 / 16, 1e-9))))
    t0 = time.perf_counter()
    oracle_pipeline(oracle, wl, users[:n])
    dt = time.perf_counter() - t0
    return n / dt, n, dt


def workload_config(wl):
    """The workload both arms report as `config`: what is computed, not how."""
    return {"workload": wl.name, "n_ant": wl.n_ant, "users": wl.k, "trials_per_step": wl.trials,
            "freq_ghz": wl.freq_hz / 1e9, "scheme": "mmse+modified_zf",
            "receivers": "mmse with its capacity on the exact Gram; modified zf from the closed form, judged on the "
                         "exact Gram; per-trial saturation interval",
            "l2": "the GPU arm flushes L2 between timed steps (256 MB write)"}


def reference_arm(args, wl):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    users = wl.users(4096)
    # each step is a bounded sample of the workload, sized from a calibration run
    t0 = time.perf_counter()
    oracle_pipeline(oracle, wl, users[:16])
    per = (time.perf_counter() - t0) / 16
    n = int(max(8, min(4096, args.ref_seconds / max(args.steps + args.warmup, 1) / max(per, 1e-9))))
    for _ in range(args.warmup):
        oracle_pipeline(oracle, wl, users[:n])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_pipeline(oracle, wl, users[:n])
    dt = time.perf_counter() - t0
    v = args.steps * n / dt
    cores = oracle.num_threads()
    line = {
        "impl": "reference", "metric": "mc_beamforming_trials_per_s", "value": v, "unit": "trials/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(wl),
        "sample_trials_per_step": n,
        "cpu_baseline": {"value": v, "unit": "trials/s", "cores": cores, "kind": "oracle",
                         "sample": f"{n} of the workload's {wl.trials} trials per step (the first {n} of its users), "
                                   f"{args.steps} steps; value = trials timed / time"},
        "e2e": {"value": v, "unit": "trials/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ GPU arm -------
# sources whose bytes the committed ncu summary of each kernel was taken on
PROFILE_SOURCES = {
    "gram_tc_kernel": ["gram_tc.cu", "gram_engine.cuh", "gen_tc.cuh", "tc_common.cuh", "chan_gen.cuh", "common.cuh"],
    "mlp_infer_tc_kernel": ["mlp_tc.cu", "mlp_common.cuh", "tc_common.cuh", "common.cuh"],
    "gram_hilo_kernel": ["bounds.cu", "gram_hilo_tc.cuh", "gen_tc.cuh", "tc_common.cuh", "chan_gen.cuh", "common.cuh"],
    "gram_tc_packed_kernel": ["batched.cu", "gram_engine.cuh", "gen_tc.cuh", "tc_common.cuh", "chan_gen.cuh",
                              "common.cuh"],
}
PROFILE_OF_KERNEL = {"gram_tc_kernel": "gram_tc_kernel_headline.md",
                     "mlp_infer_tc_kernel": "mlp_infer_tc_kernel_surrogate.md",
                     "gram_tc_packed_kernel": "gram_tc_packed_kernel_ragged.md",
                     "gram_hilo_kernel": "bounds_appendix_a.md"}


def source_hash(kernel):
    """sha256 chained over the kernel's source files (PROFILE_SOURCES order)."""
    h = ""
    for f in PROFILE_SOURCES[kernel]:
        d = hashlib.sha256(open(os.path.join(ROOT, "paper_2503_18118_gb300", "csrc", f), "rb").read()).hexdigest()
        h = hashlib.sha256((h + d).encode()).hexdigest()
    return h


def traffic_from_profile(kernel, units=None):
    """DRAM bytes per full launch recorded by the committed ncu summary of the
    kernel, valid only while the kernel's sources are unchanged.  A summary
    taken on a smaller case records its bytes per unit (dram_bytes_per_unit);
    the full launch's is that times `units`.  A kernel without a committed
    summary has no traffic figure."""
    if kernel not in PROFILE_OF_KERNEL:
        return None
    prof = os.path.join(ROOT, "profiles", PROFILE_OF_KERNEL[kernel])
    if not os.path.exists(prof):
        return None
    text = open(prof).read()
    m = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
    if not m or m.group(1) != source_hash(kernel):
        return None
    t = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+-]+)", text)
    if t:
        return float(t.group(1))
    u = re.search(r"dram_bytes_per_unit:\s*([0-9.eE+-]+)", text)
    return float(u.group(1)) * units if (u and units) else None


def ragged_bench(xl, torch, mufu_peak, count=1 << 14, tune=True):
    """Ragged batch of 2^14 instances: N = round(2^U[10,17]), K ~ U{2..64},
    ZF or MMSE with probability 1/2, SNR ~ U[0, 30] dB, users as the headline
    geometry; autotuned plan, run captured in a CUDA graph and replayed."""
    n, k, scheme, snr_db = inputs.ragged_instances(4, count)
    lam = inputs.wavelength(100e9)
    users = inputs.users_polar(4, 1, int(k.sum()), (3.0, 30.0))[0]
    snr = np.repeat(inputs.db_to_lin(snr_db), k)
    U = torch.from_numpy(users).cuda()
    P = torch.from_numpy(np.ascontiguousarray(snr)).cuda()
    t0 = time.perf_counter()
    plan = xl.BatchPlan(xl.array(1, lam), n, k, scheme, np.ones(count), prec=xl.BF16X3, tune_users=U if tune else None)
    plan_s = time.perf_counter() - t0
    out = dict(gram=torch.empty(plan.gram_total, dtype=torch.complex128, device="cuda"),
               sinr=torch.empty(plan.users_total, dtype=torch.float64, device="cuda"),
               status=torch.empty(count, dtype=torch.int32, device="cuda"),
               rate=torch.empty(count, dtype=torch.float64, device="cuda"))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.run(U, P, xl.POWER_RXSNR, **out, stream=s)  # warm
        s.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s):
            plan.run(U, P, xl.POWER_RXSNR, **out, stream=s)
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    e0.record()
    for _ in range(reps):
        graph.replay()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    # the Gram launches alone (same plan, same stream), for the roofline and
    # the split of the batch time between the Gram and the receivers
    with torch.cuda.stream(s):
        for _ in range(2):
            plan.run_gram(U, out["gram"], stream=s)
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(s)
        for _ in range(reps):
            plan.run_gram(U, out["gram"], stream=s)
        g1.record(s)
    torch.cuda.synchronize()
    gram_ms = g0.elapsed_time(g1) / reps
    info = plan.info()
    plan.close()
    entries = float((n * k).sum())
    achieved = 3.0 * entries / (gram_ms / 1e3) / 1e12
    return {"workload": "2^14 instances, N=2^U[10,17], K~U{2..64}, ZF/MMSE, SNR~U[0,30] dB, 100 GHz",
            "instances_per_s": count / (ms / 1e3), "ms_per_batch": ms, "gram_ms": gram_ms,
            "receivers_and_rates_ms": ms - gram_ms, "channel_entries": int(entries),
            "plan": info, "plan_seconds": plan_s, "cuda_graph": True, "gram": "bf16x3",
            "roofline": {"bound": "alu", "achieved": achieved, "peak": mufu_peak, "unit": "Tops/s (MUFU)",
                         "frac": achieved / mufu_peak, "kernel": "gram_tc_packed_kernel (both tilings)",
                         "traffic": traffic_from_profile("gram_tc_packed_kernel", entries),
                         "kernel_ms": gram_ms,
                         "algorithmic": "3 transcendental ops (rsqrt, sin, cos) x sum of N K channel entries",
                         "peak_source": "measured sin/cos MUFU throughput (xlmimo_measure_pipe), of measured"}}


def sweep_bench(xl, torch):
    """Capacity-saturation sweep (Secs. IV-C, V-C): 28 GHz, K = 8 users at r in
    [5, 50] m, theta in [-60, 60] deg, N = 2^6 .. 2^16, the same 1000 trials at
    every N, exact and closed-form Grams, ZF / MMSE / capacity at 0, 10 and
    20 dB with N-independent power (reference user at 27.5 m), FP64 and FP32
    exact paths; the saturation point from the per-trial intervals and from
    the analytic ergodic formula for this polar distribution."""
    wl = inputs.SWEEP
    ex = wl.extra
    U = torch.from_numpy(wl.users()).cuda()
    out = {"workload": f"{wl.name}: N=2^6..2^16, K=8, 1000 trials, 28 GHz, SNR 0/10/20 dB, t={ex['t']}",
           "n_list": ex["n_list"]}
    for name, prec in (("f64", xl.F64), ("f32", xl.F32)):
        xl.xlmimo_capacity_sweep(U[:16].contiguous(), ex["n_list"][:2], ex["snr_db"], wl.wavelength, prec=prec,
                                 t=ex["t"], ref_x=27.5)  # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = xl.xlmimo_capacity_sweep(U, ex["n_list"], ex["snr_db"], wl.wavelength, prec=prec, t=ex["t"], ref_x=27.5)
        dt = time.perf_counter() - t0
        out[name] = {"seconds": dt, "trials_per_s": len(ex["n_list"]) * wl.trials / dt,
                     "capacity_10db": [float(v) for v in r["capacity"][:, 1]],
                     "zf_rate_10db": {"exact": [float(v) for v in r["rate"][:, 0, 0, 1]],
                                      "closed_form": [float(v) for v in r["rate"][:, 1, 0, 1]]},
                     "mmse_rate_10db": [float(v) for v in r["rate"][:, 0, 1, 1]],
                     "closed_form_gram_err": [float(v) for v in r["gram_err"]],
                     "n_sat_trial_mean": float(r["sat_mean"][2])}
    ana = xl.xlmimo_saturation_analytic(xl.DIST_POLAR, 5.0, 50.0, np.deg2rad(-60.0), np.deg2rad(60.0), wl.k, ex["t"],
                                        wl.spacing)
    cap = np.array(out["f64"]["capacity_10db"])
    frac = cap / cap[-1]
    first = [int(ex["n_list"][int(np.argmax(frac >= q))]) for q in (0.9, 0.99)]
    out["saturation"] = {"analytic_n_sat": int(ana[3]), "analytic_y_up_m": float(ana[0]),
                         "analytic_near_integer": bool(ana[4]), "analytic_other_candidate": int(ana[5]),
                         "capacity_reaches_90pct_at_n": first[0], "capacity_reaches_99pct_at_n": first[1]}
    return out


def appendix_a_bench(xl, torch, max_mhz, peaks=None):
    """Appendix A / Fig. 5: the negative empirical expectation -E_K[log2 lambda^R]
    = -(1/K) log2 det R and the capacity bounds at 0 dB receive SNR, for K from
    10 to 1000 users in the Sec. V-A rectangle (x in [1, 10] m, y in [-7.5, 7.5] m,
    100 GHz, PNUSW), N = 40000 elements (beyond the K = 1000 saturation count),
    8 trials per K; the paper reports 0.064 at K = 1000."""
    lam = inputs.wavelength(100e9)
    N, B = 40000, 8
    arr = xl.array(N, lam, model=0)
    ks = [10, 50, 100, 200, 400, 600, 800, 1000]
    out = {"workload": "Sec. V-A rectangle, 100 GHz, PNUSW, N=40000, 8 trials per K, receive SNR 0 dB",
           "k": ks, "neg_expectation_mean": [], "neg_expectation_std": [], "capacity_mean": [],
           "log2_lower_mean": [], "log2_upper": [], "ms": [], "trials_per_s": []}
    U0 = torch.from_numpy(inputs.users_rect(21, 1, 10, (1.0, 10.0), (-7.5, 7.5))).cuda()
    xl.xlmimo_capacity_bounds(arr, U0, 1.0)  # warm
    flops = 0.0
    for K in ks:
        U = torch.from_numpy(inputs.users_rect(20 + K, B, K, (1.0, 10.0), (-7.5, 7.5))).cuda()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        o = xl.xlmimo_capacity_bounds(arr, U, 1.0)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        o = o.cpu().numpy()
        e = -o[:, 0] / K
        out["neg_expectation_mean"].append(float(e.mean()))
        out["neg_expectation_std"].append(float(e.std()))
        out["capacity_mean"].append(float(o[:, 1].mean()))
        out["log2_lower_mean"].append(float(o[:, 3].mean()))
        out["log2_upper"].append(float(o[0, 2]))
        out["ms"].append(ms)
        out["trials_per_s"].append(B / (ms / 1e3))
        if K == ks[-1]:
            flops = 8.0 * N * K * (K + 1) / 2 * B  # Gram complex MACs of the Hermitian half
            t_last = ms
            _, phases = xl.xlmimo_capacity_bounds_timed(arr, U, 1.0)  # the same call, its phases timed
    Kp = (ks[-1] + 63) // 64 * 64
    chol = 2 * B * 4.0 / 3.0 * Kp ** 3  # complex Cholesky of R and I + aR per trial, order Kp
    out["paper_value_at_k1000"] = 0.064
    names = ("channels", "gram_tensor_cores", "correlation", "cholesky", "bounds")
    out["phases_ms_k1000"] = dict(zip(names, phases))
    # the tensor-core Gram, timed on its own by the call's phase events: the
    # method's Gram work against the BF16 peak divided by the three products
    # of the hi/lo split (each FP32-class product costs three BF16 products)
    peaks = peaks or {}
    bf16 = float(peaks.get("bf16_tflops", 1935.2))
    t_gram = phases[1]
    issued = 3 * 2 * 128 * 128 * float(N) * (2 * Kp // 128) * (2 * Kp // 128 + 1) / 2 * B
    out["roofline"] = {"bound": "tensor", "kernel": "gram_hilo_kernel", "kernel_ms": t_gram,
                       "achieved": flops / (t_gram / 1e3) / 1e12, "peak": bf16 / 3.0, "unit": "TFLOP/s",
                       "frac": flops / (t_gram / 1e3) / 1e12 / (bf16 / 3.0),
                       "peak_source": "measured BF16 (MEASURED_PEAKS.json bf16_tflops, of measured) / 3: the "
                                      "three-product BF16 split",
                       "algorithmic": "8 flop x N K(K+1)/2 complex MACs per trial (Gram of K = 1000, N = 40000)",
                       "issued_bf16_tflops": issued / (t_gram / 1e3) / 1e12,
                       "traffic": traffic_from_profile("gram_hilo_kernel"),
                       "cholesky": {"ms": phases[3], "share_of_call": phases[3] / sum(phases),
                                    "fp64_class_tflops": chol / (phases[3] / 1e3) / 1e12,
                                    "how": "diagonal blocks FP64, panels and trailing updates double-float"}}
    return out


def ura_bench(xl, torch):
    """Uniform rectangular arrays (the planar-array extension of the footnote
    of Sec. II): the headline's users (100 GHz, K = 32, r in [3, 30] m,
    |theta| <= 60 deg, 10^4 trials, free-space spherical wave) on URAs of 16384
    elements, Gram time at BF16x3 and FP32 beside the ULA of the same element
    count, and accuracy on 64 trials against the FP64 URA path (normwise Gram
    error; MMSE sum rate at 10 dB)."""
    wl = inputs.HEADLINE
    U = torch.from_numpy(wl.users()).cuda()
    B, K = U.shape[0], U.shape[1]
    G = torch.empty((B, K, K), dtype=torch.complex128, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    snr = torch.from_numpy(wl.power(64)).cuda()
    noise = torch.from_numpy(wl.noise(64)).cuda()

    def timed(fn, reps=3, warm=1):
        for _ in range(warm):
            fn()
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    def rate(Gs):
        s, _, _ = xl.xlmimo_beamform(Gs, snr, noise, xl.MMSE, xl.POWER_RXSNR)
        return torch.log2(1 + s).sum(1).cpu().numpy()

    out = {"workload": f"{wl.name} users on 16384-element URAs (rows x columns), users in the array's horizontal plane",
           "ula_bf16x3_ms": timed(lambda: xl.xlmimo_channel_gram(xl.array(wl.n_ant, wl.wavelength, model=wl.model),
                                                                   U, xl.BF16X3, G)),
           "shapes": {}}
    for rows, cols in ((128, 128), (16, 1024)):
        arr = xl.array(cols, wl.wavelength, model=wl.model)
        r = {}
        for name, pp in (("bf16x3", xl.BF16X3), ("f32", xl.F32)):
            ms = timed(lambda: xl.xlmimo_channel_gram_ura(arr, rows, U, pp, G))
            r[name] = {"ms": ms, "trials_per_s": B / (ms / 1e3),
                       "entries_per_s": float(rows) * cols * K * B / (ms / 1e3)}
        U64 = U[:64].contiguous()
        g64 = xl.xlmimo_channel_gram_ura(arr, rows, U64, xl.F64)
        r64 = rate(g64)
        d = torch.sqrt(torch.diagonal(g64, dim1=1, dim2=2).real)
        for name, pp in (("bf16x3", xl.BF16X3), ("f32", xl.F32)):
            gx = xl.xlmimo_channel_gram_ura(arr, rows, U64, pp)
            r[name]["gram_normwise_err"] = float(((gx - g64).abs() / (d[:, :, None] * d[:, None, :])).max())
            r[name]["sumrate_rel_err"] = float(np.max(np.abs(rate(gx) - r64) / r64))
        out["shapes"][f"{rows}x{cols}"] = r
    del G, flush
    return out


def surrogate_bench(xl, torch, peaks, train_steps=None):
    """Learned correlation surrogate: labels from the exact kernel, training on
    the GPU, then the fused tensor-core inference timed at 100 GHz, N = 2^18,
    K = 64, 10^4 trials, and judged against the exact Gram and the closed form
    on modified-ZF sum rate."""
    from paper_2503_18118_gb300 import surrogate
    wl = inputs.SURROGATE
    ex = wl.extra
    K = wl.k
    trials = int(np.ceil(ex["train_pairs"] / (K * (K - 1) // 2)))
    n, freq, users = inputs.surrogate_trials(ex["train_seed"], trials, K, n_log2=ex["n_log2"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    feat, target, _ = surrogate.label_pairs(n, freq, users, base=ex["base"])
    torch.cuda.synchronize()
    label_s = time.perf_counter() - t0
    params = torch.from_numpy(inputs.mlp_init_params(ex["train_seed"])).cuda()
    tr = surrogate.Trainer(params, batch=ex["batch"], lr=ex["lr"], seed=ex["train_seed"])
    t0 = time.perf_counter()
    steps = train_steps or ex["steps"]
    log = tr.fit(feat, target, steps=steps, log_every=max(1, steps // 4))
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    del feat, target
    packed = xl.xlmimo_mlp_pack(params)

    arr = xl.array(wl.n_ant, wl.wavelength)
    B = wl.trials
    U = torch.from_numpy(wl.users()).cuda()
    G = torch.empty((B, K, K), dtype=torch.complex128, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def timed(fn, reps=5, warm=3):
        for _ in range(warm):
            fn()
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    t_cf = timed(lambda: xl.xlmimo_corr_closed_form(arr, U, G))
    t_fr = timed(lambda: xl.xlmimo_corr_closed_form_aperture(arr, U, xl.APERTURE_FRESNEL, G))
    t_sur = timed(lambda: xl.xlmimo_surrogate_gram(arr, U, packed, G, base=ex["base"]))
    t_exact = timed(lambda: xl.xlmimo_channel_gram(arr, U, xl.BF16X3, G), reps=3, warm=1)
    # the surrogate Gram is the base closed form (with the Fresnel factor when
    # the network corrects that base) followed by the network kernel
    t_base = t_fr if ex["base"] == xl.APERTURE_FRESNEL else t_cf
    t_mlp = t_sur - t_base
    rows = B * K * (K - 1) // 2
    flop_row = 2.0 * (6 * 256 + 3 * 256 * 256 + 256 * 2)
    achieved = rows * flop_row / (t_mlp / 1e3) / 1e12
    peak = float(peaks.get("bf16_tflops", 1935.2))
    del G
    # accuracy on the first 256 trials of the same workload, judged on the
    # FP64 exact Gram (parity 1e-12 against the oracle)
    res = surrogate.compare(arr, U[:256].contiguous(), packed, prec=xl.F64, base=ex["base"])
    re = res["rate_exact"]
    rows = ("cf", "mask", "fresnel", "sur")
    names = {"cf": "closed_form", "mask": "closed_form_aperture_mask", "fresnel": "closed_form_aperture_fresnel",
             "sur": "surrogate"}
    e_rate = {names[k]: float(np.mean(np.abs(res["rate_" + k] - re) / re)) for k in rows}
    e_gram = {names[k]: float(np.mean(res["gram_err_" + k])) for k in rows}
    return {
        "workload": f"{wl.name}: 100 GHz, N=2^18, K=64, 10^4 trials, r in [3,30] m",
        "training": {"pairs": int(n.size * K * (K - 1) // 2), "label_s": label_s, "steps": steps,
                     "batch": ex["batch"], "train_s": train_s, "loss": [float(l) for _, l in log],
                     "labels": "exact Gram (bf16x3), N log-uniform [2^10, 2^18], 28/100 GHz"},
        "base": "closed form x finite-aperture Fresnel factor" if ex["base"] == 2 else ex["base"],
        "gram_ms": {"exact_bf16x3": t_exact, "closed_form": t_cf, "closed_form_aperture_fresnel": t_fr,
                    "surrogate": t_sur},
        "trials_per_s": {"exact_bf16x3": B / (t_exact / 1e3), "closed_form": B / (t_cf / 1e3),
                         "closed_form_aperture_fresnel": B / (t_fr / 1e3), "surrogate": B / (t_sur / 1e3)},
        "sumrate_rel_err": dict(e_rate, trials=int(re.size), judge="exact Gram in FP64",
                                receiver="modified ZF at 10 dB judged on the exact channel (trial mean)"),
        "gram_rms_err": e_gram,
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": traffic_from_profile("mlp_infer_tc_kernel"),
                     "kernel": "mlp_infer_tc_kernel", "kernel_ms": t_mlp,
                     "kernel_ms_how": "surrogate Gram time minus its base closed form's time (both CUDA events)",
                     "algorithmic": "2 x (6x256 + 3x256^2 + 256x2) flop per pair x B K(K-1)/2 pairs",
                     "peak_source": "MEASURED_PEAKS.json bf16_tflops (of measured)"},
    }


def main():
    args = parse()
    if args.source_hash:
        print(source_hash(args.source_hash))
        return
    wl = inputs.HEADLINE
    if args.trials:
        wl.trials = args.trials
    if args.impl == "reference":
        reference_arm(args, wl)
        return

    import torch
    import torch.distributed as dist
    from paper_2503_18118_gb300 import mc
    from paper_2503_18118_gb300 import xlmimo as xl

    if args.only:
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        xl.lib()
        peaks = {}
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        mufu = xl.xlmimo_measure_pipe(xl.PIPE_SINCOS)[0] / 1e12
        run = {"ragged": lambda: ragged_bench(xl, torch, mufu, args.ragged_count, not args.no_ragged_tune),
               "appendix_a": lambda: appendix_a_bench(xl, torch, float(peaks.get("sm_max_mhz", 2070.0)), peaks),
               "sweep": lambda: sweep_bench(xl, torch),
               "surrogate": lambda: surrogate_bench(xl, torch, peaks, args.surrogate_train_steps),
               "ura": lambda: ura_bench(xl, torch)}[args.only]
        print(json.dumps({"section": args.only, "result": run()}), flush=True)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    path = args.path
    if path == "auto":
        path = "bf16x3"
    prec = PATHS[path]

    B, K, N = wl.trials, wl.k, wl.n_ant
    # weak scaling: rank r takes its own block of trials (different seed stream)
    users_h = inputs.users_polar(mc.rank_seed(wl.seed, rank), B, K, wl.r_range, wl.theta_deg)
    arr = xl.array(N, wl.wavelength, wl.spacing, 1.0, wl.model)
    stream = torch.cuda.current_stream()
    U = torch.from_numpy(users_h).cuda()
    snr = torch.from_numpy(wl.power()).cuda()
    noise = torch.from_numpy(wl.noise()).cuda()
    G = torch.empty((B, K, K), dtype=torch.complex128, device="cuda")
    flush = torch.empty((64 << 20,), dtype=torch.float32, device="cuda")  # 256 MB > L2

    out = xl.McBuffers(B, K)

    def step(gram_prec, users=None):
        """The whole path over the batch through the pipelined C entry point."""
        xl.xlmimo_mc_step(arr, U if users is None else users, snr, noise, out, prec=gram_prec, scheme=xl.MMSE,
                          cf_scheme=xl.ZF, power_mode=xl.POWER_RXSNR, t=0.9, chunks=args.chunks)

    def gram_only(gram_prec, ev):
        ev[0].record(stream)
        xl.xlmimo_channel_gram(arr, U, gram_prec, G)
        ev[1].record(stream)

    # per pipeline piece: the Gram, the closed form, the saturation interval and the two receivers (each
    # computes its trials' sum rates); per step: the two batch statistics.  (A Gram split into element
    # chunks adds a reduction launch; at this batch size every trial is one chunk.)
    pieces = args.chunks if args.chunks else 1
    launches_per_step = 5 * pieces + 2

    def timed(gram_prec, steps, warmup, sample_clocks=False):
        for _ in range(warmup):
            step(gram_prec)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(local) if sample_clocks else None
        if sampler:
            sampler.start()
            time.sleep(0.3)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush.zero_()
            evs[i][0].record(stream)
            step(gram_prec)
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clocks = sampler.stop() if sampler else None
        total_ms = sum(e[0].elapsed_time(e[1]) for e in evs)
        # the dominant kernel alone, same launch and stream, right after the timed steps
        gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush.zero_()
            gram_only(gram_prec, gev[i])
        torch.cuda.synchronize()
        gram_ms = sum(e[0].elapsed_time(e[1]) for e in gev) / steps
        return mc.max_over_ranks(total_ms, dist if world > 1 else None, "cuda"), gram_ms, clocks

    total_ms, gram_ms, clocks = timed(prec, args.steps, args.warmup, sample_clocks=(rank == 0))
    mufu_peak = xl.xlmimo_measure_pipe(xl.PIPE_SINCOS)[0] / 1e12  # Tops/s, measured on this GPU now
    ms_per_step = total_ms / args.steps
    value = mc.throughput(world, B, args.steps, total_ms)

    # plain FP64 GPU path (the metric's baseline), same pipeline, fewer steps
    fp64 = None
    if not args.no_fp64_baseline and path != "f64":
        t64, g64, _ = timed(PATHS["f64"], 2, 1)
        fp64 = {"trials_per_s": world * B * 2 / (t64 / 1e3), "gram_ms": g64, "ms_per_step": t64 / 2}

    # end to end through the C ABI from pinned host buffers: every step's inputs H2D and its result
    # D2H inside the timed region.  The inputs are double-buffered: step i + 1's copy runs on a copy
    # stream while step i computes (it waits until step i - 1 has finished with that buffer), the
    # way a caller feeds consecutive batches through the public API.
    users_pin = torch.from_numpy(users_h).pin_memory()
    rate_pin = torch.empty((B,), dtype=torch.float64).pin_memory()
    stats_pin = torch.empty((3,), dtype=torch.float64).pin_memory()
    copy_stream = torch.cuda.Stream()
    U_buf = (U, torch.empty_like(U))

    def e2e_steps(n):
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        freed = [torch.cuda.Event(), torch.cuda.Event()]
        start = torch.cuda.Event()
        start.record(stream)
        copy_stream.wait_event(start)  # no copy begins before the caller's timing starts
        U_buf[0].copy_(users_pin, non_blocking=True)  # the first step's inputs: nothing to overlap yet
        for i in range(n):
            cur, nxt = i % 2, (i + 1) % 2
            if i > 0:
                stream.wait_event(copied[cur])
            if i + 1 < n:
                with torch.cuda.stream(copy_stream):
                    if i > 0:
                        copy_stream.wait_event(freed[nxt])
                    U_buf[nxt].copy_(users_pin, non_blocking=True)
                    copied[nxt].record(copy_stream)
            step(prec, U_buf[cur])
            freed[cur].record(stream)
            rate_pin.copy_(out.rate, non_blocking=True)
            stats_pin.copy_(out.stats, non_blocking=True)

    e2e_steps(2)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps_n = max(1, min(args.steps, 5))
    e0.record(stream)
    e2e_steps(e2e_steps_n)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps_n
    e2e_value = mc.throughput(world, B, 1, mc.max_over_ranks(e2e_ms, dist if world > 1 else None, "cuda"))

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    # accuracy on sampled trials against the oracle (outside the timed region)
    import oracle
    oracle.build()
    idx = np.unique(np.linspace(0, B - 1, 64).astype(int))  # 64 trials spread over the batch
    step(prec)
    torch.cuda.synchronize()
    r_ref, _, rc_ref = oracle_pipeline(oracle, wl, users_h[idx])
    r_gpu = out.rate.cpu().numpy()[idx]
    sumrate_rel_err = float(np.max(np.abs(r_gpu - r_ref) / np.abs(r_ref)))
    rc_gpu = out.rate_cf.cpu().numpy()[idx]
    sumrate_rel_err_cf = float(np.max(np.abs(rc_gpu - rc_ref) / np.abs(rc_ref)))

    # precision study on the same workload: every Gram arithmetic, same step,
    # sum-rate error on the sampled trials against the oracle
    paths = None
    ragged = None
    sur = None
    sweep = None
    app_a = None
    ura = None
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    pipes = {"sincos_tops": mufu_peak, "rsqrt_tops": xl.xlmimo_measure_pipe(xl.PIPE_RSQRT)[0] / 1e12,
             "ffma_tflops": 2.0 * xl.xlmimo_measure_pipe(xl.PIPE_FFMA)[0] / 1e12,
             "how": "xlmimo_measure_pipe: independent dependency chains on every SM, best of 3 launches, CUDA events"}
    if not args.no_extras and world == 1:
        paths = {}
        for name in ("f64", "f32", "bf16", "bf16x3", "f16x3"):
            pp = {"f64": 0, "f32": 1, "bf16": 2, "bf16x3": 3, "f16x3": 4}[name]
            nsteps = 1 if name == "f64" else 3
            t_ms, _, _ = timed(pp, nsteps, 1)
            step(pp)
            torch.cuda.synchronize()
            rg = out.rate.cpu().numpy()[idx]
            paths[name] = {"trials_per_s": world * B * nsteps / (t_ms / 1e3),
                           "sumrate_rel_err": float(np.max(np.abs(rg - r_ref) / np.abs(r_ref)))}
        ragged = ragged_bench(xl, torch, mufu_peak)
        sweep = sweep_bench(xl, torch)
        sur = surrogate_bench(xl, torch, peaks)
        app_a = appendix_a_bench(xl, torch, float(peaks.get("sm_max_mhz", 2070.0)), peaks)
        ura = ura_bench(xl, torch)

    # peaks from unit counts and the maximum SM clock (per SM per clock:
    # 128 FP32 FMA lanes, 16 MUFU transcendental units, 2 FP64 FMA lanes)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    clk = max_mhz * 1e6
    entries = float(N) * K * B  # channel entries generated per launch
    gram_flops = 8.0 * N * K * (K + 1) / 2 * B  # complex MACs of the Hermitian half, 8 flop each
    if path == "bf16x3":
        # generation-bound.  Algorithmic count per entry: one reciprocal square
        # root (distance, amplitude) and one sine and one cosine.  The kernel
        # itself issues the sine and cosine per entry and a reciprocal square
        # root and a reciprocal per 8-element slice (the slice expansion).
        achieved = 3.0 * entries / (gram_ms / 1e3) / 1e12
        kernel_mufu = 2.0 + 2.0 / 8.0
        smem_per_entry = 20.0 if K <= 32 else 24.0  # stage writes + MMA operand reads, bytes
        roof = {"bound": "alu", "achieved": achieved, "peak": mufu_peak, "unit": "Tops/s (MUFU)",
                "frac": achieved / mufu_peak, "traffic": traffic_from_profile(KERNEL_OF_PATH[path]),
                "kernel": KERNEL_OF_PATH[path], "kernel_ms": gram_ms,
                "peak_source": "measured: sin.approx / cos.approx chains on every SM (xlmimo_measure_pipe), of measured; "
                               f"unit counts x max clock would be {sms * 16 * clk / 1e12:.3f}",
                "algorithmic": "3 transcendental ops (rsqrt, sin, cos) x N K channel entries per launch",
                "kernel_mufu_ops_per_entry": kernel_mufu,
                "mufu_busy_frac": kernel_mufu * entries / (gram_ms / 1e3) / 1e12 / mufu_peak,
                "smem_bytes_per_entry": smem_per_entry,
                "smem_frac": smem_per_entry * entries / (gram_ms / 1e3) / (sms * 128.0 * clk),
                # issued MMA work: K <= 32, M = 128, N = 64 per element; K <= 64, two 128 x 128
                "tensor_tflops": (2.0 * 128 * 64 if K <= 32 else 2 * 2.0 * 128 * 128) * N * B / (gram_ms / 1e3) / 1e12,
                "tensor_peak_tflops": float(peaks.get("bf16_tflops", 1935.2))}
    elif path == "f64":
        achieved = gram_flops / (gram_ms / 1e3) / 1e12
        peak_v = sms * 2 * 2 * clk / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak_v, "unit": "TFLOP/s", "frac": achieved / peak_v,
                "traffic": traffic_from_profile(KERNEL_OF_PATH[path]), "kernel": KERNEL_OF_PATH[path], "kernel_ms": gram_ms,
                "peak_source": f"FP64 FMA: {sms} SMs x 2 lanes x 2 flop x {max_mhz:.0f} MHz",
                "algorithmic": "8 flop x N K (K+1)/2 complex MACs per trial x trials per launch"}
    else:
        achieved = gram_flops / (gram_ms / 1e3) / 1e12
        peak_v = sms * 128 * 2 * clk / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak_v, "unit": "TFLOP/s", "frac": achieved / peak_v,
                "traffic": traffic_from_profile(KERNEL_OF_PATH[path]), "kernel": KERNEL_OF_PATH[path], "kernel_ms": gram_ms,
                "peak_source": f"FP32 FMA: {sms} SMs x 128 lanes x 2 flop x {max_mhz:.0f} MHz",
                "algorithmic": "8 flop x N K (K+1)/2 complex MACs per trial x trials per launch"}

    cpu = None
    if not args.no_cpu_baseline:
        v, n, dt = cpu_trials_per_s(oracle, wl)
        cpu = {"value": v, "unit": "trials/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"{n} trials of the workload ({dt:.1f} s), OpenMP over trials"}

    line = {
        "metric": "mc_beamforming_trials_per_s", "value": value, "unit": "trials/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": path, "data": "synthetic",
        "config": workload_config(wl),
        "gram_path": path,
        "solve": "mmse: f64 cholesky; modified zf: double-float cholesky, fp32 correction M(G-Gc)",
        "sumrate_rel_err": sumrate_rel_err,
        "sumrate_rel_err_modified_zf": sumrate_rel_err_cf,
        "fp64_baseline": fp64,
        "precisions": paths,
        "ragged": ragged,
        "sweep": sweep,
        "surrogate": sur,
        "appendix_a": app_a,
        "ura": ura,
        "speedup_vs_fp64_gpu": (value / fp64["trials_per_s"]) if fp64 else None,
        "roofline": roof,
        "pipe_peaks": pipes,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "trials/s", "h2d_bytes_per_step": int(users_h.nbytes),
                "d2h_bytes_per_step": int(rate_pin.numel() * 8 + 24)},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
