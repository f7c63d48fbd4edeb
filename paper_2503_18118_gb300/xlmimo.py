"""Python binding of libxlmimo (include/xlmimo.h): argument marshalling only.

Every function has the name of the C entry point it calls and forwards
torch CUDA tensors as raw device pointers on the current torch stream.
There is no CPU fallback: a missing or unloadable library raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

PNUSW, FSPL_USW, UPW = 0, 1, 2
F64, F32, BF16, BF16X3, F16X3 = 0, 1, 2, 3, 4
ZF, MMSE, MRC, ZF_DL = 0, 1, 2, 3
MISMATCH_FP32 = 0x100  # OR-ed into a scheme: mismatched SINR from the FP32 correction
FACTOR_FF = 0x200  # OR-ed into a matched scheme: double-float factorisation (FP64 if ill-conditioned)
POWER_ABS, POWER_RXSNR = 0, 1
DIST_RECT, DIST_POLAR = 0, 1
APERTURE_NONE, APERTURE_MASK, APERTURE_FRESNEL = 0, 1, 2
PIPE_SINCOS, PIPE_RSQRT, PIPE_FFMA = 0, 1, 2
MAX_USERS = 64
MAX_BOUNDS_USERS = 1024
MAX_URA_ROWS = 1048576
NOALLOC_SCRATCH_MIB = 16  # XLMIMO_NOALLOC_SCRATCH_MIB
PLAN_INFO_LEN = 12  # XLMIMO_PLAN_INFO_LEN
STATUS = {0: "OK", 1: "EINVAL", 2: "ECUDA", 3: "ENOMEM", 4: "ESINGULAR", 5: "ETIMEOUT", 6: "EUNSUPPORTED"}


class XlmimoError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"xlmimo error {code} ({STATUS.get(code, '?')}): {msg}")
        self.code = code


class Array(ctypes.Structure):
    _fields_ = [("n_ant", ctypes.c_int64), ("wavelength", ctypes.c_double), ("spacing", ctypes.c_double),
                ("beta0", ctypes.c_double), ("model", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class UserDist(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("a0", ctypes.c_double),
                ("a1", ctypes.c_double), ("b0", ctypes.c_double), ("b1", ctypes.c_double)]


class SweepCfg(ctypes.Structure):
    _fields_ = [("wavelength", ctypes.c_double), ("spacing", ctypes.c_double), ("beta0", ctypes.c_double),
                ("model", ctypes.c_int32), ("prec", ctypes.c_int32), ("n_count", ctypes.c_int32),
                ("snr_count", ctypes.c_int32), ("n_list", ctypes.POINTER(ctypes.c_int64)),
                ("snr_db", ctypes.POINTER(ctypes.c_double)), ("users", ctypes.c_void_p),
                ("K", ctypes.c_int32), ("B", ctypes.c_int32), ("t", ctypes.c_double), ("ref_x", ctypes.c_double)]


class SweepResult(ctypes.Structure):
    _fields_ = [("rate", ctypes.POINTER(ctypes.c_double)), ("capacity", ctypes.POINTER(ctypes.c_double)),
                ("gram_err", ctypes.POINTER(ctypes.c_double)), ("sat_mean", ctypes.c_double * 3)]


class McBatch(ctypes.Structure):
    _fields_ = [("arr", Array), ("prec", ctypes.c_int32), ("scheme", ctypes.c_int32), ("cf_scheme", ctypes.c_int32),
                ("power_mode", ctypes.c_int32), ("K", ctypes.c_int32), ("B", ctypes.c_int32),
                ("chunks", ctypes.c_int32), ("reserved", ctypes.c_int32), ("t", ctypes.c_double)] + [
        (n, ctypes.c_void_p) for n in ("users", "power", "noise", "gram", "gram_cf", "sinr", "sinr_cf", "status",
                                       "status_cf", "capacity", "rate", "rate_cf", "stats", "stats_cf", "sat")]


class Inst(ctypes.Structure):
    _fields_ = [("n_ant", ctypes.c_int64), ("k", ctypes.c_int32), ("scheme", ctypes.c_int32),
                ("user_off", ctypes.c_int64), ("gram_off", ctypes.c_int64), ("noise", ctypes.c_double)]


EXPORTS = ("xlmimo_batch_plan_create", "xlmimo_batch_run", "xlmimo_batch_plan_info", "xlmimo_batch_plan_destroy",
           "xlmimo_batch_plan_set_tiling",
           "xlmimo_mc_step", "xlmimo_channel_gram", "xlmimo_channel_gram_ura", "xlmimo_channel_gram_noalloc",
           "xlmimo_corr_closed_form", "xlmimo_corr_closed_form_aperture", "xlmimo_beamform", "xlmimo_sumrate",
           "xlmimo_saturation", "xlmimo_saturation_analytic", "xlmimo_capacity_sweep", "xlmimo_capacity_bounds",
           "xlmimo_capacity_bounds_timed",
           "xlmimo_pair_features",
           "xlmimo_mlp_forward", "xlmimo_mlp_loss", "xlmimo_mlp_work_floats", "xlmimo_mlp_backward", "xlmimo_mlp_adam",
           "xlmimo_mlp_train_step", "xlmimo_mlp_pack", "xlmimo_surrogate_gram", "xlmimo_measure_pipe", "xlmimo_shutdown",
           "xlmimo_last_error", "xlmimo_version")

MLP_IN, MLP_WIDTH, MLP_HIDDEN, MLP_OUT = 6, 256, 4, 2
MLP_PARAMS = 199682
MLP_CACHE_PER_ROW = 2 * MLP_HIDDEN * MLP_WIDTH
MLP_PACKED_BYTES = 432384

_lib = None


def lib(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libxlmimo.so (building it first when it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libxlmimo.so not found at {_build.LIB}; run paper_2503_18118_gb300.build.build()")
    L = ctypes.CDLL(_build.LIB)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    L.xlmimo_channel_gram.argtypes = [ctypes.POINTER(Array), vp, i32, i32, i32, vp, vp]
    L.xlmimo_channel_gram_ura.argtypes = [ctypes.POINTER(Array), ctypes.c_int64, vp, i32, i32, i32, vp, vp]
    L.xlmimo_mc_step.argtypes = [ctypes.POINTER(McBatch), vp]
    L.xlmimo_batch_plan_create.argtypes = [ctypes.POINTER(Array), ctypes.POINTER(Inst), i32, i32, vp,
                                           ctypes.POINTER(vp), vp]
    L.xlmimo_batch_run.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp, vp]
    L.xlmimo_batch_plan_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
    L.xlmimo_batch_plan_set_tiling.argtypes = [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp]
    L.xlmimo_batch_plan_destroy.argtypes = [vp]
    L.xlmimo_channel_gram_noalloc.argtypes = [ctypes.POINTER(Array), vp, i32, i32, i32, vp, vp]
    L.xlmimo_corr_closed_form.argtypes = [ctypes.POINTER(Array), vp, i32, i32, vp, vp]
    L.xlmimo_beamform.argtypes = [vp, vp, vp, vp, i32, i32, i32, i32, vp, vp, vp, vp]
    L.xlmimo_sumrate.argtypes = [vp, i32, i32, vp, vp, vp]
    L.xlmimo_saturation.argtypes = [vp, i32, i32, dbl, dbl, vp, vp]
    L.xlmimo_saturation_analytic.argtypes = [ctypes.POINTER(UserDist), i32, dbl, dbl, ctypes.POINTER(dbl), vp]
    L.xlmimo_capacity_sweep.argtypes = [ctypes.POINTER(SweepCfg), ctypes.POINTER(SweepResult), vp]
    L.xlmimo_corr_closed_form_aperture.argtypes = [ctypes.POINTER(Array), vp, i32, i32, i32, vp, vp]
    L.xlmimo_capacity_bounds.argtypes = [ctypes.POINTER(Array), vp, i32, i32, dbl, vp, vp]
    L.xlmimo_capacity_bounds_timed.argtypes = [ctypes.POINTER(Array), vp, i32, i32, dbl, vp, vp, vp]
    L.xlmimo_pair_features.argtypes = [ctypes.POINTER(Array), vp, i32, i32, i32, vp, vp, vp, vp, vp, vp]
    L.xlmimo_mlp_forward.argtypes = [vp, vp, i32, vp, vp, vp]
    L.xlmimo_mlp_loss.argtypes = [vp, vp, vp, i32, vp, vp, vp]
    L.xlmimo_mlp_work_floats.argtypes = [i32]
    L.xlmimo_mlp_work_floats.restype = i64
    L.xlmimo_mlp_backward.argtypes = [vp, vp, vp, vp, i32, vp, vp, vp]
    L.xlmimo_mlp_adam.argtypes = [vp, vp, vp, vp, i64, dbl, dbl, dbl, dbl, vp]
    L.xlmimo_mlp_train_step.argtypes = [vp, vp, vp, vp, i64, dbl, vp, vp, vp, i32, vp, vp, vp, vp, vp]
    L.xlmimo_mlp_pack.argtypes = [vp, vp, vp]
    L.xlmimo_surrogate_gram.argtypes = [ctypes.POINTER(Array), vp, i32, i32, i32, vp, vp, vp]
    L.xlmimo_measure_pipe.argtypes = [i32, ctypes.POINTER(dbl), vp]
    L.xlmimo_last_error.restype = ctypes.c_char_p
    for f in EXPORTS:
        if f not in ("xlmimo_last_error", "xlmimo_mlp_work_floats"):
            getattr(L, f).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc):
    if rc != 0:
        raise XlmimoError(rc, lib().xlmimo_last_error().decode())


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _dev(t, dtype, name, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.device.index != torch.cuda.current_device():
        # the library launches on the current device: a pointer into another
        # GPU's memory is refused here rather than dereferenced there
        raise ValueError(f"{name} is on {t.device}, the current device is cuda:{torch.cuda.current_device()}")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def array(n_ant, wavelength, spacing=None, beta0=1.0, model=FSPL_USW) -> Array:
    return Array(int(n_ant), float(wavelength), float(0.5 * wavelength if spacing is None else spacing),
                 float(beta0), int(model), 0)


def xlmimo_version() -> int:
    return int(lib().xlmimo_version())


def xlmimo_shutdown() -> None:
    """Release the library's per-device pipeline stream and events."""
    _check(lib().xlmimo_shutdown())


def xlmimo_channel_gram(arr: Array, users: torch.Tensor, prec: int = F32, gram: torch.Tensor | None = None,
                        stream=None) -> torch.Tensor:
    """Exact Gram matrices H^H H, complex128 [B][K][K]."""
    B, K = users.shape[0], users.shape[1]
    if gram is None:
        gram = torch.empty((B, K, K), dtype=torch.complex128, device=users.device)
    _check(lib().xlmimo_channel_gram(ctypes.byref(arr), _dev(users, torch.float64, "users", (B, K, 2)), K, B,
                                     int(prec), _dev(gram, torch.complex128, "gram", (B, K, K)), _stream(stream)))
    return gram


def xlmimo_channel_gram_ura(arr: Array, rows: int, users: torch.Tensor, prec: int = F32,
                            gram: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Exact Gram matrices of a URA of `rows` rows of arr.n_ant elements
    (users in the plane z = 0), complex128 [B][K][K]."""
    B, K = users.shape[0], users.shape[1]
    if gram is None:
        gram = torch.empty((B, K, K), dtype=torch.complex128, device=users.device)
    _check(lib().xlmimo_channel_gram_ura(ctypes.byref(arr), ctypes.c_int64(int(rows)),
                                         _dev(users, torch.float64, "users", (B, K, 2)), K, B, int(prec),
                                         _dev(gram, torch.complex128, "gram", (B, K, K)), _stream(stream)))
    return gram


class McBuffers:
    """Device buffers of one Monte-Carlo step over B trials of K users."""

    def __init__(self, B, K, device="cuda", capacity=True, closed_form=True, saturation=True):
        f64, c128, i32 = torch.float64, torch.complex128, torch.int32
        e = lambda shape, dt: torch.empty(shape, dtype=dt, device=device)
        self.gram = e((B, K, K), c128)
        self.gram_cf = e((B, K, K), c128) if closed_form else None
        self.sinr = e((B, K), f64)
        self.sinr_cf = e((B, K), f64) if closed_form else None
        self.status = e((B,), i32)
        self.status_cf = e((B,), i32) if closed_form else None
        self.capacity = e((B,), f64) if capacity else None
        self.rate = e((B,), f64)
        self.rate_cf = e((B,), f64) if closed_form else None
        self.stats = e((3,), f64)
        self.stats_cf = e((3,), f64) if closed_form else None
        self.sat = e((B, 3), f64) if saturation else None


def xlmimo_mc_step(arr: Array, users: torch.Tensor, power: torch.Tensor, noise: torch.Tensor, out: McBuffers,
                   prec: int = BF16X3, scheme: int = MMSE, cf_scheme: int = ZF, power_mode: int = POWER_RXSNR,
                   t: float = 0.9, chunks: int = 0, stream=None) -> McBuffers:
    """One pipelined Monte-Carlo step (exact Gram, receivers, rates, closed-form
    path, saturation) over the batch; results land in `out`."""
    B, K = users.shape[0], users.shape[1]
    ptr = lambda x, dt, name, shape: None if x is None else _dev(x, dt, name, shape)
    f64, c128, i32 = torch.float64, torch.complex128, torch.int32
    job = McBatch(arr, int(prec), int(scheme), int(cf_scheme if out.gram_cf is not None else -1), int(power_mode),
                  K, B, int(chunks), 0, float(t if out.sat is not None else 0.0),
                  _dev(users, f64, "users", (B, K, 2)), _dev(power, f64, "power", (B, K)),
                  _dev(noise, f64, "noise", (B,)), _dev(out.gram, c128, "gram", (B, K, K)),
                  ptr(out.gram_cf, c128, "gram_cf", (B, K, K)), _dev(out.sinr, f64, "sinr", (B, K)),
                  ptr(out.sinr_cf, f64, "sinr_cf", (B, K)), _dev(out.status, i32, "status", (B,)),
                  ptr(out.status_cf, i32, "status_cf", (B,)), ptr(out.capacity, f64, "capacity", (B,)),
                  _dev(out.rate, f64, "rate", (B,)), ptr(out.rate_cf, f64, "rate_cf", (B,)),
                  ptr(out.stats, f64, "stats", (3,)), ptr(out.stats_cf, f64, "stats_cf", (3,)),
                  ptr(out.sat, f64, "sat", (B, 3)))
    _check(lib().xlmimo_mc_step(ctypes.byref(job), _stream(stream)))
    return out


def xlmimo_channel_gram_noalloc(arr: Array, users: torch.Tensor, prec: int = F32, gram: torch.Tensor | None = None,
                                stream=None) -> torch.Tensor:
    """Exact Gram matrices like xlmimo_channel_gram, for callers that cannot
    allocate device memory while they run (a host that reserves the GPU's
    memory for its own pool, or a latency-critical loop that cannot accept
    cudaMalloc / cudaFree).  The library itself allocates nothing here: the
    split partial sums use a fixed 16 MiB device array, so a batch whose split
    needs more is rejected.  Calls that overlap on the GPU race on that array.
    Pass `gram` to avoid the one torch allocation this wrapper would make."""
    B, K = users.shape[0], users.shape[1]
    if gram is None:
        gram = torch.empty((B, K, K), dtype=torch.complex128, device=users.device)
    _check(lib().xlmimo_channel_gram_noalloc(ctypes.byref(arr), _dev(users, torch.float64, "users", (B, K, 2)), K, B,
                                             int(prec), _dev(gram, torch.complex128, "gram", (B, K, K)),
                                             _stream(stream)))
    return gram


def xlmimo_corr_closed_form(arr: Array, users: torch.Tensor, gram: torch.Tensor | None = None,
                            stream=None) -> torch.Tensor:
    """Closed-form Gram matrices of modified ZF, complex128 [B][K][K]."""
    B, K = users.shape[0], users.shape[1]
    if gram is None:
        gram = torch.empty((B, K, K), dtype=torch.complex128, device=users.device)
    _check(lib().xlmimo_corr_closed_form(ctypes.byref(arr), _dev(users, torch.float64, "users", (B, K, 2)), K, B,
                                         _dev(gram, torch.complex128, "gram", (B, K, K)), _stream(stream)))
    return gram


def xlmimo_capacity_bounds(arr: Array, users: torch.Tensor, snr: float, out: torch.Tensor | None = None,
                           stream=None) -> torch.Tensor:
    """Appendix A per trial, float64 [B][4]: log2 det R, log2 det(I + snr R),
    log2 U = K log2(1 + snr), log2 L = log2 det R + log2 U (users [B][K][2],
    K <= MAX_BOUNDS_USERS, snr linear)."""
    B, K = users.shape[0], users.shape[1]
    if out is None:
        out = torch.empty((B, 4), dtype=torch.float64, device=users.device)
    _check(lib().xlmimo_capacity_bounds(ctypes.byref(arr), _dev(users, torch.float64, "users", (B, K, 2)), K, B,
                                        float(snr), _dev(out, torch.float64, "out", (B, 4)), _stream(stream)))
    return out


def xlmimo_capacity_bounds_timed(arr: Array, users: torch.Tensor, snr: float, out: torch.Tensor | None = None,
                                 stream=None):
    """(xlmimo_capacity_bounds's output, [5] device milliseconds of its phases:
    channels, tensor-core Gram, correlation matrices, Cholesky, bounds).
    Synchronous."""
    B, K = users.shape[0], users.shape[1]
    if out is None:
        out = torch.empty((B, 4), dtype=torch.float64, device=users.device)
    ms = (ctypes.c_float * 5)()
    _check(lib().xlmimo_capacity_bounds_timed(ctypes.byref(arr), _dev(users, torch.float64, "users", (B, K, 2)), K,
                                              B, float(snr), _dev(out, torch.float64, "out", (B, 4)),
                                              ctypes.cast(ms, ctypes.c_void_p), _stream(stream)))
    return out, [float(v) for v in ms]


def xlmimo_corr_closed_form_aperture(arr: Array, users: torch.Tensor, mode: int, gram: torch.Tensor | None = None,
                                     stream=None) -> torch.Tensor:
    """Closed form with the finite-aperture correction `mode` (APERTURE_*), complex128 [B][K][K]."""
    B, K = users.shape[0], users.shape[1]
    if gram is None:
        gram = torch.empty((B, K, K), dtype=torch.complex128, device=users.device)
    _check(lib().xlmimo_corr_closed_form_aperture(ctypes.byref(arr), _dev(users, torch.float64, "users", (B, K, 2)), K,
                                                  B, int(mode), _dev(gram, torch.complex128, "gram", (B, K, K)),
                                                  _stream(stream)))
    return gram


def xlmimo_beamform(gram_filter: torch.Tensor, power: torch.Tensor, noise: torch.Tensor, scheme: int,
                    power_mode: int = POWER_ABS, gram_true: torch.Tensor | None = None, capacity: bool = False,
                    sinr: torch.Tensor | None = None, status: torch.Tensor | None = None,
                    cap: torch.Tensor | None = None, stream=None):
    """(sinr [B][K] float64, status [B] int32, capacity [B] float64 or None)."""
    B, K = gram_filter.shape[0], gram_filter.shape[1]
    dev = gram_filter.device
    if sinr is None:
        sinr = torch.empty((B, K), dtype=torch.float64, device=dev)
    if status is None:
        status = torch.empty((B,), dtype=torch.int32, device=dev)
    if capacity and cap is None:
        cap = torch.empty((B,), dtype=torch.float64, device=dev)
    gt = None if gram_true is None else _dev(gram_true, torch.complex128, "gram_true", (B, K, K))
    _check(lib().xlmimo_beamform(_dev(gram_filter, torch.complex128, "gram_filter", (B, K, K)), gt,
                                 _dev(power, torch.float64, "power", (B, K)), _dev(noise, torch.float64, "noise", (B,)),
                                 K, B, int(scheme), int(power_mode), _dev(sinr, torch.float64, "sinr", (B, K)),
                                 _dev(status, torch.int32, "status", (B,)),
                                 None if cap is None else _dev(cap, torch.float64, "cap", (B,)), _stream(stream)))
    return sinr, status, cap


def xlmimo_sumrate(sinr: torch.Tensor, rate: torch.Tensor | None = None, stats: torch.Tensor | None = None,
                   want_stats: bool = True, stream=None):
    """(rate [B], stats [3] = {mean, M2, count} or None)."""
    B, K = sinr.shape
    if rate is None:
        rate = torch.empty((B,), dtype=torch.float64, device=sinr.device)
    if want_stats and stats is None:
        stats = torch.empty((3,), dtype=torch.float64, device=sinr.device)
    _check(lib().xlmimo_sumrate(_dev(sinr, torch.float64, "sinr", (B, K)), K, B,
                                _dev(rate, torch.float64, "rate", (B,)),
                                None if stats is None else _dev(stats, torch.float64, "stats", (3,)), _stream(stream)))
    return rate, stats


def xlmimo_saturation(users: torch.Tensor, t: float, spacing: float, sat: torch.Tensor | None = None,
                      stream=None) -> torch.Tensor:
    """Per-trial {y_up, y_down, n_sat}, float64 [B][3]."""
    B, K = users.shape[0], users.shape[1]
    if sat is None:
        sat = torch.empty((B, 3), dtype=torch.float64, device=users.device)
    _check(lib().xlmimo_saturation(_dev(users, torch.float64, "users", (B, K, 2)), K, B, float(t), float(spacing),
                                   _dev(sat, torch.float64, "sat", (B, 3)), _stream(stream)))
    return sat


def xlmimo_measure_pipe(pipe: int, stream=None):
    """(operations per second, best launch ms) of one pipe -- synchronous."""
    out = (ctypes.c_double * 2)()
    _check(lib().xlmimo_measure_pipe(int(pipe), out, _stream(stream)))
    return out[0], out[1]


def xlmimo_saturation_analytic(kind: int, a0: float, a1: float, b0: float, b1: float, K: int, t: float,
                               spacing: float, stream=None):
    """(E[y_up], E[y_down], aperture/spacing v, ceil(v), near-integer flag,
    the other candidate count) -- synchronous."""
    d = UserDist(int(kind), 0, float(a0), float(a1), float(b0), float(b1))
    out = (ctypes.c_double * 6)()
    _check(lib().xlmimo_saturation_analytic(ctypes.byref(d), int(K), float(t), float(spacing), out, _stream(stream)))
    return tuple(out)


def xlmimo_capacity_sweep(users: torch.Tensor, n_list, snr_db, wavelength: float, spacing: float | None = None,
                          beta0: float = 1.0, model: int = FSPL_USW, prec: int = F32, t: float = 0.9,
                          ref_x: float = 1.0, stream=None) -> dict:
    """Synchronous sweep over array sizes; returns host numpy arrays."""
    import numpy as np
    B, K = users.shape[0], users.shape[1]
    n_arr = (ctypes.c_int64 * len(n_list))(*[int(n) for n in n_list])
    s_arr = (ctypes.c_double * len(snr_db))(*[float(s) for s in snr_db])
    cfg = SweepCfg(float(wavelength), float(0.5 * wavelength if spacing is None else spacing), float(beta0),
                   int(model), int(prec), len(n_list), len(snr_db), n_arr, s_arr,
                   _dev(users, torch.float64, "users", (B, K, 2)), K, B, float(t), float(ref_x))
    rate = np.zeros((len(n_list), 2, 2, len(snr_db)))
    cap = np.zeros((len(n_list), len(snr_db)))
    err = np.zeros((len(n_list),))
    res = SweepResult(rate.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                      cap.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                      err.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), (ctypes.c_double * 3)())
    _check(lib().xlmimo_capacity_sweep(ctypes.byref(cfg), ctypes.byref(res), _stream(stream)))
    return {"rate": rate, "capacity": cap, "gram_err": err, "sat_mean": tuple(res.sat_mean)}


class BatchPlan:
    """A ragged batch of instances (own N, K, receiver, noise) sharing the array
    geometry of `arr` (its n_ant is ignored).  Users, powers and SINRs are packed
    per instance in order; Gram matrices are packed K_i x K_i blocks."""

    def __init__(self, arr: Array, n_ant, k, scheme, noise, prec: int = BF16X3, tune_users: torch.Tensor | None = None,
                 stream=None):
        import numpy as np
        n_ant, k = np.asarray(n_ant, np.int64), np.asarray(k, np.int64)
        scheme, noise = np.asarray(scheme, np.int64), np.asarray(noise, np.float64)
        self.count = len(n_ant)
        self.k = k
        self.user_off = np.concatenate([[0], np.cumsum(k)[:-1]]).astype(np.int64)
        self.gram_off = np.concatenate([[0], np.cumsum(k * k)[:-1]]).astype(np.int64)
        self.users_total = int(k.sum())
        self.gram_total = int((k * k).sum())
        insts = (Inst * self.count)(*[Inst(int(n_ant[i]), int(k[i]), int(scheme[i]), int(self.user_off[i]),
                                           int(self.gram_off[i]), float(noise[i])) for i in range(self.count)])
        h = ctypes.c_void_p()
        tu = None if tune_users is None else _dev(tune_users, torch.float64, "tune_users", (self.users_total, 2))
        _check(lib().xlmimo_batch_plan_create(ctypes.byref(arr), insts, self.count, int(prec), tu, ctypes.byref(h),
                                              _stream(stream)))
        self._h = h

    def set_tiling(self, chunk: int, mode: int, narrow_kmax: int, pack: int = 1, stream=None):
        """Pin the tiling (element chunk, launch mode, narrow cut-off, packing), overriding the tuner."""
        _check(lib().xlmimo_batch_plan_set_tiling(self._h, int(chunk), int(mode), int(narrow_kmax), int(pack),
                                                  _stream(stream)))

    def run(self, users, power, power_mode, gram, sinr, status, rate, stream=None):
        U, n = self.users_total, self.count
        _check(lib().xlmimo_batch_run(self._h, _dev(users, torch.float64, "users", (U, 2)),
                                      _dev(power, torch.float64, "power", (U,)), int(power_mode),
                                      _dev(gram, torch.complex128, "gram", (self.gram_total,)),
                                      _dev(sinr, torch.float64, "sinr", (U,)), _dev(status, torch.int32, "status", (n,)),
                                      _dev(rate, torch.float64, "rate", (n,)), _stream(stream)))

    def run_gram(self, users, gram, stream=None):
        """The plan's Gram matrices only (no receivers)."""
        _check(lib().xlmimo_batch_run(self._h, _dev(users, torch.float64, "users", (self.users_total, 2)), None, 0,
                                      _dev(gram, torch.complex128, "gram", (self.gram_total,)), None, None, None,
                                      _stream(stream)))

    def info(self) -> dict:
        v = (ctypes.c_int64 * PLAN_INFO_LEN)()
        _check(lib().xlmimo_batch_plan_info(self._h, v))
        keys = ("items", "chunk", "mode", "small", "large", "workspace_bytes", "tuned", "candidates", "narrow_kmax",
                "wide_ctas", "pack", "narrow_ctas")
        return dict(zip(keys, list(v)))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().xlmimo_batch_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- learned correlation surrogate -------------------------------------------------------------

def _opt(t, dtype, name, shape=None):
    return ctypes.c_void_p(0) if t is None else _dev(t, dtype, name, shape)


def xlmimo_pair_features(arr: Array, users: torch.Tensor, gram: torch.Tensor | None = None,
                         gram_cf: torch.Tensor | None = None, weights: bool = False, base: int = APERTURE_NONE,
                         stream=None):
    """(feat [B*P][6], target [B*P][2] or None, weight [B*P] or None), float32, P = K(K-1)/2;
    targets G/G~ - F with F the aperture factor `base`."""
    B, K = users.shape[0], users.shape[1]
    rows = B * (K * (K - 1) // 2)
    dev = users.device
    feat = torch.empty((rows, MLP_IN), dtype=torch.float32, device=dev)
    target = torch.empty((rows, MLP_OUT), dtype=torch.float32, device=dev) if gram is not None else None
    weight = torch.empty((rows,), dtype=torch.float32, device=dev) if weights else None
    _check(lib().xlmimo_pair_features(ctypes.byref(arr), _dev(users, torch.float64, "users", (B, K, 2)), K, B,
                                      int(base), _opt(gram, torch.complex128, "gram", (B, K, K)),
                                      _opt(gram_cf, torch.complex128, "gram_cf", (B, K, K)),
                                      _dev(feat, torch.float32, "feat"), _opt(target, torch.float32, "target"),
                                      _opt(weight, torch.float32, "weight"), _stream(stream)))
    return feat, target, weight


def xlmimo_mlp_forward(params: torch.Tensor, x: torch.Tensor, cache: torch.Tensor | None = None,
                       out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Network output [M][2] float32 (cache, if given, receives z and h of every hidden layer)."""
    M = x.shape[0]
    if out is None:
        out = torch.empty((M, MLP_OUT), dtype=torch.float32, device=x.device)
    _check(lib().xlmimo_mlp_forward(_dev(params, torch.float32, "params", (MLP_PARAMS,)),
                                    _dev(x, torch.float32, "x", (M, MLP_IN)), M,
                                    _dev(out, torch.float32, "out", (M, MLP_OUT)),
                                    _opt(cache, torch.float32, "cache", (M * MLP_CACHE_PER_ROW,)), _stream(stream)))
    return out


def xlmimo_mlp_loss(out: torch.Tensor, target: torch.Tensor, weight: torch.Tensor | None = None,
                    dout: torch.Tensor | None = None, loss: torch.Tensor | None = None, stream=None):
    """(dout [M][2], loss [1]) float32."""
    M = out.shape[0]
    if dout is None:
        dout = torch.empty_like(out)
    if loss is None:
        loss = torch.empty((1,), dtype=torch.float32, device=out.device)
    _check(lib().xlmimo_mlp_loss(_dev(out, torch.float32, "out", (M, MLP_OUT)),
                                 _dev(target, torch.float32, "target", (M, MLP_OUT)),
                                 _opt(weight, torch.float32, "weight", (M,)), M,
                                 _dev(dout, torch.float32, "dout", (M, MLP_OUT)), _dev(loss, torch.float32, "loss"),
                                 _stream(stream)))
    return dout, loss


def xlmimo_mlp_work_floats(M: int) -> int:
    return int(lib().xlmimo_mlp_work_floats(int(M)))


def xlmimo_mlp_backward(params: torch.Tensor, x: torch.Tensor, cache: torch.Tensor, dout: torch.Tensor,
                        grad: torch.Tensor | None = None, work: torch.Tensor | None = None, stream=None):
    """Gradient [MLP_PARAMS] float32 of the loss whose output gradient is dout."""
    M = x.shape[0]
    if grad is None:
        grad = torch.empty((MLP_PARAMS,), dtype=torch.float32, device=x.device)
    if work is None:
        work = torch.empty((max(1, xlmimo_mlp_work_floats(M)),), dtype=torch.float32, device=x.device)
    _check(lib().xlmimo_mlp_backward(_dev(params, torch.float32, "params", (MLP_PARAMS,)),
                                     _dev(x, torch.float32, "x", (M, MLP_IN)),
                                     _dev(cache, torch.float32, "cache", (M * MLP_CACHE_PER_ROW,)),
                                     _dev(dout, torch.float32, "dout", (M, MLP_OUT)), M,
                                     _dev(grad, torch.float32, "grad", (MLP_PARAMS,)), _dev(work, torch.float32, "work"),
                                     _stream(stream)))
    return grad


def xlmimo_mlp_adam(params: torch.Tensor, m: torch.Tensor, v: torch.Tensor, grad: torch.Tensor, step: int,
                    lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, stream=None):
    for t, n in ((params, "params"), (m, "m"), (v, "v"), (grad, "grad")):
        _dev(t, torch.float32, n, (MLP_PARAMS,))
    _check(lib().xlmimo_mlp_adam(_dev(params, torch.float32, "params"), _dev(m, torch.float32, "m"),
                                 _dev(v, torch.float32, "v"), _dev(grad, torch.float32, "grad"), int(step), float(lr),
                                 float(beta1), float(beta2), float(eps), _stream(stream)))


def xlmimo_mlp_train_step(params, m, v, grad, step: int, lr: float, x, target, weight, out, cache, work, loss,
                          stream=None):
    """Forward, loss, backward and Adam on one batch (all buffers caller-owned, see the C header)."""
    M = x.shape[0]
    _check(lib().xlmimo_mlp_train_step(
        _dev(params, torch.float32, "params", (MLP_PARAMS,)), _dev(m, torch.float32, "m", (MLP_PARAMS,)),
        _dev(v, torch.float32, "v", (MLP_PARAMS,)), _dev(grad, torch.float32, "grad", (MLP_PARAMS,)), int(step),
        float(lr), _dev(x, torch.float32, "x", (M, MLP_IN)), _dev(target, torch.float32, "target", (M, MLP_OUT)),
        _opt(weight, torch.float32, "weight", (M,)), M, _dev(out, torch.float32, "out", (M, MLP_OUT)),
        _dev(cache, torch.float32, "cache", (M * MLP_CACHE_PER_ROW,)), _dev(work, torch.float32, "work"),
        _opt(loss, torch.float32, "loss"), _stream(stream)))


def xlmimo_mlp_pack(params: torch.Tensor, packed: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """BF16 inference image (uint8 [MLP_PACKED_BYTES]) for xlmimo_surrogate_gram."""
    if packed is None:
        packed = torch.empty((MLP_PACKED_BYTES,), dtype=torch.uint8, device=params.device)
    _check(lib().xlmimo_mlp_pack(_dev(params, torch.float32, "params", (MLP_PARAMS,)),
                                 _dev(packed, torch.uint8, "packed", (MLP_PACKED_BYTES,)), _stream(stream)))
    return packed


def xlmimo_surrogate_gram(arr: Array, users: torch.Tensor, packed: torch.Tensor, gram: torch.Tensor | None = None,
                          base: int = APERTURE_NONE, stream=None) -> torch.Tensor:
    """Surrogate Gram matrices, complex128 [B][K][K]: closed form times (F + t), F the
    aperture factor `base` the network was trained with, t from the network."""
    B, K = users.shape[0], users.shape[1]
    if gram is None:
        gram = torch.empty((B, K, K), dtype=torch.complex128, device=users.device)
    _check(lib().xlmimo_surrogate_gram(ctypes.byref(arr), _dev(users, torch.float64, "users", (B, K, 2)), K, B,
                                       int(base), _dev(packed, torch.uint8, "packed", (MLP_PACKED_BYTES,)),
                                       _dev(gram, torch.complex128, "gram", (B, K, K)), _stream(stream)))
    return gram

