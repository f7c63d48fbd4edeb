"""Plain FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA product path never does: it
shares no code, header, table or helper with anything here.

``xlmimo_oracle.c`` holds the per-trial arithmetic (explicit channel vectors,
explicit inner products, Gauss-Jordan inverses, pivot-product determinants);
``ergodic.py`` holds the ergodic saturation analysis (SciPy quadrature and
incomplete beta).  ``build()`` compiles the C part with gcc into
``liboracle.so`` next to this file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xlmimo_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

PNUSW, FSPL, UPW = 0, 1, 2
ZF, MMSE, MRC, ZF_DL = 0, 1, 2, 3
POWER_ABS, POWER_RXSNR = 0, 1


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, FP64, OpenMP over trials)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        i64, c_int, c_double = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        L.oracle_num_threads.restype = c_int
        L.oracle_channel.argtypes = [c_int, i64, c_double, c_double, c_double, c_double, c_double, dp]
        L.oracle_gram.argtypes = [c_int, i64, c_double, c_double, c_double, dp, c_int, c_int, dp]
        L.oracle_gram_ura.argtypes = [c_int, i64, i64, c_double, c_double, c_double, dp, c_int, c_int, dp]
        L.oracle_closed_form.argtypes = [c_int, i64, c_double, c_double, c_double, dp, c_int, c_int, dp]
        L.oracle_beamform.argtypes = [dp, dp, dp, dp, c_int, c_int, c_int, c_int, dp, ip, dp]
        L.oracle_sumrate.argtypes = [dp, c_int, c_int, dp, dp]
        L.oracle_saturation.argtypes = [dp, c_int, c_int, c_double, c_double, dp]
        for f in ("oracle_channel", "oracle_gram", "oracle_gram_ura", "oracle_closed_form", "oracle_beamform",
                  "oracle_sumrate", "oracle_saturation"):
            getattr(L, f).restype = c_int
        _lib = L
    return _lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def channel(model, n_ant, wavelength, spacing, beta0, x, y):
    """h[n], n = 0..N-1, complex128."""
    out = np.empty((n_ant, 2), np.float64)
    rc = lib().oracle_channel(model, n_ant, wavelength, spacing, beta0, x, y, _dp(out))
    assert rc == 0
    return out[:, 0] + 1j * out[:, 1]


def gram(model, n_ant, wavelength, spacing, beta0, users):
    """Exact Gram H^H H, complex128 [B][K][K], G[b,i,j] = h_i^H h_j."""
    users = _f64(users)
    B, K, _ = users.shape
    out = np.empty((B, K, K, 2), np.float64)
    rc = lib().oracle_gram(model, n_ant, wavelength, spacing, beta0, _dp(users), K, B, _dp(out))
    if rc:
        raise MemoryError("oracle_gram failed")
    return out[..., 0] + 1j * out[..., 1]


def gram_ura(model, n_ant, rows, wavelength, spacing, beta0, users):
    """Exact Gram of a URA of `rows` rows of `n_ant` elements (square lattice
    of the given spacing in the y-z plane, users in the plane z = 0),
    complex128 [B][K][K]."""
    users = _f64(users)
    B, K, _ = users.shape
    out = np.empty((B, K, K, 2), np.float64)
    rc = lib().oracle_gram_ura(model, n_ant, rows, wavelength, spacing, beta0, _dp(users), K, B, _dp(out))
    if rc:
        raise MemoryError("oracle_gram_ura failed")
    return out[..., 0] + 1j * out[..., 1]


def closed_form(model, n_ant, wavelength, spacing, beta0, users):
    """Closed-form Gram of modified ZF (Eqs. 4, 6), complex128 [B][K][K]."""
    users = _f64(users)
    B, K, _ = users.shape
    out = np.empty((B, K, K, 2), np.float64)
    rc = lib().oracle_closed_form(model, n_ant, wavelength, spacing, beta0, _dp(users), K, B, _dp(out))
    assert rc == 0
    return out[..., 0] + 1j * out[..., 1]


def _c2r(g):
    g = np.ascontiguousarray(g, dtype=np.complex128)
    return np.ascontiguousarray(np.stack([g.real, g.imag], axis=-1))


def beamform(gram_filter, power, noise, scheme, power_mode=POWER_ABS, gram_true=None,
             want_capacity=False):
    """Per-user SINR of a ZF / MMSE / MRC receiver built from gram_filter and
    evaluated on gram_true (defaults to gram_filter).  Returns
    (sinr [B][K], status [B], capacity [B] or None)."""
    gf = _c2r(gram_filter)
    B, K = gf.shape[0], gf.shape[1]
    gt = None if gram_true is None else _c2r(gram_true)
    power = _f64(np.broadcast_to(power, (B, K)))
    noise = _f64(np.broadcast_to(noise, (B,)))
    sinr = np.empty((B, K), np.float64)
    status = np.empty((B,), np.int32)
    cap = np.empty((B,), np.float64) if want_capacity else None
    rc = lib().oracle_beamform(_dp(gf), _dp(gt), _dp(power), _dp(noise), K, B, scheme, power_mode,
                               _dp(sinr), status.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(cap))
    if rc:
        raise MemoryError("oracle_beamform failed")
    return sinr, status, cap


def sumrate(sinr):
    """(rate [B], stats {mean, M2, count})."""
    sinr = _f64(sinr)
    B, K = sinr.shape
    rate = np.empty((B,), np.float64)
    stats = np.empty((3,), np.float64)
    lib().oracle_sumrate(_dp(sinr), K, B, _dp(rate), _dp(stats))
    return rate, stats


def saturation(users, t, spacing):
    """Per-trial (y_up, y_down, n_sat) of Eqs. (15)-(16)."""
    users = _f64(users)
    B, K, _ = users.shape
    out = np.empty((B, 3), np.float64)
    lib().oracle_saturation(_dp(users), K, B, t, spacing, _dp(out))
    return out
