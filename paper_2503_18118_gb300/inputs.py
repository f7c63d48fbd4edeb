"""Seeded synthetic inputs (user geometry, powers, noise) for the Monte-Carlo
workloads.  Holds none of the method's arithmetic: it only draws positions
and per-trial scalars, which both the CUDA path and the CPU oracle then take
as inputs.

Every draw uses NumPy's counter-based Philox generator keyed by the seed;
arrays are drawn in trial-major order so that the first b trials of a batch
do not depend on the batch size.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

C_LIGHT = 299_792_458.0


def wavelength(freq_hz: float) -> float:
    return C_LIGHT / freq_hz


def _gen(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=int(seed)))


def users_polar(seed: int, B: int, K: int, r_range, theta_deg=(-60.0, 60.0)) -> np.ndarray:
    """[B][K][2] float64 user positions (x, y): distance r ~ U[r_range],
    angle from broadside theta ~ U[theta_deg], x = r cos theta, y = r sin theta."""
    u = _gen(seed).random((B, K, 2))
    r = r_range[0] + (r_range[1] - r_range[0]) * u[..., 0]
    th = np.deg2rad(theta_deg[0] + (theta_deg[1] - theta_deg[0]) * u[..., 1])
    return np.ascontiguousarray(np.stack([r * np.cos(th), r * np.sin(th)], axis=-1))


def users_rect(seed: int, B: int, K: int, x_range, y_range) -> np.ndarray:
    """[B][K][2] float64 users uniform on a rectangle x ~ U[x_range], y ~ U[y_range]."""
    u = _gen(seed).random((B, K, 2))
    x = x_range[0] + (x_range[1] - x_range[0]) * u[..., 0]
    y = y_range[0] + (y_range[1] - y_range[0]) * u[..., 1]
    return np.ascontiguousarray(np.stack([x, y], axis=-1))


def db_to_lin(db):
    return 10.0 ** (np.asarray(db, dtype=np.float64) / 10.0)


@dataclass
class Workload:
    """One synthetic Monte-Carlo workload."""
    name: str
    freq_hz: float
    n_ant: int
    k: int
    trials: int
    r_range: tuple
    theta_deg: tuple = (-60.0, 60.0)
    model: int = 1            # 0 PNUSW, 1 free-space USW, 2 UPW
    scheme: int = 1           # 0 ZF, 1 MMSE, 2 MRC
    snr_db: float = 10.0      # per-user received SNR
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def wavelength(self) -> float:
        return wavelength(self.freq_hz)

    @property
    def spacing(self) -> float:
        return 0.5 * self.wavelength

    def users(self, trials: int | None = None) -> np.ndarray:
        return users_polar(self.seed, self.trials if trials is None else trials, self.k,
                           self.r_range, self.theta_deg)

    def power(self, trials: int | None = None) -> np.ndarray:
        """Per-user received SNR (linear), [B][K]."""
        B = self.trials if trials is None else trials
        return np.full((B, self.k), float(db_to_lin(self.snr_db)), np.float64)

    def noise(self, trials: int | None = None) -> np.ndarray:
        B = self.trials if trials is None else trials
        return np.ones((B,), np.float64)


# 28 GHz, half-wavelength ULA, N = 256, K = 4 users at r in [5, 50] m and
# theta in [-60, 60] deg, free-space spherical-wave channel, ZF at 10 dB.
SMALL_FP64 = Workload("ula28ghz_n256_k4_zf", 28e9, 256, 4, 100, (5.0, 50.0), scheme=0, seed=1)

# 100 GHz, N = 16384, K = 32 users at r in [3, 30] m, MMSE at 10 dB, 10^4 trials.
HEADLINE = Workload("ula100ghz_n16384_k32_mmse", 100e9, 16384, 32, 10_000, (3.0, 30.0), scheme=1, seed=3)

# Saturation sweep: 28 GHz geometry, K = 8, N = 2^6 .. 2^16, 1000 trials per N.
SWEEP = Workload("ula28ghz_k8_sweep", 28e9, 65536, 8, 1000, (5.0, 50.0), scheme=0, seed=2,
                 extra={"n_list": [2 ** e for e in range(6, 17)], "snr_db": [0.0, 10.0, 20.0], "t": 0.9})


# Learned surrogate: trained on 10^7 pairs from K = 64 trials with N
# log-uniform in [2^10, 2^18] and a carrier of 28 GHz (r in [5, 50] m) or
# 100 GHz (r in [3, 30] m); evaluated at 100 GHz, N = 2^18, K = 64, 10^4 trials.
# base 2: the network corrects the closed form times the finite-aperture
# Fresnel factor.
SURROGATE = Workload("ula100ghz_n262144_k64_surrogate", 100e9, 262144, 64, 10_000, (3.0, 30.0), scheme=0, seed=5,
                     extra={"train_pairs": 10_000_000, "n_log2": (10.0, 18.0), "train_seed": 5, "eval_seed": 6,
                            "steps": 8000, "batch": 16384, "lr": 1e-3, "base": 2})


def ragged_instances(seed: int, count: int, n_log2=(10.0, 17.0), k_range=(2, 64),
                     snr_db=(0.0, 30.0)):
    """Per-instance (N, K, scheme, snr_db) for a ragged batch: N = round(2^U[n_log2]),
    K ~ U{k_range}, scheme ZF/MMSE with probability 1/2 each, SNR ~ U[snr_db]."""
    g = _gen(seed)
    u = g.random((count, 4))
    n = np.rint(2.0 ** (n_log2[0] + (n_log2[1] - n_log2[0]) * u[:, 0])).astype(np.int64)
    k = (k_range[0] + np.floor(u[:, 1] * (k_range[1] - k_range[0] + 1))).astype(np.int32)
    k = np.minimum(k, k_range[1])
    scheme = (u[:, 2] >= 0.5).astype(np.int32)
    snr = snr_db[0] + (snr_db[1] - snr_db[0]) * u[:, 3]
    return n, k, scheme, snr


def mlp_init_params(seed: int, dims=(6, 256, 256, 256, 256, 2)) -> np.ndarray:
    """Initial network parameters, float32, in the library's layout (per layer
    W [in][out] row-major, then b [out]): W ~ U(-1/sqrt(in), 1/sqrt(in)), b = 0."""
    g = _gen(seed)
    parts = []
    for a, b in zip(dims[:-1], dims[1:]):
        lim = 1.0 / math.sqrt(a)
        parts.append(((g.random((a, b)) * 2.0 - 1.0) * lim).reshape(-1))
        parts.append(np.zeros(b))
    return np.concatenate(parts).astype(np.float32)


def surrogate_trials(seed: int, trials: int, k: int, n_log2=(10.0, 18.0), bands=((28e9, (5.0, 50.0)), (100e9, (3.0, 30.0))),
                     theta_deg=(-60.0, 60.0)):
    """Training trials of the correlation surrogate: per trial N = round(2^U[n_log2]),
    a carrier band drawn uniformly from `bands` (frequency, distance range), and
    k users drawn as in users_polar.  Returns (n [T] int64, freq [T], users [T][k][2])."""
    g = _gen(seed)
    u = g.random((trials, 2))
    n = np.rint(2.0 ** (n_log2[0] + (n_log2[1] - n_log2[0]) * u[:, 0])).astype(np.int64)
    band = np.minimum((u[:, 1] * len(bands)).astype(np.int64), len(bands) - 1)
    freq = np.array([bands[b][0] for b in band])
    w = g.random((trials, k, 2))
    users = np.empty((trials, k, 2))
    for t in range(trials):
        lo, hi = bands[band[t]][1]
        r = lo + (hi - lo) * w[t, :, 0]
        th = np.deg2rad(theta_deg[0] + (theta_deg[1] - theta_deg[0]) * w[t, :, 1])
        users[t, :, 0] = r * np.cos(th)
        users[t, :, 1] = r * np.sin(th)
    return n, freq, users


def deg(x):
    return math.radians(x)
