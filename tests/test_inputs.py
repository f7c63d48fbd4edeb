"""The seeded input generators that the CUDA path and the oracle both draw
from: deterministic per seed, trial-major (the first b trials of a batch do
not depend on the batch size, which the sampled full-size checks and the
oracle's timed sample rely on), and within the ranges each workload states."""
import math
import os
import re

import numpy as np
import pytest

from paper_2503_18118_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_users_are_trial_major_and_seeded():
    a = inputs.users_polar(3, 100, 32, (3.0, 30.0))
    b = inputs.users_polar(3, 7, 32, (3.0, 30.0))
    assert np.array_equal(a[:7], b)
    assert np.array_equal(a, inputs.users_polar(3, 100, 32, (3.0, 30.0)))
    assert not np.array_equal(a[:7], inputs.users_polar(4, 7, 32, (3.0, 30.0)))
    r = inputs.users_rect(9, 50, 8, (1.0, 10.0), (-7.5, 7.5))
    assert np.array_equal(r[:5], inputs.users_rect(9, 5, 8, (1.0, 10.0), (-7.5, 7.5)))
    # the workload's own draw is the same generator
    wl = inputs.HEADLINE
    assert np.array_equal(wl.users(16), inputs.users_polar(wl.seed, 16, wl.k, wl.r_range, wl.theta_deg))


def test_polar_and_rect_ranges():
    u = inputs.users_polar(1, 2000, 16, (3.0, 30.0), (-60.0, 60.0))
    assert u.shape == (2000, 16, 2) and u.dtype == np.float64 and u.flags.c_contiguous
    r = np.hypot(u[..., 0], u[..., 1])
    th = np.degrees(np.arctan2(u[..., 1], u[..., 0]))
    assert r.min() >= 3.0 and r.max() <= 30.0
    assert th.min() >= -60.0 - 1e-9 and th.max() <= 60.0 + 1e-9
    assert (u[..., 0] > 0).all()  # users in front of the array
    # uniform in r and theta: means near the midpoints
    assert abs(r.mean() - 16.5) < 0.2 and abs(th.mean()) < 0.8
    v = inputs.users_rect(2, 2000, 16, (1.0, 10.0), (-7.5, 7.5))
    assert v[..., 0].min() >= 1.0 and v[..., 0].max() <= 10.0
    assert v[..., 1].min() >= -7.5 and v[..., 1].max() <= 7.5


def test_workload_scalars():
    wl = inputs.HEADLINE
    assert math.isclose(wl.wavelength, 299_792_458.0 / 100e9) and math.isclose(wl.spacing, wl.wavelength / 2)
    assert (wl.n_ant, wl.k, wl.trials, wl.seed) == (16384, 32, 10_000, 3)
    p = wl.power(5)
    assert p.shape == (5, 32) and np.allclose(p, 10.0)  # 10 dB received SNR
    assert np.array_equal(wl.noise(5), np.ones(5))
    assert inputs.SMALL_FP64.scheme == 0 and inputs.HEADLINE.scheme == 1


def test_ragged_instances_recipe():
    n, k, scheme, snr = inputs.ragged_instances(4, 1 << 14)
    assert n.dtype == np.int64 and k.dtype == np.int32
    assert n.min() >= 2 ** 10 and n.max() <= 2 ** 17
    assert k.min() == 2 and k.max() == 64  # both ends of U{2..64} occur at this count
    counts = np.bincount(k, minlength=65)[2:]
    assert counts.min() > 0.7 * counts.mean()  # every user count about equally often
    assert set(np.unique(scheme)) == {0, 1} and abs(scheme.mean() - 0.5) < 0.02
    assert snr.min() >= 0.0 and snr.max() <= 30.0
    # log-uniform N: the median near 2^13.5
    assert abs(np.log2(np.median(n)) - 13.5) < 0.1
    n2, k2, _, _ = inputs.ragged_instances(4, 100)
    assert np.array_equal(n2, n[:100]) and np.array_equal(k2, k[:100])


def test_mlp_init_layout_matches_header():
    text = open(os.path.join(ROOT, "include", "xlmimo.h")).read()
    nparams = int(re.search(r"#define\s+XLMIMO_MLP_PARAMS\s+(\d+)", text).group(1))
    p = inputs.mlp_init_params(1)
    assert p.dtype == np.float32 and p.size == nparams
    off = 0
    for a, b in zip((6, 256, 256, 256, 256), (256, 256, 256, 256, 2)):
        W = p[off:off + a * b]
        bias = p[off + a * b:off + a * b + b]
        assert np.abs(W).max() <= 1.0 / math.sqrt(a) and np.abs(W).max() > 0.9 / math.sqrt(a)
        assert not bias.any()
        off += a * b + b
    assert off == nparams
    assert np.array_equal(p, inputs.mlp_init_params(1))


def test_surrogate_trials_bands():
    n, freq, users = inputs.surrogate_trials(5, 400, 8)
    assert n.min() >= 2 ** 10 and n.max() <= 2 ** 18
    assert set(np.unique(freq)) == {28e9, 100e9}
    r = np.hypot(users[..., 0], users[..., 1])
    lo = np.where(freq == 28e9, 5.0, 3.0)[:, None]
    hi = np.where(freq == 28e9, 50.0, 30.0)[:, None]
    assert (r >= lo - 1e-12).all() and (r <= hi + 1e-12).all()


@pytest.mark.parametrize("name", ["SMALL_FP64", "HEADLINE", "SWEEP", "SURROGATE"])
def test_workloads_draw_in_front_of_the_array(name):
    wl = getattr(inputs, name)
    u = wl.users(64)
    assert u.shape == (64, wl.k, 2) and (u[..., 0] > 0).all()
