"""Appendix A on the GPU (xlmimo_capacity_bounds) against the oracle.

Tolerance: the channel entries come from the FP32 generator (phase error
below 1e-5 rad, amplitude to FP32 rounding: 3 eps_h per correlation entry
with eps_h = 1e-5).  They are stored as h = hi + lo in BF16 (unit roundoff
2^-8), so |h - hi - lo| <= 2^-16 |h|, and the Gram drops lo*lo (<= 2^-16 of
|h_i,n||h_j,n|): each product is within 3 * 2^-16 of |h_i,n||h_j,n|, whose sum
is at most |h_i||h_j|.  The tensor cores' FP32 accumulation rounds towards
zero over periods of 48 products-of-16 before round-to-nearest totals:
below 2e-6 of |h_i||h_j|.  So |dR_ij| <= EPS_R = 3 eps_h + 3 * 2^-16 + 2e-6;
the Cholesky factorisations are FP64.  To first order d log det M =
tr(M^-1 dM), so |d log2 det R| <= ||R^-1||_F ||dR||_F / ln 2
<= EPS_R K^1.5 / (lambda_min ln 2), and for M = I + a R the same with
a / (1 + a lambda_min) for 1 / lambda_min; lambda_min is the oracle's.
"""
import math

import numpy as np
import pytest
import torch

from oracle import bounds as obounds
from paper_2503_18118_gb300 import inputs

pytestmark = pytest.mark.gpu

LAM100 = inputs.wavelength(100e9)
EPS_H = 1e-5
EPS_R = 3 * EPS_H + 3 * 2.0 ** -16 + 2e-6


@pytest.fixture(scope="module")
def xl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_18118_gb300 import xlmimo
    xlmimo.lib()
    return xlmimo


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _tols(G, a):
    R = obounds.correlation(G)
    lmin = np.linalg.eigvalsh(R)[:, 0]
    K = R.shape[-1]
    t_r = EPS_R * K ** 1.5 / (lmin * math.log(2)) + 1e-12
    t_c = EPS_R * K ** 1.5 * a / ((1 + a * lmin) * math.log(2)) + 1e-12
    return t_r, t_c


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("K,N,B", [(1, 100, 3), (2, 257, 3), (31, 1000, 2), (33, 4099, 2), (64, 2048, 2),
                                   (100, 3000, 2)])
@pytest.mark.parametrize("snr", [1.0, 1000.0])
def test_bounds_match_oracle(xl, orc, model, K, N, B, snr):
    users = inputs.users_rect(40 + K + N, B, K, (1.0, 10.0), (-7.5, 7.5))
    arr = xl.array(N, LAM100, model=model)
    out = xl.xlmimo_capacity_bounds(arr, dev(users), snr).cpu().numpy()
    G = orc.gram(model, N, LAM100, LAM100 / 2, 1.0, users)
    ref = obounds.bounds(G, snr)
    t_r, t_c = _tols(G, snr)
    assert np.all(np.abs(out[:, 0] - ref[:, 0]) <= t_r)
    assert np.all(np.abs(out[:, 1] - ref[:, 1]) <= t_c)
    assert np.allclose(out[:, 2], ref[:, 2], rtol=1e-14)
    assert np.allclose(out[:, 3], out[:, 0] + out[:, 2], rtol=0, atol=1e-12)


def test_orthogonal_users(xl):
    """DFT-orthogonal far-field users: R = I, both bounds tight."""
    N, K = 64, 8
    th = np.arcsin(2.0 * np.arange(-K // 2, K // 2) / N)
    users = np.stack([40.0 * np.cos(th), 40.0 * np.sin(th)], axis=-1)[None]
    out = xl.xlmimo_capacity_bounds(xl.array(N, LAM100, model=2), dev(users), 3.0).cpu().numpy()
    assert abs(out[0, 0]) < 1e-6 and abs(out[0, 1] - 2.0 * K) < 1e-6


def test_fig5_scale_properties(xl):
    """The Fig. 5 workload at K = 1000 (N = 40000, Sec. V-A rectangle): the
    inequalities of Appendix A hold for every trial, and the negative
    empirical expectation is positive and below 1."""
    users = inputs.users_rect(5, 2, 1000, (1.0, 10.0), (-7.5, 7.5))
    out = xl.xlmimo_capacity_bounds(xl.array(40000, LAM100, model=0), dev(users), 1.0).cpu().numpy()
    assert np.all(np.isfinite(out))
    assert np.all(out[:, 0] < 0)
    assert np.all(out[:, 3] <= out[:, 1] + 1e-6) and np.all(out[:, 1] <= out[:, 2] + 1e-6)
    e = -out[:, 0] / 1000
    assert np.all((e > 0) & (e < 1))


def test_empty_batch_and_errors(xl):
    arr = xl.array(100, LAM100)
    out = xl.xlmimo_capacity_bounds(arr, torch.empty((0, 5, 2), dtype=torch.float64, device="cuda"), 1.0)
    assert out.shape == (0, 4)
    with pytest.raises(RuntimeError):
        xl.xlmimo_capacity_bounds(arr, dev(inputs.users_rect(1, 1, 4, (1.0, 10.0), (-7.5, 7.5))), -1.0)


def test_bounds_timed_matches_untimed(xl):
    """The phase-timed variant gives the same bounds, bit for bit, with five
    positive phase times (the Gram and the Cholesky present at K = 200)."""
    users = inputs.users_rect(33, 2, 200, (1.0, 10.0), (-7.5, 7.5))
    arr = xl.array(3000, LAM100, model=0)
    a = xl.xlmimo_capacity_bounds(arr, dev(users), 1.0).cpu().numpy()
    b, ms = xl.xlmimo_capacity_bounds_timed(arr, dev(users), 1.0)
    assert np.array_equal(a, b.cpu().numpy())
    assert len(ms) == 5 and all(t > 0.0 for t in ms)
    _, ms0 = xl.xlmimo_capacity_bounds_timed(arr, dev(users[:0]), 1.0)
    assert ms0 == [0.0] * 5
