"""Pins of the oracle's ergodic saturation point: Eq. (17) against the
Appendix B integral, the trapezoid CDF against direct integration of the
user density, K = 1 and K -> infinity limits (Eqs. 19-20), Monte Carlo
agreement, and the paper's printed order of magnitude for Fig. 4."""
import json
import math
import os

import numpy as np
import pytest

from paper_2503_18118_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
PAPER = json.load(open(os.path.join(HERE, "golden", "paper_values.json")))
T = PAPER["saturation_threshold_t"]["value"]


@pytest.fixture(scope="module")
def erg():
    from oracle import ergodic
    return ergodic


SETTINGS = [((1.0, 10.0), (-7.5, 7.5), 100), ((1.0, 2.0), (-7.5, 7.5), 10),
            ((1.0, 10.0), (-7.5, 7.5), 1), ((2.0, 3.0), (0.0, 20.0), 8), ((5.0, 9.0), (-1.0, 1.0), 3)]


@pytest.mark.parametrize("xr,yr,K", SETTINGS)
def test_eq17_equals_appendix_b_integral(erg, xr, yr, K):
    a = erg.expected_y_up_eq17(*xr, *yr, T, K)
    b = erg.expected_y_up_appendix_b(*xr, *yr, T, K)
    assert abs(a - b) <= 1e-9 * abs(b) + 1e-12


def test_garbled_factor_matters(erg):
    """The (2N+1) factor of Eq. (17) cannot be dropped: without it the formula
    misses the Appendix B value by far more than quadrature error."""
    xr, yr, K = (1.0, 10.0), (-7.5, 7.5), 3
    L1, R1, L2, R2 = erg.rect_corners(*xr, *yr, T)
    s = (R1 - L1) / (2 * (R2 - R1))
    with_factor = s ** K * (R1 - L1) / (2 * (K + 1) * (2 * K + 1))
    without = s ** K * (R1 - L1) / (2 * (K + 1))
    b = erg.expected_y_up_appendix_b(*xr, *yr, T, K)
    a = erg.expected_y_up_eq17(*xr, *yr, T, K)
    assert abs((a + with_factor - without) - b) > 1e3 * abs(a - b) + 1e-10


@pytest.mark.parametrize("z", [1.0, 3.7, 9.0, 14.5, 20.0, 24.0])
def test_trapezoid_cdf_equals_direct(erg, z):
    xr, yr = (1.0, 10.0), (-7.5, 7.5)
    assert abs(erg.rect_cdf_appendix_b(z, *xr, *yr, T) - erg.rect_cdf_direct(z, *xr, *yr, T)) < 1e-11


def test_single_user_mean(erg):
    """K = 1: E[z] = a E[x] + E[y]."""
    a = erg.slope(T)
    for xr, yr in (((1.0, 10.0), (-7.5, 7.5)), ((2.0, 3.0), (0.0, 20.0))):
        ref = a * sum(xr) / 2 + sum(yr) / 2
        assert abs(erg.expected_y_up_eq17(*xr, *yr, T, 1) - ref) < 1e-12 * abs(ref) + 1e-12


def test_limits_eq19_eq20_and_monotone(erg):
    """E[y_up] increases with K towards R2 (Eq. 19); E[y_down] towards
    y_min - a x_max (Eq. 20)."""
    xr, yr = (1.0, 10.0), (-7.5, 7.5)
    L1, R1, L2, R2 = erg.rect_corners(*xr, *yr, T)
    vals = [erg.expected_y_up_eq17(*xr, *yr, T, K) for K in (1, 2, 5, 20, 100, 1000, 100000)]
    assert all(b > a for a, b in zip(vals, vals[1:]))
    # the gap to the corner point decays like the Appendix C bound, K^{-1/2}
    K = 100000
    bound = math.sqrt(2) * math.sqrt((R1 - L1) * (R2 - R1)) * math.gamma(1.5) * K ** -0.5
    assert 0 < R2 - vals[-1] <= 1.05 * bound
    dn = erg.expected_y_down_eq18(*xr, *yr, T, K)
    assert 0 < dn - (yr[0] - erg.slope(T) * xr[1]) <= 1.05 * bound


def test_beta_term_decay_appendix_c(erg):
    """Appendix C: the incomplete-beta term is below
    sqrt(2) sqrt((R1-L1)(R2-R1)) Gamma(3/2) K^{-1/2} asymptotically and decays."""
    from scipy import special
    xr, yr = (1.0, 10.0), (-7.5, 7.5)
    L1, R1, L2, R2 = erg.rect_corners(*xr, *yr, T)
    s = (R1 - L1) / (2 * (R2 - R1))
    prev = None
    for K in (10, 100, 1000, 10000):
        term = math.sqrt(2) * K * math.sqrt((R1 - L1) * (R2 - R1)) * special.betainc(1.5, K, s) * special.beta(1.5, K)
        bound = math.sqrt(2) * math.sqrt((R1 - L1) * (R2 - R1)) * special.gamma(1.5) * K ** -0.5
        assert term <= bound * 1.05
        if prev is not None:
            assert term < prev
        prev = term


def test_monte_carlo_rect(orc, erg):
    """Per-trial y_up / y_down of Eqs. (15)-(16) averaged over 2e5 trials agree
    with Eqs. (17)-(18) within 5 standard errors."""
    xr, yr, K = (1.0, 2.0), (-7.5, 7.5), 10
    users = inputs.users_rect(21, 200_000, K, xr, yr)
    sat = orc.saturation(users, T, 1.0)
    up, dn = sat[:, 0], sat[:, 1]
    e_up = erg.expected_y_up_eq17(*xr, *yr, T, K)
    e_dn = erg.expected_y_down_eq18(*xr, *yr, T, K)
    se = up.std() / math.sqrt(len(up))
    assert abs(up.mean() - e_up) < 5 * se
    assert abs(dn.mean() - e_dn) < 5 * dn.std() / math.sqrt(len(dn))


def test_monte_carlo_polar(orc, erg):
    """Polar users (the Monte-Carlo workloads' distribution): the Appendix B
    definition evaluated by quadrature agrees with Monte Carlo, and the
    polar CDF agrees with the empirical CDF."""
    K = 8
    users = inputs.users_polar(22, 100_000, K, (5.0, 50.0))
    sat = orc.saturation(users, T, 1.0)
    up, dn = erg.expected_interval_polar(5.0, 50.0, math.radians(-60), math.radians(60), T, K)
    assert abs(sat[:, 0].mean() - up) < 5 * sat[:, 0].std() / math.sqrt(len(sat))
    assert abs(sat[:, 1].mean() - dn) < 5 * sat[:, 1].std() / math.sqrt(len(sat))
    a = erg.slope(T)
    z = a * users[..., 0].ravel() + users[..., 1].ravel()
    for q in (10.0, 30.0, 60.0):
        emp = (z <= q).mean()
        assert abs(emp - erg.polar_cdf(q, 5.0, 50.0, math.radians(-60), math.radians(60), T)) < 5e-3


def test_polar_matches_rect_when_degenerate(erg):
    """A thin annular sector around broadside is nearly a rectangle: both
    routes agree to the shape error."""
    r0, r1, th = 4.0, 6.0, math.radians(0.5)
    up_p, _ = erg.expected_interval_polar(r0, r1, -th, th, T, 5)
    up_r = erg.expected_y_up_eq17(r0, r1, -r0 * math.sin(th), r0 * math.sin(th), T, 5)
    assert abs(up_p - up_r) < 2e-2


def test_fig4_saturation_order_of_magnitude(erg):
    """Sec. V-C prints "around 10^4 antennas" for the Fig. 4 setting; the
    analytic count 2 (E[y_up] - E[y_down]) / lambda must be of that order."""
    s = PAPER["fig4_setting"]
    lam = inputs.wavelength(s["freq_hz"])
    up = erg.expected_y_up_eq17(*s["x_range_m"], *s["y_range_m"], T, s["K"])
    dn = erg.expected_y_down_eq18(*s["x_range_m"], *s["y_range_m"], T, s["K"])
    v, n = erg.saturation_antennas(up, dn, lam / 2)
    order = PAPER["fig4_saturation_antennas_order"]["value"]
    assert order / 2 <= n <= order * 2
    assert n == math.ceil(v)
