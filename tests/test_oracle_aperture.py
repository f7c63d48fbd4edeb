"""Pins of the aperture-aware closed form (oracle/aperture.py): the
stationary point and the phase curvature against the exact pair phase
(finite differences), the Fresnel factor against direct quadrature of the
quadratic phase, its limits, and its effect against the exact Gram."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import aperture as ap

LAM = 0.0107069


def phase(y, xi, yi, xj, yj):
    return 2 * math.pi / LAM * (math.hypot(xi, y - yi) - math.hypot(xj, y - yj))


def test_stationary_point_and_curvature_by_finite_differences():
    xi, yi, xj, yj = 4.0, 1.0, 9.0, 6.0   # line y = x - 3 meets the axis at y = -3
    ys, p2 = ap.stationary(xi, yi, xj, yj, LAM)
    assert abs(ys + 3.0) < 1e-12
    h = 1e-4
    d1 = (phase(ys + h, xi, yi, xj, yj) - phase(ys - h, xi, yi, xj, yj)) / (2 * h)
    d2 = (phase(ys + h, xi, yi, xj, yj) - 2 * phase(ys, xi, yi, xj, yj) + phase(ys - h, xi, yi, xj, yj)) / h ** 2
    assert abs(d1) < 1e-6 * abs(d2)
    assert abs(d2 - p2) < 1e-4 * abs(p2)
    assert ap.stationary(3.0, 1.0, 3.0, 5.0, LAM)[0] == math.inf


def test_fresnel_factor_equals_quadrature_of_the_quadratic_phase():
    """Inside the cut F is the integral of the quadratic phase over the
    aperture divided by the infinite one.  With the lower edge far (counted at
    its limit, int_{-inf}^0 e^{j s pi t^2/2} dt = (1 + j s)/2) and the upper
    edge at u_hi = (H - y*) sqrt(|phi''|/pi), that is
    F = ((1 + j s)/2 + int_0^{u_hi} e^{j s pi t^2/2} dt) / (1 + j s);
    the finite part is taken by adaptive quadrature, not Fresnel integrals."""
    xi, yi, xj, yj = 4.0, 7.0, 9.0, 12.0   # line y = x + 3: y* = 3
    ys, p2 = ap.stationary(xi, yi, xj, yj, LAM)
    assert abs(ys - 3.0) < 1e-12
    sc = math.sqrt(abs(p2) / math.pi)
    sg = math.copysign(1.0, p2)
    checked = 0
    for u_hi in (-1.9, -0.6, -0.2, 0.0, 0.3, 1.5, 1.99):
        H = ys + u_hi / sc
        n = 2 * H / (LAM / 2)
        assert (-H - ys) * sc < -ap.U_CUT   # the lower edge is beyond the cut
        re = integrate.quad(lambda t: math.cos(math.pi * t * t / 2), 0.0, u_hi, epsabs=1e-14)[0]
        im = integrate.quad(lambda t: sg * math.sin(math.pi * t * t / 2), 0.0, u_hi, epsabs=1e-14)[0]
        want = ((1 + 1j * sg) / 2 + re + 1j * im) / (1 + 1j * sg)
        got = ap.factor(ap.FRESNEL, xi, yi, xj, yj, n, LAM, LAM / 2)
        assert abs(got - want) < 1e-10, (u_hi, got, want)
        checked += 1
    assert checked == 7


def test_fresnel_factor_limits():
    xi, yi, xj, yj = 4.0, 1.0, 9.0, 6.0
    ys, p2 = ap.stationary(xi, yi, xj, yj, LAM)
    # stationary point exactly on the upper edge, lower edge far: one half
    H = abs(ys)
    n = 2 * H / (LAM / 2)
    # here ys = -3 < 0, so the lower edge -H coincides with ys
    assert abs(ap.factor(ap.FRESNEL, xi, yi, xj, yj, n, LAM, LAM / 2) - 0.5) < 1e-12
    # both edges far: one;  stationary point far outside: zero
    assert ap.factor(ap.FRESNEL, xi, yi, xj, yj, 1e6, LAM, LAM / 2) == 1.0
    assert ap.factor(ap.FRESNEL, xi, yi, xj, yj, 100, LAM, LAM / 2) == 0.0
    assert ap.factor(ap.MASK, xi, yi, xj, yj, 1e6, LAM, LAM / 2) == 1.0
    assert ap.factor(ap.MASK, xi, yi, xj, yj, 100, LAM, LAM / 2) == 0.0
    assert ap.factor(ap.NONE, xi, yi, xj, yj, 100, LAM, LAM / 2) == 1.0


@pytest.mark.parametrize("case", ["edge", "outside"])
def test_factor_moves_the_closed_form_towards_the_exact_gram(orc, case):
    """Exact inner products (oracle Gram) for a pair whose stationary point is
    near an aperture edge, or outside the aperture: the corrected entry is
    closer to the exact one than the paper's closed form."""
    if case == "edge":
        xi, yi, xj, yj = 4.0, 1.0, 9.0, 6.0
        ys, p2 = ap.stationary(xi, yi, xj, yj, LAM)
        N = int(round(2 * abs(ys) / (LAM / 2)))  # edge at the stationary point
        modes = (ap.FRESNEL,)
    else:
        xi, yi, xj, yj = 4.0, 1.0, 5.0, 2.0      # y* = -3, outside an aperture of +-1 m
        N = int(round(2.0 / (LAM / 2)))
        modes = (ap.MASK, ap.FRESNEL)
    users = np.array([[[xi, yi], [xj, yj]]])
    G = orc.gram(orc.FSPL, N, LAM, LAM / 2, 1.0, users)
    Gc = orc.closed_form(orc.FSPL, N, LAM, LAM / 2, 1.0, users)
    for mode in modes:
        F = ap.factors(mode, users, N, LAM, LAM / 2)
        Ga = ap.apply(Gc, F)
        assert abs(Ga[0, 0, 1] - G[0, 0, 1]) < 0.5 * abs(Gc[0, 0, 1] - G[0, 0, 1]), mode
        assert Ga[0, 1, 0] == np.conj(Ga[0, 0, 1])
