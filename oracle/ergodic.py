"""Ergodic capacity-saturation point, plain FP64 with SciPy (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
module.  It shares nothing with the CUDA library.

Sec. IV-A gives the per-user saturation coordinates
    y_up^i = x_i t / sqrt(1 - t^2) + y_i,   y_down^i = -x_i t / sqrt(1 - t^2) + y_i
and, for several users, y_up = max_i y_up^i, y_down = min_i y_down^i (Eqs. 15-16).
Sec. IV-B gives E[y_up] in closed form (Eq. 17) for users uniform on a
rectangle, and Appendix B defines it as E[y_up] = int y dF_z(y)^K with z the
per-user coordinate.  The antenna count that spans [E[y_down], E[y_up]] is
the aperture divided by the element spacing (Sec. IV-C).

Readings taken where the paper is garbled:
  * Eq. (17), fourth term: the factor "(2N+1)" uses an undefined N; it is
    read as (2K+1).  With that reading Eq. (17) equals the Appendix B
    integral (the tests check this to 1e-9 relative).
  * Appendix B writes z = x t/(1-t^2) + y without the square root; the
    coordinate of Sec. IV-A, x t / sqrt(1-t^2) + y, is used.
  * For users drawn in polar coordinates (distance r, angle theta from
    broadside, x = r cos theta, y = r sin theta) the rectangle formula does not
    apply; the Appendix B definition E[y_up] = int y d(F_z^K) is evaluated with
    F_z obtained by integrating the uniform (r, theta) density.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, special


def slope(t: float) -> float:
    """a = t / sqrt(1 - t^2), the factor multiplying x_i in Eqs. (13)-(16)."""
    return t / math.sqrt(1.0 - t * t)


def single_user_min_antennas(x: float, t: float, wavelength: float) -> float:
    """Sec. IV-A: a user at (x, 0) saturates once M >= 4 x t / (lambda sqrt(1-t^2))."""
    return 4.0 * x * t / (wavelength * math.sqrt(1.0 - t * t))


def rect_corners(x_min, x_max, y_min, y_max, t):
    """L1, R1, L2, R2 of Sec. IV-B (below Eq. 17)."""
    a = slope(t)
    L1 = a * x_min + y_min
    R1 = min(a * x_min + y_max, a * x_max + y_min)
    L2 = max(a * x_min + y_max, a * x_max + y_min)
    R2 = a * x_max + y_max
    return L1, R1, L2, R2


def expected_y_up_eq17(x_min, x_max, y_min, y_max, t, K):
    """Eq. (17), fourth term read with (2K+1)."""
    L1, R1, L2, R2 = rect_corners(x_min, x_max, y_min, y_max, t)
    q = (L2 - 2.0 * R1 + R2) / (2.0 * (R2 - R1))
    s = (R1 - L1) / (2.0 * (R2 - R1))
    inc_beta = special.betainc(1.5, K, s) * special.beta(1.5, K)  # B(s; 3/2, K), not regularised
    return (R2
            - q ** K * (L2 - 2.0 * R1 + R2) / (2.0 * (K + 1))
            - q ** K * (R1 - L1)
            - s ** K * (R1 - L1) / (2.0 * (K + 1) * (2 * K + 1))
            - math.sqrt(2.0) * K * math.sqrt((R1 - L1) * (R2 - R1)) * inc_beta)


def expected_y_down_eq18(x_min, x_max, y_min, y_max, t, K):
    """Eq. (18): E[y_down] = y_min + y_max - E[y_up]."""
    return y_min + y_max - expected_y_up_eq17(x_min, x_max, y_min, y_max, t, K)


def rect_pdf_appendix_b(z, x_min, x_max, y_min, y_max, t):
    """Trapezoidal density of z_i (Appendix B, first display)."""
    L1, R1, L2, R2 = rect_corners(x_min, x_max, y_min, y_max, t)
    D1 = L2 - R1 + R2 - L1
    D2 = R1 - L1
    if L1 <= z < R1:
        return 2.0 / D1 / D2 * (z - L1)
    if R1 <= z < L2:
        return 2.0 / D1
    if L2 <= z <= R2:
        return (R2 - z) * 2.0 / D1 / D2
    return 0.0


def rect_cdf_appendix_b(z, x_min, x_max, y_min, y_max, t):
    """CDF of z_i (Appendix B, second display)."""
    L1, R1, L2, R2 = rect_corners(x_min, x_max, y_min, y_max, t)
    D1 = L2 - R1 + R2 - L1
    D2 = R1 - L1
    if z < L1:
        return 0.0
    if z < R1:
        return (z - L1) ** 2 / (D1 * D2)
    if z < L2:
        return (R1 - L1) / D1 + 2.0 / D1 * (z - R1)
    if z < R2:
        return 1.0 - (z - R2) ** 2 / (D1 * D2)
    return 1.0


def expected_y_up_appendix_b(x_min, x_max, y_min, y_max, t, K):
    """Appendix B: E[y_up] = int_{L1}^{R2} y K F_z(y)^{K-1} f_z(y) dy."""
    L1, R1, L2, R2 = rect_corners(x_min, x_max, y_min, y_max, t)

    def integrand(y):
        F = rect_cdf_appendix_b(y, x_min, x_max, y_min, y_max, t)
        return y * K * F ** (K - 1) * rect_pdf_appendix_b(y, x_min, x_max, y_min, y_max, t)

    total = 0.0
    for lo, hi in ((L1, R1), (R1, L2), (L2, R2)):
        if hi > lo:
            v, _ = integrate.quad(integrand, lo, hi, epsabs=0.0, epsrel=1e-13, limit=400)
            total += v
    return total


def rect_cdf_direct(z, x_min, x_max, y_min, y_max, t):
    """P(a x + y <= z) for x ~ U[x_min, x_max], y ~ U[y_min, y_max], by
    integrating the product density directly (no use of the trapezoid form)."""
    a = slope(t)
    dy = y_max - y_min

    def cond(x):
        return min(1.0, max(0.0, (z - a * x - y_min) / dy))

    kinks = sorted(v for v in ((z - y_min) / a, (z - y_max) / a) if x_min < v < x_max)
    v, _ = integrate.quad(cond, x_min, x_max, points=kinks or None, epsabs=0.0, epsrel=1e-13, limit=400)
    return v / (x_max - x_min)


def polar_cdf(z, r_min, r_max, th_min, th_max, t, sign=+1.0):
    """P(a x + sign*y <= z) for r ~ U[r_min, r_max], theta ~ U[th_min, th_max]
    (radians), x = r cos theta, y = r sin theta; by integrating the uniform
    (r, theta) density over theta with the r-conditional probability inside."""
    a = slope(t)
    dr = r_max - r_min

    def cond(th):
        c = a * math.cos(th) + sign * math.sin(th)
        if c > 0.0:
            return min(1.0, max(0.0, (z / c - r_min) / dr))
        if c < 0.0:
            return min(1.0, max(0.0, (r_max - z / c) / dr))
        return 1.0 if z >= 0.0 else 0.0

    # the conditional probability has kinks where z / c(theta) hits r_min or r_max
    pts = []
    amp = math.hypot(a, 1.0)
    phi = math.atan2(sign * 1.0, a)  # c(theta) = amp * cos(theta - phi)
    for rr in (r_min, r_max):
        v = z / (rr * amp)
        if -1.0 <= v <= 1.0:
            base = math.acos(v)
            for cand in (phi + base, phi - base):
                for k in (-1, 0, 1):
                    th = cand + 2.0 * math.pi * k
                    if th_min < th < th_max:
                        pts.append(th)
    v, _ = integrate.quad(cond, th_min, th_max, points=sorted(pts) or None, epsabs=0.0,
                          epsrel=1e-13, limit=400)
    return v / (th_max - th_min)


def _polar_support(r_min, r_max, th_min, th_max, t, sign):
    a = slope(t)
    ths = np.linspace(th_min, th_max, 20001)
    c = a * np.cos(ths) + sign * np.sin(ths)
    vals = np.concatenate([r_min * c, r_max * c])
    lo, hi = float(vals.min()), float(vals.max())
    pad = 1e-9 * max(1.0, abs(lo), abs(hi))
    return lo - pad, hi + pad


def expected_max_polar(r_min, r_max, th_min, th_max, t, K, sign=+1.0):
    """E[max_k (a x_k + sign*y_k)] for K i.i.d. polar users:
    int z d(F^K) = z_hi - int_{z_lo}^{z_hi} F(z)^K dz (integration by parts
    of the Appendix B definition, F from polar_cdf)."""
    lo, hi = _polar_support(r_min, r_max, th_min, th_max, t, sign)
    f = lambda z: polar_cdf(z, r_min, r_max, th_min, th_max, t, sign) ** K
    v, _ = integrate.quad(f, lo, hi, epsabs=0.0, epsrel=1e-12, limit=800)
    return hi - v


def expected_interval_polar(r_min, r_max, th_min, th_max, t, K):
    """(E[y_up], E[y_down]) for polar users.  y_down = min_k(-a x_k + y_k)
    = -max_k(a x_k - y_k)."""
    up = expected_max_polar(r_min, r_max, th_min, th_max, t, K, +1.0)
    dn = -expected_max_polar(r_min, r_max, th_min, th_max, t, K, -1.0)
    return up, dn


def saturation_antennas(up, down, spacing):
    """Number of elements spanning [E[y_down], E[y_up]] (Sec. IV-C), as the
    real ratio and its ceiling."""
    v = (up - down) / spacing
    return v, int(math.ceil(v))
