"""Aperture-aware closed form (test infrastructure only; not the paper's).

The off-diagonal closed form (Eq. 6, and its free-space analogue) is a
stationary-phase value: it assumes the stationary point of the pair phase
    phi(y) = 2 pi (r_i(y) - r_j(y)) / lambda,   G_ij = sum_n a_n e^{j phi(y_n)},
lies inside the array and that the aperture extends to infinity around it.
The stationary point is where an element sees both users in the same
direction, i.e. where the line through the two users meets the array axis:
    y* = y_i - x_i (y_j - y_i) / (x_j - x_i)
(no stationary point when x_i = x_j).  Over an aperture [-H, H], H = N
spacing / 2, the quadratic approximation phi(y*) + phi''(y*) (y - y*)^2 / 2,
    phi'' = (2 pi / lambda) (x_i^2 / r_i^3 - x_j^2 / r_j^3)  at y*,
integrates to the infinite-aperture value times
    F = [(C(u_hi) - C(u_lo)) + j s (S(u_hi) - S(u_lo))] / (1 + j s),
    u = (edge - y*) sqrt(|phi''| / pi),  s = sign(phi''),
with the Fresnel integrals C(u) + j S(u) = int_0^u e^{j pi t^2 / 2} dt.

Two factors correct the closed form (off-diagonal entries multiplied by F,
the conjugate mirrored, the diagonal untouched):
  MASK    F = 1 if |y*| <= H else 0 (the stationary-phase term is dropped
          when its point lies outside the aperture);
  FRESNEL F as above, except that an edge farther than U_CUT = 2 Fresnel
          lengths counts at its limit C = S = sign(u)/2: beyond the
          transition the quadratic model's oscillating tail has the wrong
          phase (the true phase is not quadratic far from y*), and keeping it
          was measured to double the sum-rate error.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import fresnel

NONE, MASK, FRESNEL = 0, 1, 2
U_CUT = 2.0


def stationary(xi, yi, xj, yj, wavelength):
    """(y*, phi''(y*)) of the pair phase; y* = inf when x_i = x_j."""
    if xj == xi:
        return math.inf, 0.0
    ys = yi - xi * (yj - yi) / (xj - xi)
    ri = math.hypot(xi, ys - yi)
    rj = math.hypot(xj, ys - yj)
    return ys, 2.0 * math.pi / wavelength * (xi * xi / ri ** 3 - xj * xj / rj ** 3)


def _cs(u):
    if abs(u) > U_CUT:
        return math.copysign(0.5, u), math.copysign(0.5, u)
    s, c = fresnel(u)
    return float(c), float(s)


def factor(mode, xi, yi, xj, yj, n_ant, wavelength, spacing):
    """The correction F of one pair (complex)."""
    if mode == NONE:
        return 1.0 + 0.0j
    H = 0.5 * n_ant * spacing
    ys, p2 = stationary(xi, yi, xj, yj, wavelength)
    if mode == MASK:
        return 1.0 + 0.0j if abs(ys) <= H else 0.0j
    if not math.isfinite(ys) or p2 == 0.0:
        return 0.0j
    sc = math.sqrt(abs(p2) / math.pi)
    ch, sh = _cs((H - ys) * sc)
    cl, sl = _cs((-H - ys) * sc)
    sg = 1.0 if p2 > 0 else -1.0
    return ((ch - cl) + 1j * sg * (sh - sl)) / (1.0 + 1j * sg)


def factors(mode, users, n_ant, wavelength, spacing):
    """[B * K(K-1)/2] F of every pair i < j in row order."""
    users = np.asarray(users, np.float64)
    B, K, _ = users.shape
    out = []
    for b in range(B):
        for i in range(K):
            for j in range(i + 1, K):
                out.append(factor(mode, *users[b, i], *users[b, j], n_ant, wavelength, spacing))
    return np.array(out, np.complex128)


def apply(Gc, F):
    """Off-diagonal G~_ij F_ij (rows in pair order), conjugate mirrored."""
    B, K, _ = Gc.shape
    out = Gc.copy()
    q = 0
    for b in range(B):
        for i in range(K):
            for j in range(i + 1, K):
                v = Gc[b, i, j] * F[q]
                out[b, i, j] = v
                out[b, j, i] = np.conj(v)
                q += 1
    return out
