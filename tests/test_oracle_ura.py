"""Pins of the URA Gram of the oracle (the planar array of the footnote of
Sec. II): one row is the ULA of Sec. II-A; the PNUSW received power is the
solid angle of the aperture rectangle (the two-dimensional counterpart of
Eq. (4)) within the midpoint-rule error; the Gram splits into per-row ULA
Grams of users moved to x' = sqrt(x^2 + z^2); the planar wave of a user at
elevation 0 is the same on every row."""
import math

import numpy as np
import pytest

from paper_2503_18118_gb300 import inputs

LAM100 = inputs.wavelength(100e9)


def _users(seed, B, K, xr=(0.5, 3.0), yr=(-1.0, 1.0)):
    return inputs.users_rect(seed, B, K, xr, yr)


@pytest.mark.parametrize("model", [0, 1, 2])
def test_one_row_is_the_ula(orc, model):
    users = _users(1, 3, 5)
    G1 = orc.gram_ura(model, 300, 1, LAM100, LAM100 / 2, 2.0, users)
    G0 = orc.gram(model, 300, LAM100, LAM100 / 2, 2.0, users)
    assert np.array_equal(G1, G0)


def _solid_angle(x, y, N, R, d):
    """Solid angle of the rectangle [-N d/2, N d/2] x [-R d/2, R d/2] of the
    y-z plane seen from (x, y, 0): the double integral of x / r^3, whose
    antiderivative is F(a, b) = atan(a b / (x sqrt(x^2 + a^2 + b^2)))."""
    F = lambda a, b: math.atan(a * b / (x * math.sqrt(x * x + a * a + b * b)))
    a1, a2 = -N * d / 2 - y, N * d / 2 - y
    b1, b2 = -R * d / 2, R * d / 2
    return F(a2, b2) - F(a1, b2) - F(a2, b1) + F(a1, b1)


@pytest.mark.parametrize("N,R", [(256, 64), (64, 256), (200, 33)])
def test_pnusw_power_is_the_solid_angle(orc, N, R):
    """sum_elements x / r^3 is the midpoint rule, cells d x d, for the solid
    angle of the aperture, so G_kk d^2 / beta0 = Omega up to the rule's
    leading error (d^2 / 24) * integral of the Laplacian of x / r^3 over the
    rectangle; the Laplacian is x (9 rho^2 - 6 x^2) / (x^2 + rho^2)^{7/2},
    at most 6 / x^4 in magnitude, so the relative error is below
    (d^2 / 4) (x^2 + rho_max^2)^{3/2} / x^5 (rho_max: the farthest corner)."""
    d = LAM100 / 2
    beta0 = 3.0
    users = _users(10 + R, 2, 6)
    G = orc.gram_ura(0, N, R, LAM100, d, beta0, users)
    for b in range(users.shape[0]):
        for k in range(users.shape[1]):
            x, y = users[b, k]
            om = _solid_angle(x, y, N, R, d)
            rho2 = (N * d / 2 + abs(y)) ** 2 + (R * d / 2) ** 2
            bound = (d * d / 4) * (x * x + rho2) ** 1.5 / x ** 5
            got = np.real(G[b, k, k]) * d * d / beta0
            assert abs(got - om) <= 1.5 * bound * om
            assert abs(np.imag(G[b, k, k])) == 0.0


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("R", [2, 5])
def test_rows_are_ulas_of_moved_users(orc, model, R):
    """Row q (height z_q) sees user (x, y) like a ULA sees (x', y) with
    x' = sqrt(x^2 + z_q^2); the PNUSW amplitude keeps the projection on the
    array normal, sqrt(x / r) = sqrt(x' / r) sqrt(x / x'), so
    G = sum_q diag(w_q) G_ULA(x'_q) diag(w_q), w_q = sqrt(x / x'_q) for PNUSW
    and 1 in free space."""
    N, d = 150, LAM100 / 2
    users = _users(20 + R, 2, 7)
    G = orc.gram_ura(model, N, R, LAM100, d, 1.0, users)
    acc = np.zeros_like(G)
    for q in range(R):
        z = (q - (R - 1) / 2) * d
        moved = users.copy()
        moved[..., 0] = np.sqrt(users[..., 0] ** 2 + z * z)
        w = np.sqrt(users[..., 0] / moved[..., 0]) if model == 0 else np.ones(users.shape[:2])
        acc += w[:, :, None] * orc.gram(model, N, LAM100, d, 1.0, moved) * w[:, None, :]
    dg = np.sqrt(np.real(np.einsum("bii->bi", G)))
    err = np.abs(G - acc) / (dg[:, :, None] * dg[:, None, :])
    # both sides round r to FP64: phase error ~ 8 eps 2 pi r / lambda per element
    assert err.max() <= 8 * np.finfo(float).eps * (1 + 2 * math.pi * 4.0 / LAM100)


def test_planar_wave_is_row_independent(orc):
    users = _users(3, 2, 6, xr=(20.0, 40.0), yr=(-20.0, 20.0))
    G = orc.gram_ura(2, 128, 6, LAM100, LAM100 / 2, 1.0, users)
    G0 = orc.gram(2, 128, LAM100, LAM100 / 2, 1.0, users)
    assert np.allclose(G, 6 * G0, rtol=1e-13, atol=1e-13 * np.abs(G0).max())


def test_hermitian_positive_semidefinite(orc):
    users = _users(4, 2, 12)
    G = orc.gram_ura(0, 64, 16, LAM100, LAM100 / 2, 1.0, users)
    assert np.allclose(G, np.conj(np.swapaxes(G, 1, 2)), rtol=0, atol=0)
    assert np.all(np.linalg.eigvalsh(G) > -1e-12 * np.abs(G).max())
