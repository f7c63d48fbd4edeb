"""Pins of oracle/bounds.py (Appendix A): the 2x2 determinant written out,
the paper's inequalities (Hadamard, Schur-Horn / Schur convexity), exactly
orthogonal users where both bounds are tight, one user, and the eigenvalue
route to the empirical expectation of Fig. 5."""
import math

import numpy as np
import pytest

from oracle import bounds
from paper_2503_18118_gb300 import inputs

LAM100 = inputs.wavelength(100e9)


def _sec5a(orc, seed, B, K, N, model=0):
    # Sec. V-A geometry: x ~ U[1, 10] m, y ~ U[-7.5, 7.5] m, 100 GHz, half-wavelength ULA
    users = inputs.users_rect(seed, B, K, (1.0, 10.0), (-7.5, 7.5))
    return orc.gram(model, N, LAM100, LAM100 / 2, 1.0, users)


def test_two_users_closed_form(orc):
    """det R = 1 - |r|^2 and det(I + diag(a)^1/2 R diag(a)^1/2) =
    (1 + a1)(1 + a2) - a1 a2 |r|^2, with r from the Gram entries."""
    G = _sec5a(orc, 1, 8, 2, 300)
    a = np.array([0.5, 7.0])
    out = bounds.bounds(G, a)
    r2 = np.abs(G[:, 0, 1]) ** 2 / (np.real(G[:, 0, 0]) * np.real(G[:, 1, 1]))
    assert np.allclose(out[:, 0], np.log2(1.0 - r2), rtol=1e-12, atol=1e-13)
    assert np.allclose(out[:, 1], np.log2((1 + a[0]) * (1 + a[1]) - a[0] * a[1] * r2), rtol=1e-12)
    assert np.allclose(out[:, 2], math.log2(1.5) + math.log2(8.0))
    assert np.allclose(out[:, 3], out[:, 0] + out[:, 2])


@pytest.mark.parametrize("K,N", [(6, 64), (20, 512), (40, 2048)])
def test_hadamard_and_schur_horn(orc, K, N):
    """Appendix A: log2 L <= C <= log2 U and log2 det R <= 0; with lambda_i the
    eigenvalues of P^1/2 R P^1/2, sum log2(1 + 1/a_i) <= sum log2(1 + 1/lambda_i)."""
    G = _sec5a(orc, 10 + K, 5, K, N)
    g = np.random.Generator(np.random.Philox(key=K))
    a = 10 ** g.uniform(0.0, 3.0, (5, K))  # receive SNR 0..30 dB
    out = bounds.bounds(G, a)
    assert np.all(out[:, 0] <= 1e-12)
    assert np.all(out[:, 3] <= out[:, 1] + 1e-9)
    assert np.all(out[:, 1] <= out[:, 2] + 1e-9)
    R = bounds.correlation(G)
    s = np.sqrt(a)
    lam = np.linalg.eigvalsh(s[:, :, None] * R * s[:, None, :])
    assert np.all(np.sum(np.log2(1 + 1 / a), axis=1) <= np.sum(np.log2(1 + 1 / lam), axis=1) + 1e-9)


def test_orthogonal_users_make_both_bounds_tight(orc):
    """Far-field (UPW) users whose steering vectors are DFT columns of the
    half-wavelength ULA (sin theta_k = 2k/N) are exactly orthogonal: R = I,
    log2 det R = 0 and C = log2 U = log2 L."""
    N, K = 64, 8
    th = np.arcsin(2.0 * np.arange(-K // 2, K // 2) / N)
    users = np.stack([40.0 * np.cos(th), 40.0 * np.sin(th)], axis=-1)[None]
    G = orc.gram(2, N, LAM100, LAM100 / 2, 1.0, users)
    out = bounds.bounds(G, 3.0)
    assert abs(out[0, 0]) < 1e-10
    assert abs(out[0, 1] - K * 2.0) < 1e-10  # log2(1 + 3) = 2 per user
    assert abs(out[0, 3] - out[0, 2]) < 1e-10
    assert abs(bounds.neg_expectation(G)[0]) < 1e-11


def test_single_user(orc):
    G = _sec5a(orc, 3, 4, 1, 100)
    out = bounds.bounds(G, 2.0)
    assert np.allclose(out[:, 0], 0.0, atol=1e-15)
    assert np.allclose(out[:, 1], math.log2(3.0), rtol=1e-14)


def test_expectation_from_eigenvalues(orc):
    """-E_K[log2 lambda^R] from LAPACK's eigenvalues of R (eigvalsh) equals the
    log-determinant route (slogdet), and lies in [0, inf)."""
    G = _sec5a(orc, 7, 6, 24, 700)
    lam = np.linalg.eigvalsh(bounds.correlation(G))
    e_eig = -np.mean(np.log2(lam), axis=1)
    e = bounds.neg_expectation(G)
    assert np.allclose(e, e_eig, rtol=1e-10, atol=1e-13)
    assert np.all(e >= -1e-14)


def test_amplitude_scale_invariance(orc):
    """R, and with it every quantity of Appendix A at given receive SNRs, is
    invariant under a common amplitude (beta0) and under any per-user scaling
    of the channel vectors."""
    users = inputs.users_rect(9, 3, 10, (1.0, 10.0), (-7.5, 7.5))
    G1 = orc.gram(0, 400, LAM100, LAM100 / 2, 1.0, users)
    G2 = orc.gram(0, 400, LAM100, LAM100 / 2, 37.0, users)
    d = np.exp(np.linspace(-2, 2, 10))
    G3 = G1 * d[None, :, None] * d[None, None, :]
    for Gx in (G2, G3):
        assert np.allclose(bounds.bounds(Gx, 1.0), bounds.bounds(G1, 1.0), rtol=1e-11, atol=1e-12)
