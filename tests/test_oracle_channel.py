"""Pins of the oracle's channel, Gram and closed-form Gram against things
other than itself: 50-digit brute force, amplitude identities, the exact
Dirichlet kernel of the planar-wave model, the closed forms of Eqs. (4)-(8)
and their limits."""
import math

import numpy as np
import pytest

from paper_2503_18118_gb300 import inputs

LAM100 = inputs.wavelength(100e9)
LAM28 = inputs.wavelength(28e9)


def phase_tol(rmax, lam):
    """FP64 bound for quantities that carry a phase 2 pi r / lambda: a few ulps
    of the phase magnitude, the dominant rounding error of every entry."""
    return 8 * np.finfo(float).eps * (1.0 + 2 * math.pi * rmax / lam)


def normwise(G, Gref):
    d = np.sqrt(np.abs(np.einsum("...ii->...i", Gref)))
    return float(np.max(np.abs(G - Gref) / (d[..., :, None] * d[..., None, :])))


def test_brute_force_mpmath(orc):
    """Tiny case (N <= 16, K = 3) in 50-digit arithmetic: channel entries and
    Gram entries match to FP64 rounding."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    users = np.array([[[2.0, 0.3], [3.5, -1.25], [1.2, 0.9]]])
    lam, N = LAM28, 13
    sp = lam / 2
    # FP64 evaluates the phase 2 pi r / lambda (about 10^3 rad here) with an
    # absolute error of a few ulps of its magnitude; that bounds the relative
    # error of every entry and, summed, of every normalised Gram entry.
    rmax = float(np.hypot(users[0, :, 0], np.abs(users[0, :, 1]) + N * sp).max())
    tol = phase_tol(rmax, lam)
    for model in (orc.PNUSW, orc.FSPL, orc.UPW):
        G = orc.gram(model, N, lam, sp, 1.0, users)[0]
        H = []
        for (x, y) in users[0]:
            x, y = mp.mpf(x), mp.mpf(y)
            col = []
            for n in range(N):
                yn = (mp.mpf(n) - mp.mpf(N - 1) / 2) * mp.mpf(sp)
                if model == orc.UPW:
                    r0 = mp.sqrt(x * x + y * y)
                    path = r0 - yn * y / r0
                    v = mp.exp(-2j * mp.pi * path / mp.mpf(lam)) / r0
                else:
                    r = mp.sqrt(x * x + (yn - y) ** 2)
                    ph = mp.exp(-2j * mp.pi * r / mp.mpf(lam))
                    v = ph / r * mp.sqrt(x / r) if model == orc.PNUSW else mp.mpf(lam) / (4 * mp.pi * r) * ph
                col.append(v)
            H.append(col)
        h0 = orc.channel(model, N, lam, sp, 1.0, float(users[0, 0, 0]), float(users[0, 0, 1]))
        for n in range(N):
            assert abs(complex(H[0][n]) - h0[n]) <= tol * abs(complex(H[0][n]))
        Gm = np.array([[complex(mp.fsum(mp.conj(H[i][n]) * H[j][n] for n in range(N))) for j in range(3)]
                       for i in range(3)])
        assert normwise(G, Gm) < tol


@pytest.mark.parametrize("model", [0, 1, 2])
def test_gram_structure(orc, model):
    """Hermitian, positive semidefinite, |rho_ij| <= 1, diagonal equal to the
    sum of squared amplitudes (PNUSW: beta0 x / r^3; free space:
    (lambda/4pi)^2 / r^2; UPW: N beta0 / r0^2)."""
    users = inputs.users_polar(7, 4, 5, (5.0, 50.0))
    N, lam = 300, LAM28
    sp = lam / 2
    beta0 = 1.7
    G = orc.gram(model, N, lam, sp, beta0, users)
    assert np.allclose(G, np.conj(np.swapaxes(G, 1, 2)), rtol=0, atol=1e-15 * np.abs(G).max())
    for b in range(G.shape[0]):
        ev = np.linalg.eigvalsh(G[b])
        assert ev.min() > -1e-12 * ev.max()
        d = np.sqrt(np.real(np.diag(G[b])))
        rho = np.abs(G[b]) / np.outer(d, d)
        assert rho.max() <= 1.0 + 1e-12
    yn = (np.arange(N) - (N - 1) / 2) * sp
    x = users[..., 0][..., None]
    y = users[..., 1][..., None]
    r2 = x ** 2 + (yn - y) ** 2
    if model == 0:
        diag = beta0 * (x / r2 ** 1.5).sum(-1)
    elif model == 1:
        diag = ((lam / (4 * math.pi)) ** 2 / r2).sum(-1)
    else:
        diag = N * beta0 / (x[..., 0] ** 2 + y[..., 0] ** 2)
    assert np.allclose(np.real(np.einsum("bii->bi", G)), diag, rtol=1e-13, atol=0)


def test_upw_equals_dirichlet(orc):
    """Planar-wave model: the explicit inner products equal the exact
    Dirichlet-kernel closed form (pins element positions, conjugation and the
    phase sign)."""
    users = inputs.users_polar(11, 3, 6, (5.0, 50.0))
    for N in (1, 2, 17, 256):
        G = orc.gram(orc.UPW, N, LAM100, LAM100 / 2, 1.0, users)
        Gc = orc.closed_form(orc.UPW, N, LAM100, LAM100 / 2, 1.0, users)
        rmax = float(np.hypot(users[..., 0], users[..., 1]).max()) + N * LAM100 / 4
        assert normwise(Gc, G) <= phase_tol(rmax, LAM100)


def test_far_field_limit(orc):
    """Far beyond the Rayleigh distance 2 D^2 / lambda the spherical-wave
    correlation approaches the planar-wave (Dirichlet) correlation."""
    N, lam = 16, LAM28
    D = N * lam / 2
    rayl = 2 * D * D / lam
    th = np.deg2rad(np.array([10.0, -25.0]))
    r = 4000.0 * rayl
    users = np.stack([r * np.cos(th), r * np.sin(th)], -1)[None]
    Gs = orc.gram(orc.FSPL, N, lam, lam / 2, 1.0, users)[0]
    Gp = orc.gram(orc.UPW, N, lam, lam / 2, 1.0, users)[0]
    rs = Gs[0, 1] / np.sqrt(Gs[0, 0].real * Gs[1, 1].real)
    rp = Gp[0, 1] / np.sqrt(Gp[0, 0].real * Gp[1, 1].real)
    assert abs(rs - rp) < 1e-3


def test_power_closed_form_eq4_and_limit_eq5(orc):
    """Eq. (4) approximates the exact received power (Riemann-sum error,
    shrinking with N) and tends to Eq. (5), 4 beta0 / (lambda x)."""
    users = np.array([[[1.5, 0.0], [3.0, 1.2], [6.0, -2.0]]])
    lam = LAM100
    errs = []
    for N in (1024, 8192, 65536):
        G = orc.gram(orc.PNUSW, N, lam, lam / 2, 1.0, users)[0]
        Gc = orc.closed_form(orc.PNUSW, N, lam, lam / 2, 1.0, users)[0]
        errs.append(np.max(np.abs(np.diag(G).real - np.diag(Gc).real) / np.diag(G).real))
    assert errs[-1] < 1e-6 and errs[0] < 1e-4
    Gc = orc.closed_form(orc.PNUSW, 2 ** 40, lam, lam / 2, 1.0, users)[0]
    assert np.allclose(np.diag(Gc).real, 4.0 / (lam * users[0, :, 0]), rtol=1e-9)


def test_single_user_saturation_bound(orc):
    """Sec. IV-A: at y = 0 the power ratio P/P_lim of Eq. (4) reaches t exactly
    at M = 4 x t / (lambda sqrt(1 - t^2)); below it the ratio is smaller."""
    from oracle import ergodic
    lam, t, x = LAM100, 0.9, 1.5
    M = ergodic.single_user_min_antennas(x, t, lam)
    users = np.array([[[x, 0.0]]])
    lim = 4.0 / (lam * x)
    hi = orc.closed_form(orc.PNUSW, int(math.ceil(M)), lam, lam / 2, 1.0, users)[0, 0, 0].real / lim
    lo = orc.closed_form(orc.PNUSW, int(math.floor(M)), lam, lam / 2, 1.0, users)[0, 0, 0].real / lim
    assert lo < t <= hi
    assert hi - t < 1e-4


def test_correlation_closed_form_eq6(orc):
    """Eq. (6) (stationary phase) matches the exact off-diagonal Gram entry once
    the stationary point lies inside the aperture; its magnitude and phase both
    converge (a conjugation or sign error fails this)."""
    users = np.array([[[3.0, 0.5], [5.0, -1.0], [4.0, 2.0]]])
    lam = LAM100
    prev = None
    for N in (16384, 65536):
        G = orc.gram(orc.PNUSW, N, lam, lam / 2, 1.0, users)
        Gc = orc.closed_form(orc.PNUSW, N, lam, lam / 2, 1.0, users)
        e = normwise(Gc, G)
        if prev is not None:
            assert e < prev
        prev = e
    assert prev < 1e-4
    Gf = orc.gram(orc.FSPL, 65536, lam, lam / 2, 1.0, users)
    Gcf = orc.closed_form(orc.FSPL, 65536, lam, lam / 2, 1.0, users)
    assert normwise(Gcf, Gf) < 5e-3


def test_correlation_n_independent_and_limit_eq8(orc):
    """The closed-form off-diagonal G~(i,j) = rho_ij sqrt(P_i P_j) / P does not
    depend on N, and rho_ij tends to Eq. (8): sqrt(lambda)|cos gamma| / (2 sqrt(d))."""
    users = np.array([[[3.0, 0.5], [5.0, -1.0]]])
    lam = LAM100
    vals = [orc.closed_form(orc.PNUSW, N, lam, lam / 2, 1.0, users)[0, 0, 1] for N in (64, 4096, 1 << 20)]
    assert np.allclose(vals, vals[0], rtol=1e-12, atol=0)
    Gc = orc.closed_form(orc.PNUSW, 1 << 50, lam, lam / 2, 1.0, users)[0]
    rho = Gc[0, 1] / np.sqrt(Gc[0, 0].real * Gc[1, 1].real)
    dx, dy = 3.0 - 5.0, 0.5 - (-1.0)
    d = math.hypot(dx, dy)
    lim = math.sqrt(lam) * abs(dx) / d / (2 * math.sqrt(d))
    assert abs(abs(rho) - lim) < 1e-9 * lim
    phase = -1.0 * (2 * math.pi * d / lam - math.pi / 4)  # sgn(3 - 5) = -1, Eq. (7)
    assert abs(np.angle(rho * np.exp(-1j * phase))) < 1e-9
