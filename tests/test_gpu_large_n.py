"""Exact Gram matrices of an array longer than 2^31 elements (element indices
past 32 bits), where the oracle's explicit sums would take hours: checked
against closed forms that hold at any N.

* Free-space spherical wave, diagonal: with element n at n d - c from the
  user's projection (c = y + (N-1) d / 2) and x the user's distance to the
  array axis,
      G_kk = (lambda / 4 pi)^2 / d^2 * sum_{n=0}^{N-1} 1 / ((n - p)^2 + q^2),
  p = c / d, q = x / d.  Each half of the sum (elements on either side of the
  user) is a difference of digamma values:
      sum_{k=0}^{M-1} 1 / ((k + s)^2 + q^2) = Im[psi(s - i q + M) - psi(s - i q)] / q,
  from 1 / ((k + s)^2 + q^2) = Im[1 / (k + s - i q)] / q and
  sum_{k=0}^{M-1} 1 / (k + z) = psi(z + M) - psi(z).  Users sit beside
  element 2^31 + 2^20, so every element that carries their power has an
  index beyond 2^31.
* Planar wave: the whole Gram is the Dirichlet kernel of the angular offset
  (the oracle's closed form, pinned against its explicit sums at small N).
"""
import math

import numpy as np
import pytest

from paper_2503_18118_gb300 import inputs

torch = pytest.importorskip("torch")
special = pytest.importorskip("scipy.special")

LAM = inputs.wavelength(100e9)
D = LAM / 2
N_BIG = 2 ** 31 + 2 ** 21


@pytest.fixture(scope="module")
def xl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_18118_gb300 import xlmimo
    xlmimo.lib()
    return xlmimo


def half_sum(s, q, M):
    """sum_{k=0}^{M-1} 1 / ((k + s)^2 + q^2), s > 0, by the digamma difference."""
    z = complex(s, -q)
    return float((special.psi(z + M) - special.psi(z)).imag) / q


def fspl_diagonal(x, y, N, lam, d):
    c = y + (N - 1) * d / 2
    p, q = c / d, x / d
    n0 = int(math.floor(p))
    assert 0 <= n0 < N - 1 and p > n0  # the user's projection lies between two elements
    right = half_sum(n0 + 1 - p, q, N - n0 - 1)  # elements n0 + 1 .. N - 1
    left = half_sum(p - n0, q, n0 + 1)  # elements n0 .. 0
    return (lam / (4 * math.pi)) ** 2 / d ** 2 * (right + left)


def users_past_2_31():
    """Four users beside elements 2^31 + 2^20 + offset, at 3.3 to 17 m from the array."""
    xs = np.array([3.3, 17.0, 4.2, 9.0])
    n = 2 ** 31 + 2 ** 20 + np.array([0.37, 0.81, 1000.25, -2500.5])
    ys = (n - (N_BIG - 1) / 2) * D
    return np.stack([xs, ys], -1)[None]


def test_digamma_half_sum_matches_direct_sum():
    """The closed form of the half sums against the plain sum where that is
    cheap (M well above q, as on the large array: no cancellation between the
    two digamma values)."""
    for s, q, M in ((0.37, 1100.0, 50000), (0.81, 3.5, 100000), (0.25, 2000.0, 400000), (0.63, 6000.0, 3000000)):
        k = np.arange(M)
        direct = float(np.sum(1.0 / ((k + s) ** 2 + q ** 2)))
        assert abs(half_sum(s, q, M) - direct) <= 1e-13 * direct, (s, q, M)


# Recursive FP64 summation of n positive terms errs by at most (n - 1) 2^-53
# of their sum; n <= N whatever the element split, and each term carries a
# few roundings of its own.  A wrong element index instead moves the entries
# by O(1).
SUM_TOL_F64 = 4 * N_BIG * 2.0 ** -53


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol", [(0, SUM_TOL_F64), (3, 2e-5)])
def test_fspl_diagonal_past_2_31_elements(xl, prec, tol):
    """FP64 SIMT and BF16 hi/lo tensor-core Gram of one trial on 2^31 + 2^21
    elements: the diagonal against the digamma closed form (FP64: the
    recursive-summation bound; BF16 hi/lo: its tensor-core class, the
    periodic drain keeping the accumulation error flat in N); the matrix
    Hermitian with |G_ij|^2 <= G_ii G_jj."""
    u = users_past_2_31()
    arr = xl.array(N_BIG, LAM, D, 1.0, xl.FSPL_USW)
    G = xl.xlmimo_channel_gram(arr, torch.from_numpy(u).cuda(), prec).cpu().numpy()[0]
    want = np.array([fspl_diagonal(x, y, N_BIG, LAM, D) for x, y in u[0]])
    diag = np.real(np.diag(G))
    assert np.all(np.abs(diag - want) <= tol * want), (diag, want)
    assert np.all(np.imag(np.diag(G)) == 0)
    assert np.array_equal(G, G.conj().T)
    assert np.all(np.abs(G) ** 2 <= np.outer(diag, diag) * (1 + 1e-9))


def users_near_broadside_offsets():
    """Four users whose sin(theta) differ by 0.6 / N to 3.1 / N: the Dirichlet
    kernel D_N(v), v = d (sin theta_j - sin theta_i) / lambda, is then of
    order N, so each off-diagonal entry is a coherent sum over the whole array
    and depends on every element's position."""
    s = math.sin(0.3) + np.array([0.0, 0.6, 1.7, 3.1]) / N_BIG
    r = np.array([5.0, 12.0, 20.0, 7.0])
    return np.stack([r * np.sqrt(1 - s * s), r * s], -1)[None]


@pytest.mark.gpu
def test_planar_wave_gram_past_2_31_elements(xl, orc):
    """FP64 Gram of the planar-wave model on 2^31 + 2^21 elements against the
    exact Dirichlet-kernel form, within the FP64 rounding of the largest
    element phase (elements reach ~1.6e6 m from the centre); the users'
    off-diagonal entries are a sizeable fraction of the diagonal."""
    u = users_near_broadside_offsets()
    arr = xl.array(N_BIG, LAM, D, 1.0, xl.UPW)
    G = xl.xlmimo_channel_gram(arr, torch.from_numpy(u).cuda(), 0).cpu().numpy()
    R = orc.closed_form(orc.UPW, N_BIG, LAM, D, 1.0, u)
    rr = np.hypot(u[0, :, 0], u[0, :, 1])
    assert np.min(np.abs(R[0]) * np.outer(rr, rr)) > 0.1 * N_BIG  # every entry a coherent sum
    rmax = float(np.hypot(u[..., 0], u[..., 1]).max()) + N_BIG * D / 2
    tol = 8 * np.finfo(float).eps * (1.0 + 2 * math.pi * rmax / LAM) + SUM_TOL_F64
    d = np.sqrt(np.abs(np.einsum("...ii->...i", R)))
    err = float(np.max(np.abs(G - R) / (d[..., :, None] * d[..., None, :])))
    assert err <= tol, (err, tol)
    assert np.allclose(np.real(np.einsum("...ii->...i", G)), N_BIG / np.hypot(u[..., 0], u[..., 1]) ** 2,
                       rtol=SUM_TOL_F64, atol=0)


def test_closed_forms_match_oracle_sums_at_moderate_n(orc):
    """The two expected values the large-array tests use, against the oracle's
    explicit inner products where those are cheap (N = 100,001): the digamma
    diagonal for users placed the same way (beside an element, 3.3 to 17 m from
    the array), and the Dirichlet form for users whose sin(theta) differ by
    fractions of 1/N (every entry a coherent sum)."""
    n = 100_001
    xs = np.array([3.3, 17.0, 4.2, 9.0])
    idx = 70_000 + np.array([0.37, 0.81, 1000.25, -2500.5])
    u = np.stack([xs, (idx - (n - 1) / 2) * D], -1)[None]
    G = orc.gram(orc.FSPL, n, LAM, D, 1.0, u)[0]
    want = np.array([fspl_diagonal(x, y, n, LAM, D) for x, y in u[0]])
    assert np.allclose(np.real(np.diag(G)), want, rtol=1e-12, atol=0)
    s = math.sin(0.3) + np.array([0.0, 0.6, 1.7, 3.1]) / n
    r = np.array([5.0, 12.0, 20.0, 7.0])
    v = np.stack([r * np.sqrt(1 - s * s), r * s], -1)[None]
    Gp = orc.gram(orc.UPW, n, LAM, D, 1.0, v)
    Rp = orc.closed_form(orc.UPW, n, LAM, D, 1.0, v)
    assert np.min(np.abs(Rp[0]) * np.outer(r, r)) > 0.1 * n
    d = np.sqrt(np.abs(np.einsum("...ii->...i", Rp)))
    rmax = float(r.max()) + n * D / 2
    assert float(np.max(np.abs(Gp - Rp) / (d[..., :, None] * d[..., None, :]))) <= \
        8 * np.finfo(float).eps * (1.0 + 2 * math.pi * rmax / LAM) + 4 * n * 2.0 ** -53
