"""URA Gram on the GPU (xlmimo_channel_gram_ura) against the oracle's plain
3-D definition on the same seeded users.

Tolerances are those of the ULA Gram at each precision (the URA is a sum of
per-row ULA Grams of moved users): normwise max_ij |dG_ij| / sqrt(G_ii G_jj)
<= 1e-5 (FP32), 2e-5 (BF16x3 and FP16x3), and for FP64 the rounding
bound of the phase, 8 eps (1 + 2 pi r_max / lambda), averaged over the
N * rows independent element errors of the spherical models (not for the
planar wave, whose distance to the array centre is common to all elements).
"""
import math

import numpy as np
import pytest

from paper_2503_18118_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LAM100 = inputs.wavelength(100e9)
TOL = {1: 1e-5, 3: 2e-5, 4: 2e-5}


@pytest.fixture(scope="module")
def xl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_18118_gb300 import xlmimo
    xlmimo.lib()
    return xlmimo


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def normwise(G, Gref):
    d = np.sqrt(np.abs(np.einsum("...ii->...i", Gref)))
    return float(np.max(np.abs(G - Gref) / (d[..., :, None] * d[..., None, :])))


def f64_tol(users, N, R, model):
    d = LAM100 / 2
    rmax = float(np.sqrt(users[..., 0] ** 2 + (np.abs(users[..., 1]) + N * d / 2) ** 2 + (R * d / 2) ** 2).max())
    avg = 1.0 if model == 2 else math.sqrt(N * R)
    return max(1e-12, 8 * np.finfo(float).eps * (1 + 2 * math.pi * rmax / LAM100) / avg)


# rows of a multiple of 128 elements take the tensor-core Gram's URA mode at
# BF16 hi/lo (one trial: element chunks that cross rows)
CASES = [(64, 2, 4, 3), (100, 5, 8, 2), (257, 8, 33, 2), (64, 64, 64, 1), (1000, 3, 32, 2),
         (128, 4, 8, 3), (256, 7, 32, 2), (128, 33, 64, 2), (384, 2, 33, 3), (1024, 64, 16, 1),
         (1, 3, 1, 2), (128, 5, 1, 2)]


@pytest.mark.parametrize("model", [0, 1, 2])
@pytest.mark.parametrize("N,R,K,B", CASES)
@pytest.mark.parametrize("prec", [0, 1, 3, 4])
def test_gram_ura_matches_oracle(xl, orc, prec, model, N, R, K, B):
    users = inputs.users_rect(N + R + K, B, K, (0.5, 3.0), (-1.5, 1.5))
    G = xl.xlmimo_channel_gram_ura(xl.array(N, LAM100, model=model), R, dev(users), prec).cpu().numpy()
    ref = orc.gram_ura(model, N, R, LAM100, LAM100 / 2, 1.0, users)
    tol = f64_tol(users, N, R, model) if prec == 0 else TOL[prec]
    assert normwise(G, ref) <= tol
    assert np.allclose(G, np.conj(np.swapaxes(G, 1, 2)), rtol=0, atol=0)


@pytest.mark.parametrize("prec", [0, 1, 3])
def test_one_row_is_the_ula_call(xl, prec):
    users = dev(inputs.users_rect(7, 4, 8, (0.5, 3.0), (-1.5, 1.5)))
    arr = xl.array(500, LAM100, model=0)
    G1 = xl.xlmimo_channel_gram_ura(arr, 1, users, prec)
    G0 = xl.xlmimo_channel_gram(arr, users, prec)
    assert torch.equal(G1, G0)


def test_workspace_chunks(xl, orc):
    """Enough rows that the 1 GiB workspace holds fewer trials than the batch
    (K = 64, 512 row pairs: 34 MB a trial, at most 31 trials a chunk, 19 after
    rounding to whole waves of 152 x 2 Gram CTAs); trials on both sides of
    those boundaries and the last one against the oracle."""
    N, R, K, B = 16, 1024, 64, 40
    users = inputs.users_rect(99, B, K, (0.5, 3.0), (-1.5, 1.5))
    G = xl.xlmimo_channel_gram_ura(xl.array(N, LAM100, model=0), R, dev(users), 1).cpu().numpy()
    for b in (0, 18, 19, 30, 31, 37, 38, 39):
        ref = orc.gram_ura(0, N, R, LAM100, LAM100 / 2, 1.0, users[b:b + 1])
        assert normwise(G[b:b + 1], ref) <= 1e-5


def test_invalid_user_gives_nan(xl):
    users = inputs.users_rect(5, 3, 4, (0.5, 3.0), (-1.5, 1.5))
    users[1, 2, 0] = -1.0
    G = xl.xlmimo_channel_gram_ura(xl.array(64, LAM100, model=0), 4, dev(users), 1).cpu().numpy()
    assert np.all(np.isnan(G[1]))
    assert np.all(np.isfinite(G[0])) and np.all(np.isfinite(G[2]))


def test_ura_receivers_end_to_end(xl, orc):
    """URA Gram (FP32) -> ZF and MMSE receivers -> sum rate, against the
    oracle's URA Gram through the oracle's receivers: sum rate relative
    <= 1e-4, the end-to-end bound of the FP32 ULA path."""
    N, R, K, B = 128, 16, 8, 6
    users = inputs.users_rect(12, B, K, (0.5, 3.0), (-1.5, 1.5))
    p = np.full((B, K), 100.0)
    s2 = np.ones(B)
    G = xl.xlmimo_channel_gram_ura(xl.array(N, LAM100, model=0), R, dev(users), 1)
    Gr = orc.gram_ura(0, N, R, LAM100, LAM100 / 2, 1.0, users)
    for scheme in (xl.ZF, xl.MMSE):
        s, st, _ = xl.xlmimo_beamform(G, dev(p), dev(s2), scheme, xl.POWER_RXSNR)
        s_ref, st_ref, _ = orc.beamform(Gr, p, s2, scheme, orc.POWER_RXSNR)
        assert np.all(st_ref == 0) and np.all(np.isin(st.cpu().numpy(), [0, 1]))
        r = np.sum(np.log2(1 + s.cpu().numpy()), axis=1)
        r_ref = np.sum(np.log2(1 + s_ref), axis=1)
        assert np.max(np.abs(r - r_ref) / r_ref) <= 1e-4


def test_empty_batch(xl):
    users = torch.empty((0, 4, 2), dtype=torch.float64, device="cuda")
    G = xl.xlmimo_channel_gram_ura(xl.array(128, LAM100, model=0), 3, users, xl.BF16X3)
    assert G.shape == (0, 4, 4)
