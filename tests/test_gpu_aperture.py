"""The aperture-aware closed form on the GPU against oracle/aperture.py.

Tolerance: the closed form's own FP32 trigonometry (2e-6 of |G~_ij|) plus the
FP32 Fresnel series of the factor (~1e-5).  Pairs whose mask decision or
Fresnel cut sits within rounding of its threshold (| |y*| - H | < 1e-9 H,
| |u| - 2 | < 1e-3) may fall on either side in the two precisions and are
left out of the element-wise comparison (a handful at most)."""
import math

import numpy as np
import pytest
import torch

from oracle import aperture as ap
from paper_2503_18118_gb300 import inputs
from paper_2503_18118_gb300 import xlmimo as X

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def borderline(users, n, lam):
    B, K, _ = users.shape
    H = 0.5 * n * lam / 2
    out = []
    for b in range(B):
        for i in range(K):
            for j in range(i + 1, K):
                ys, p2 = ap.stationary(*users[b, i], *users[b, j], lam)
                bad = math.isfinite(ys) and abs(abs(ys) - H) < 1e-9 * H
                if math.isfinite(ys) and p2 != 0.0:
                    sc = math.sqrt(abs(p2) / math.pi)
                    for e in (H, -H):
                        bad |= abs(abs((e - ys) * sc) - ap.U_CUT) < 1e-3
                out.append(bad)
    return np.array(out)


CASES = [
    (100e9, 16384, 16, 20, (3.0, 30.0), 31),
    (100e9, 1024, 8, 30, (3.0, 30.0), 32),
    (28e9, 2048, 12, 25, (5.0, 50.0), 33),
    (28e9, 262144, 6, 5, (5.0, 50.0), 34),
]


@pytest.mark.parametrize("f,n,K,B,r,seed", CASES)
@pytest.mark.parametrize("mode", [X.APERTURE_MASK, X.APERTURE_FRESNEL])
def test_closed_form_aperture_matches_oracle(orc, f, n, K, B, r, seed, mode):
    lam = inputs.wavelength(f)
    users = inputs.users_polar(seed, B, K, r)
    arr = X.array(n, lam)
    got = X.xlmimo_corr_closed_form_aperture(arr, dev(users), mode).cpu().numpy()
    Gc = orc.closed_form(orc.FSPL, n, lam, lam / 2, 1.0, users)
    F = ap.factors(mode, users, n, lam, lam / 2)
    want = ap.apply(Gc, F)
    iu = np.triu_indices(K, 1)
    keep = ~borderline(users, n, lam).reshape(B, -1)
    assert keep.mean() > 0.95
    g, w, c = got[:, iu[0], iu[1]], want[:, iu[0], iu[1]], Gc[:, iu[0], iu[1]]
    err = np.abs(g - w)[keep]
    assert np.all(err <= 3e-5 * np.abs(c)[keep]), float(np.max(err / np.abs(c)[keep]))
    assert np.allclose(np.diagonal(got, axis1=1, axis2=2), np.diagonal(Gc, axis1=1, axis2=2), rtol=1e-9, atol=0)
    assert np.array_equal(got, np.conj(np.transpose(got, (0, 2, 1))))
    if mode == X.APERTURE_MASK:  # entries are the closed form or exactly zero
        zero = np.abs(w) == 0
        assert np.all(g[zero & keep] == 0)


def test_aperture_closed_form_is_closer_to_exact_at_moderate_n():
    """At N = 4096 (100 GHz) most stationary points lie outside the aperture;
    both corrections must reduce the normwise error against the exact Gram."""
    lam = inputs.wavelength(100e9)
    users = dev(inputs.users_polar(35, 40, 16, (3.0, 30.0)))
    arr = X.array(4096, lam)
    G = X.xlmimo_channel_gram(arr, users, X.F64)
    d = torch.sqrt(torch.diagonal(G, dim1=1, dim2=2).real)
    nrm = d[:, :, None] * d[:, None, :]

    def err(Gh):
        return float(((Gh - G).abs() / nrm).max())

    e_cf = err(X.xlmimo_corr_closed_form(arr, users))
    e_m = err(X.xlmimo_corr_closed_form_aperture(arr, users, X.APERTURE_MASK))
    e_f = err(X.xlmimo_corr_closed_form_aperture(arr, users, X.APERTURE_FRESNEL))
    assert e_m < 0.5 * e_cf and e_f < 0.5 * e_cf, (e_cf, e_m, e_f)
