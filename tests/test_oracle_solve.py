"""Pins of the oracle's receivers, rates and capacity: textbook formulas via
NumPy/LAPACK, SINRs recomputed from explicit receive vectors, special cases
(diagonal Gram, one user), the capacity identities and the Appendix A bounds."""
import numpy as np
import pytest

from paper_2503_18118_gb300 import inputs

LAM = inputs.wavelength(28e9)


def _case(orc, seed=5, B=6, K=5, N=64, model=1):
    users = inputs.users_polar(seed, B, K, (5.0, 50.0))
    G = orc.gram(model, N, LAM, LAM / 2, 1.0, users)
    g = np.random.Generator(np.random.Philox(key=seed + 100))
    p = 10 ** g.uniform(-0.5, 2.0, (B, K)) / np.real(np.einsum("bii->bi", G))
    s2 = g.uniform(0.5, 2.0, B)
    return users, G, p, s2


def test_zf_mmse_mrc_textbook(orc):
    """Matched receivers against the textbook closed forms computed with
    numpy.linalg: ZF p_k / (s2 [G^-1]_kk); MMSE 1 / [(I + s2^-1 P^1/2 G P^1/2)^-1]_kk - 1;
    MRC p_k G_kk^2 / (sum_{j!=k} p_j |G_kj|^2 + s2 G_kk)."""
    _, G, p, s2 = _case(orc)
    B, K = p.shape
    zf, st, _ = orc.beamform(G, p, s2, orc.ZF)
    mm, _, _ = orc.beamform(G, p, s2, orc.MMSE)
    mr, _, _ = orc.beamform(G, p, s2, orc.MRC)
    assert (st == 0).all()
    for b in range(B):
        Gi = np.linalg.inv(G[b])
        ref_zf = p[b] / (s2[b] * np.real(np.diag(Gi)))
        Ph = np.diag(np.sqrt(p[b]))
        A = np.eye(K) + Ph @ G[b] @ Ph / s2[b]
        ref_mm = 1.0 / np.real(np.diag(np.linalg.inv(A))) - 1.0
        gd = np.real(np.diag(G[b]))
        itf = (np.abs(G[b]) ** 2 * p[b][None, :]).sum(1) - p[b] * gd ** 2
        ref_mr = p[b] * gd ** 2 / (itf + s2[b] * gd)
        assert np.allclose(zf[b], ref_zf, rtol=1e-9)
        assert np.allclose(mm[b], ref_mm, rtol=1e-9)
        assert np.allclose(mr[b], ref_mr, rtol=1e-12)


def test_sinr_from_explicit_receive_vectors(orc):
    """Mismatched receiver (built from the closed-form Gram, judged on the true
    channel) against SINRs computed from explicit receive vectors
    w_k = column k of H M^H and explicit channel vectors h_j."""
    users = inputs.users_polar(3, 2, 4, (5.0, 50.0))
    N = 96
    B, K = users.shape[:2]
    G = orc.gram(orc.FSPL, N, LAM, LAM / 2, 1.0, users)
    Gc = orc.closed_form(orc.FSPL, N, LAM, LAM / 2, 1.0, users)
    p = np.full((B, K), 3.0) / np.real(np.einsum("bii->bi", G)).mean()
    s2 = np.array([0.7, 1.3])
    for scheme in (orc.ZF, orc.MMSE, orc.MRC):
        sinr, st, _ = orc.beamform(Gc, p, s2, scheme, gram_true=G)
        assert (st == 0).all()
        for b in range(B):
            H = np.stack([orc.channel(orc.FSPL, N, LAM, LAM / 2, 1.0, *users[b, k]) for k in range(K)], 1)
            if scheme == orc.ZF:
                M = np.linalg.inv(Gc[b])
            elif scheme == orc.MMSE:
                M = np.linalg.inv(Gc[b] + s2[b] * np.diag(1.0 / p[b]))
            else:
                M = np.eye(K)
            W = H @ M.conj().T
            for k in range(K):
                w = W[:, k]
                gains = np.abs(w.conj() @ H) ** 2
                ref = p[b, k] * gains[k] / ((p[b] * gains).sum() - p[b, k] * gains[k] + s2[b] * np.vdot(w, w).real)
                assert abs(sinr[b, k] - ref) <= 1e-9 * ref


def test_diagonal_gram_and_single_user(orc):
    """Orthogonal users: every receiver gives p_k G_kk / s2.  One user: same."""
    d = np.array([[2.0, 0.5, 3.0]])
    G = np.zeros((1, 3, 3), complex)
    G[0][np.diag_indices(3)] = d[0]
    p = np.array([[1.0, 4.0, 0.25]])
    for scheme in (0, 1, 2):
        s, st, _ = orc.beamform(G, p, 0.5, scheme)
        assert np.allclose(s, p * d / 0.5, rtol=1e-14)
    G1 = np.array([[[7.5 + 0j]]])
    for scheme in (0, 1, 2):
        s, _, _ = orc.beamform(G1, np.array([[2.0]]), 3.0, scheme)
        assert abs(s[0, 0] - 5.0) < 1e-14


def test_two_users_closed_form(orc):
    """K = 2 ZF: [G^-1]_11 = G_22 / det G, so SINR_1 = p_1 det(G) / (s2 G_22)."""
    G = np.array([[[3.0, 1.0 - 0.5j], [1.0 + 0.5j, 2.0]]])
    det = 3.0 * 2.0 - abs(1.0 - 0.5j) ** 2
    s, _, _ = orc.beamform(G, np.array([[1.5, 0.5]]), 0.25, orc.ZF)
    assert np.allclose(s[0], [1.5 * det / (0.25 * 2.0), 0.5 * det / (0.25 * 3.0)], rtol=1e-14)


def test_rx_snr_power_mode(orc):
    """power_mode 1 sets p_k = snr_k s2 / G_kk from the true Gram diagonal."""
    _, G, _, s2 = _case(orc)
    snr = np.full(G.shape[:2], 10.0)
    p = snr * s2[:, None] / np.real(np.einsum("bii->bi", G))
    a, _, ca = orc.beamform(G, snr, s2, orc.MMSE, orc.POWER_RXSNR, want_capacity=True)
    b_, _, cb = orc.beamform(G, p, s2, orc.MMSE, orc.POWER_ABS, want_capacity=True)
    assert np.allclose(a, b_, rtol=1e-13) and np.allclose(ca, cb, rtol=1e-13)


def test_capacity_identities_and_ordering(orc):
    """Eq. (9) with per-user powers: equals the eigenvalue sum and LAPACK's
    log-determinant; ordering R_ZF <= R_MMSE <= C <= log2 U (Hadamard) and
    log2 L <= C (Appendix A lower bound with det R)."""
    _, G, p, s2 = _case(orc, K=6, N=48)
    B, K = p.shape
    _, _, cap = orc.beamform(G, p, s2, orc.MMSE, want_capacity=True)
    rz, _ = orc.sumrate(orc.beamform(G, p, s2, orc.ZF)[0])
    rm, _ = orc.sumrate(orc.beamform(G, p, s2, orc.MMSE)[0])
    for b in range(B):
        Ph = np.diag(np.sqrt(p[b]))
        S = Ph @ G[b] @ Ph / s2[b]
        ev = np.linalg.eigvalsh(S)
        c_eig = np.log2(1.0 + ev).sum()
        sign, ld = np.linalg.slogdet(np.eye(K) + S)
        assert abs(cap[b] - c_eig) < 1e-10 * abs(c_eig) + 1e-12
        assert abs(cap[b] - ld / np.log(2)) < 1e-10 * abs(c_eig) + 1e-12
        a = np.real(np.diag(S))
        logU = np.log2(1 + a).sum()
        d = np.sqrt(np.real(np.diag(G[b])))
        R = G[b] / np.outer(d, d)
        logL = np.linalg.slogdet(R)[1] / np.log(2) + logU
        assert rz[b] <= rm[b] + 1e-9
        assert rm[b] <= cap[b] + 1e-9
        assert cap[b] <= logU + 1e-9
        assert logL <= cap[b] + 1e-9


def test_mmse_rate_equals_capacity(orc):
    """The MMSE-SIC identity: sum_k log2(1 + SINR_k^MMSE) <= C with equality
    only with SIC; for a diagonal Gram all three coincide."""
    G = np.zeros((1, 4, 4), complex)
    G[0][np.diag_indices(4)] = [1.0, 2.0, 0.5, 4.0]
    p = np.ones((1, 4))
    s, _, cap = orc.beamform(G, p, 1.0, orc.MMSE, want_capacity=True)
    r, _ = orc.sumrate(s)
    assert abs(r[0] - cap[0]) < 1e-13


def test_singular_receiver_flagged(orc):
    """A rank-deficient Gram (two users with one channel) gives status 4 for ZF."""
    G = np.array([[[1.0, 1.0], [1.0, 1.0]]], complex)
    s, st, _ = orc.beamform(G, np.ones((1, 2)), 1.0, orc.ZF)
    assert st[0] == 4 and (s == 0).all()
    s, st, _ = orc.beamform(G, np.ones((1, 2)), 1.0, orc.MMSE)
    assert st[0] == 0 and np.isfinite(s).all()


def test_sumrate_stats(orc):
    g = np.random.Generator(np.random.Philox(key=9))
    sinr = g.uniform(0, 50, (37, 7))
    rate, st = orc.sumrate(sinr)
    assert np.allclose(rate, np.log2(1 + sinr).sum(1), rtol=1e-14)
    assert abs(st[0] - rate.mean()) < 1e-12 and abs(st[1] - rate.var() * 37) < 1e-9 and st[2] == 37


@pytest.mark.parametrize("t", [0.5, 0.9])
def test_per_trial_saturation(orc, t):
    """Eqs. (13)-(16) on a hand-made case: one user spans 2 a x; two users take
    the outer bounds."""
    a = t / np.sqrt(1 - t * t)
    users = np.array([[[2.0, 1.0], [2.0, 1.0]], [[1.0, 0.0], [3.0, -4.0]]])
    out = orc.saturation(users, t, 0.01)
    assert np.allclose(out[0, :2], [2 * a + 1, -2 * a + 1])
    assert np.allclose(out[1, :2], [max(a, 3 * a - 4), min(-a, -3 * a - 4)])
    assert out[0, 2] == np.ceil((4 * a) / 0.01)


@pytest.mark.parametrize("closed", [False, True])
def test_downlink_zf_from_explicit_precoder(orc, closed):
    """Downlink ZF (scheme ZF_DL): the SINR from an explicit precoder W = beta H Gf^-1
    with ||W||_F^2 = P_T and the users' explicit channel vectors, built from the
    exact Gram or from the closed form (modified ZF) and judged on the exact channel."""
    B, K, N = 4, 5, 256
    users = inputs.users_polar(31, B, K, (5.0, 50.0))
    G = orc.gram(1, N, LAM, LAM / 2, 1.0, users)
    Gf = orc.closed_form(1, N, LAM, LAM / 2, 1.0, users) if closed else G
    g = np.random.Generator(np.random.Philox(key=77))
    p = 10 ** g.uniform(-6.0, -4.0, (B, K))
    s2 = g.uniform(0.5, 2.0, B)
    s, st, _ = orc.beamform(Gf, p, s2, orc.ZF_DL, 0, gram_true=G)
    for b in range(B):
        H = np.stack([orc.channel(1, N, LAM, LAM / 2, 1.0, *users[b, k]) for k in range(K)], axis=1)
        W = H @ np.linalg.inv(Gf[b])
        W *= np.sqrt(p[b].sum() / np.sum(np.abs(W) ** 2))
        E = H.conj().T @ W  # E[k, j]: what user k receives of stream j
        sig = np.abs(np.diag(E)) ** 2
        itf = np.sum(np.abs(E) ** 2, axis=1) - sig
        ref = sig / (itf + s2[b])
        if st[b] == 0:
            assert np.allclose(s[b], ref, rtol=1e-8)
    if not closed:
        tr = np.real(np.trace(np.linalg.inv(G), axis1=1, axis2=2))
        assert np.allclose(s, (p.sum(1) / (s2 * tr))[:, None], rtol=1e-10)  # all users equal
