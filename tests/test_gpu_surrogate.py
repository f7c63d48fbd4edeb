"""Parity of the surrogate's kernels with the FP64 oracle (oracle/mlp.py),
and the gain of a network trained on the GPU over the closed form alone.

Tolerances.  The three 256 x 256 layers round their operands to BF16 (ulp
2^-8 relative); an FP32 sum that differs from the FP64 one in the last bits
can round an activation to the neighbouring BF16 value, which moves a
downstream pre-activation by about 2^-8 |h w|.  Such flips are rare (a few
per thousand activations), so the tests bound the typical error tightly
(90th percentile, FP32 level) and the worst case at a few BF16 ulps of the
layer scale.  Inference adds the FP32 hardware tanh in SiLU (relative error
~2^-11, which moves roughly an eighth of the BF16-rounded activations by one
BF16 ulp relative to the oracle's exact SiLU).  Three rounded layers then
carry output errors of a few 2^-8 of the output scale, before the network's
own gain; the inference test bounds the median at 4e-3 and the worst pair at
2e-2 of the output scale."""
import math

import numpy as np
import pytest
import torch

from oracle import mlp
from paper_2503_18118_gb300 import inputs, surrogate
from paper_2503_18118_gb300 import xlmimo as X

pytestmark = pytest.mark.gpu
Q = (1, 2, 3)


def params_np(seed, scale=1.0):
    p = inputs.mlp_init_params(seed)
    if scale != 1.0:
        p = p * np.float32(scale)
    return p


def feats_np(seed, M):
    g = np.random.Generator(np.random.Philox(key=seed))
    return g.uniform(-1.2, 1.2, size=(M, 6)).astype(np.float32)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("M", [1, 63, 300, 4097])
def test_forward_matches_oracle(M):
    p = params_np(11, 2.0)
    x = feats_np(12, M)
    cache = torch.empty((M * X.MLP_CACHE_PER_ROW,), dtype=torch.float32, device="cuda")
    out = X.xlmimo_mlp_forward(dev(p), dev(x), cache=cache).cpu().numpy().astype(np.float64)
    ref, rcache = mlp.forward(mlp.unflatten(p), x.astype(np.float64), qlayers=Q)
    err = np.abs(out - ref)
    scale = max(1.0, float(np.abs(ref).max()))
    assert np.quantile(err, 0.9) <= 1e-5 * scale
    assert err.max() <= 2e-3 * scale
    c = cache.cpu().numpy().reshape(4, 2, M, 256).astype(np.float64)
    for l in range(4):
        h_in, z = rcache[l]
        h_next = rcache[l + 1][0]
        assert np.quantile(np.abs(c[l, 0] - z), 0.9) <= 1e-5 * max(1.0, np.abs(z).max())
        assert np.abs(c[l, 0] - z).max() <= 2e-3 * max(1.0, np.abs(z).max())
        assert np.abs(c[l, 1] - h_next).max() <= 2e-3 * max(1.0, np.abs(h_next).max())


@pytest.mark.parametrize("M,weighted", [(7, False), (1000, True)])
def test_loss_matches_oracle(M, weighted):
    g = np.random.Generator(np.random.Philox(key=M))
    out = g.normal(size=(M, 2)).astype(np.float32)
    tg = g.normal(size=(M, 2)).astype(np.float32)
    w = g.random(M).astype(np.float32) if weighted else None
    dout, loss = X.xlmimo_mlp_loss(dev(out), dev(tg), dev(w) if weighted else None)
    rl, rd = mlp.mse(out.astype(np.float64), tg.astype(np.float64), None if w is None else w.astype(np.float64))
    assert abs(loss.item() - rl) <= 1e-5 * rl
    assert np.allclose(dout.cpu().numpy(), rd, rtol=1e-5, atol=1e-12)


@pytest.mark.parametrize("M", [5, 513, 2048])
def test_backward_matches_oracle(M):
    """Gradients of the whole network against the oracle's (pinned by finite
    differences): per tensor, relative L2 error."""
    p = params_np(21, 2.0)
    x = feats_np(22, M)
    g = np.random.Generator(np.random.Philox(key=23))
    tg = g.normal(scale=0.3, size=(M, 2)).astype(np.float32)
    pd = dev(p)
    cache = torch.empty((M * X.MLP_CACHE_PER_ROW,), dtype=torch.float32, device="cuda")
    out = X.xlmimo_mlp_forward(pd, dev(x), cache=cache)
    dout, _ = X.xlmimo_mlp_loss(out, dev(tg))
    grad = X.xlmimo_mlp_backward(pd, dev(x), cache, dout).cpu().numpy().astype(np.float64)
    P = mlp.unflatten(p)
    ro, rc = mlp.forward(P, x.astype(np.float64), qlayers=Q)
    _, rd = mlp.mse(ro, tg.astype(np.float64))
    rg = mlp.flatten(mlp.backward(P, rc, rd, qlayers=Q))
    o = 0
    for (W, b) in P:
        for n in (W.size, b.size):
            a, r = grad[o:o + n], rg[o:o + n]
            assert np.linalg.norm(a - r) <= 2e-3 * np.linalg.norm(r) + 1e-12, (o, n)
            o += n


def test_adam_matches_oracle():
    """FP32 Adam against the FP64 definition.  Bounds: each FP32 operation
    rounds to 2^-24 relative, so m is good to a few ulps of the sum of the
    magnitudes of its two terms (they may cancel), v (no cancellation) to a
    few ulps of itself, and the step to the propagated error of m plus a few
    ulps of the step and of p."""
    g = np.random.Generator(np.random.Philox(key=31))
    n = X.MLP_PARAMS
    p, gr = g.normal(size=n).astype(np.float32), g.normal(size=n).astype(np.float32)
    m, v = (g.normal(size=n) * 0.1).astype(np.float32), (g.random(n) * 0.01).astype(np.float32)
    pd, md, vd = dev(p), dev(m), dev(v)
    step, lr, b1, b2, eps = 3, 1e-3, 0.9, 0.999, 1e-8
    X.xlmimo_mlp_adam(pd, md, vd, dev(gr), step, lr)
    P = [[p.astype(np.float64), np.zeros(0)]]
    M_ = [[m.astype(np.float64), np.zeros(0)]]
    V_ = [[v.astype(np.float64), np.zeros(0)]]
    G_ = [(gr.astype(np.float64), np.zeros(0))]
    new = mlp.adam(P, G_, M_, V_, step, lr, b1, b2, eps)
    u = 2.0 ** -24
    tol_m = 8 * u * (b1 * np.abs(m) + (1 - b1) * np.abs(gr))
    assert np.all(np.abs(md.cpu().numpy() - M_[0][0]) <= tol_m)
    assert np.allclose(vd.cpu().numpy(), V_[0][0], rtol=8 * u, atol=0)
    c1, c2 = 1 / (1 - b1 ** step), 1 / (1 - b2 ** step)
    den = np.sqrt(V_[0][0] * c2) + eps
    upd = lr * M_[0][0] * c1 / den
    tol_p = 4 * u * np.abs(new[0][0]) + lr * c1 * tol_m / den + 16 * u * np.abs(upd)
    assert np.all(np.abs(pd.cpu().numpy() - new[0][0]) <= tol_p)


def small_case(K=6, B=3, n=4096, f=100e9, r=(3.0, 30.0), seed=41):
    users = inputs.users_polar(seed, B, K, r)
    return users, n, inputs.wavelength(f)


def test_pair_features_targets_weights(orc):
    users, n, lam = small_case()
    B, K = users.shape[:2]
    G = orc.gram(orc.FSPL, n, lam, lam / 2, 1.0, users)
    Gc = orc.closed_form(orc.FSPL, n, lam, lam / 2, 1.0, users)
    arr = X.array(n, lam)
    f, t, w = X.xlmimo_pair_features(arr, dev(users), dev(G), dev(Gc), weights=True)
    assert np.allclose(f.cpu().numpy(), mlp.pair_features(users, n, lam, lam / 2), rtol=0, atol=2e-6)
    assert np.allclose(t.cpu().numpy(), mlp.pair_targets(G, Gc), rtol=1e-6, atol=1e-7)
    assert np.allclose(w.cpu().numpy(), mlp.pair_weights(Gc), rtol=1e-6, atol=0)


def test_surrogate_constant_network_is_exact_scaling(orc):
    """A network whose only nonzero parameter is the output bias predicts the
    same t for every pair: the surrogate must be exactly G~ (1 + t) off the
    diagonal, Hermitian, with the closed-form diagonal."""
    users, n, lam = small_case(K=23, B=37)  # 253 pairs per trial: ragged last CTA
    p = np.zeros(X.MLP_PARAMS, np.float32)
    p[-2:] = [0.25, -0.5]
    arr = X.array(n, lam)
    gs = X.xlmimo_surrogate_gram(arr, dev(users), X.xlmimo_mlp_pack(dev(p))).cpu().numpy()
    Gc = orc.closed_form(orc.FSPL, n, lam, lam / 2, 1.0, users)
    K = users.shape[1]
    off = ~np.eye(K, dtype=bool)
    rows = users.shape[0] * K * (K - 1) // 2
    want = mlp.apply_correction(Gc, np.tile([0.25, -0.5], (rows, 1)))
    tol = 3e-6 * np.abs(Gc[:, off])  # the closed form's FP32-trig tolerance (2e-6) times |1 + t|
    assert np.all(np.abs(gs[:, off] - want[:, off]) <= tol + 1e-300)
    assert np.allclose(np.diagonal(gs, axis1=1, axis2=2), np.diagonal(Gc, axis1=1, axis2=2), rtol=1e-9, atol=0)
    assert np.array_equal(gs, np.conj(np.transpose(gs, (0, 2, 1))))


@pytest.mark.parametrize("K,B", [(2, 1), (8, 5), (64, 3)])
def test_surrogate_matches_oracle(orc, K, B):
    """Tensor-core inference of a random network against the oracle network
    (BF16 layers, exact SiLU) applied to the oracle's closed form."""
    users, n, lam = small_case(K=K, B=B, seed=50 + K)
    p = params_np(60 + K, 3.0)
    arr = X.array(n, lam)
    gs = X.xlmimo_surrogate_gram(arr, dev(users), X.xlmimo_mlp_pack(dev(p))).cpu().numpy()
    Gc = orc.closed_form(orc.FSPL, n, lam, lam / 2, 1.0, users)
    tr, _ = mlp.forward(mlp.unflatten(p), mlp.pair_features(users, n, lam, lam / 2), qlayers=Q)
    want = mlp.apply_correction(Gc, tr)
    iu = np.triu_indices(K, 1)
    tg = gs[:, iu[0], iu[1]] / Gc[:, iu[0], iu[1]] - 1.0
    tw = want[:, iu[0], iu[1]] / Gc[:, iu[0], iu[1]] - 1.0
    scale = float(np.abs(tr).max())
    assert scale > 0.05  # the network is not trivially small
    err = np.abs(tg - tw)
    assert err.max() <= 2e-2 * max(1.0, scale)
    assert np.quantile(err, 0.5) <= 4e-3 * max(1.0, scale)
    assert np.array_equal(gs, np.conj(np.transpose(gs, (0, 2, 1))))


@pytest.mark.parametrize("base", [1, 2])
def test_pair_targets_and_constant_network_with_aperture_base(orc, base):
    """Targets G/G~ - F and the surrogate G~ (F + t) for the aperture factors."""
    from oracle import aperture as ap
    users, n, lam = small_case(K=9, B=6, n=2048, f=100e9, seed=44)
    G = orc.gram(orc.FSPL, n, lam, lam / 2, 1.0, users)
    Gc = orc.closed_form(orc.FSPL, n, lam, lam / 2, 1.0, users)
    F = ap.factors(base, users, n, lam, lam / 2)
    arr = X.array(n, lam)
    _, t, _ = X.xlmimo_pair_features(arr, dev(users), dev(G), dev(Gc), base=base)
    want = mlp.pair_targets(G, Gc) + np.stack([1.0 - F.real, -F.imag], 1)
    assert np.allclose(t.cpu().numpy(), want, rtol=0, atol=3e-5 * max(1.0, float(np.abs(want).max())))
    p = np.zeros(X.MLP_PARAMS, np.float32)
    p[-2:] = [0.125, 0.0625]
    gs = X.xlmimo_surrogate_gram(arr, dev(users), X.xlmimo_mlp_pack(dev(p)), base=base).cpu().numpy()
    K = users.shape[1]
    iu = np.triu_indices(K, 1)
    w = Gc[:, iu[0], iu[1]] * (F.reshape(users.shape[0], -1) + 0.125 + 0.0625j)
    assert np.all(np.abs(gs[:, iu[0], iu[1]] - w) <= 3e-5 * np.abs(Gc[:, iu[0], iu[1]]))


def test_surrogate_full_size_sampled(orc):
    """The benchmark's surrogate workload at full size (10^4 trials, K = 64, N =
    2^18, 100 GHz, Fresnel base) in the configuration the bench times; the
    oracle network on the oracle closed form checks sampled trials."""
    from oracle import aperture as ap
    wl = inputs.SURROGATE
    users = wl.users()
    B, K, n, lam = wl.trials, wl.k, wl.n_ant, wl.wavelength
    p = params_np(91, 1.5)
    arr = X.array(n, lam)
    gs = X.xlmimo_surrogate_gram(arr, dev(users), X.xlmimo_mlp_pack(dev(p)), base=X.APERTURE_FRESNEL)
    gh = gs.cpu().numpy()
    assert np.isfinite(gh).all()
    assert np.array_equal(gh, np.conj(np.transpose(gh, (0, 2, 1))))
    idx = np.array([0, 1, B // 2, B - 1])
    u = users[idx]
    Gc = orc.closed_form(orc.FSPL, n, lam, lam / 2, 1.0, u)
    F = ap.factors(ap.FRESNEL, u, n, lam, lam / 2)
    tr, _ = mlp.forward(mlp.unflatten(p), mlp.pair_features(u, n, lam, lam / 2), qlayers=Q)
    want = ap.apply(Gc, F + tr[:, 0] + 1j * tr[:, 1])
    iu = np.triu_indices(K, 1)
    c = np.abs(Gc[:, iu[0], iu[1]])
    err = np.abs(gh[idx][:, iu[0], iu[1]] - want[:, iu[0], iu[1]]) / c
    # pairs whose Fresnel cut sits within rounding of |u| = 2 may take either side
    from test_gpu_aperture import borderline
    keep = ~borderline(u, n, lam).reshape(len(idx), -1)
    assert keep.mean() > 0.99
    scale = max(1.0, float(np.abs(tr).max()))
    assert np.quantile(err[keep], 0.5) <= 4e-3 * scale
    assert err[keep].max() <= 2e-2 * scale


def test_surrogate_empty_and_single_user():
    arr = X.array(1024, 0.01)
    packed = X.xlmimo_mlp_pack(dev(np.zeros(X.MLP_PARAMS, np.float32)))
    u0 = torch.empty((0, 4, 2), dtype=torch.float64, device="cuda")
    assert X.xlmimo_surrogate_gram(arr, u0, packed).shape == (0, 4, 4)
    u1 = dev(inputs.users_polar(3, 2, 1, (5.0, 50.0)))
    g1 = X.xlmimo_surrogate_gram(arr, u1, packed)
    assert torch.equal(g1, X.xlmimo_corr_closed_form(arr, u1))


def test_trained_surrogate_beats_closed_form():
    """Trains the network on the GPU on pairs labelled by the exact kernel
    (N log-uniform in [2^10, 2^18], 28 and 100 GHz), then judges it on fresh
    100 GHz trials at N = 2^18 against the closed form alone: the surrogate's
    Gram error and its modified-ZF sum-rate error must both be smaller."""
    n, freq, users = inputs.surrogate_trials(71, 600, 32)
    feat, target, _ = surrogate.label_pairs(n, freq, users)
    assert torch.isfinite(target).all()
    params = dev(inputs.mlp_init_params(72))
    tr = surrogate.Trainer(params, batch=4096, lr=1e-3, seed=73)
    log = tr.fit(feat, target, steps=1500, log_every=500)
    assert log[-1][1] < 0.5 * log[0][1]
    packed = X.xlmimo_mlp_pack(params)
    arr = X.array(262144, inputs.wavelength(100e9))
    u = dev(inputs.users_polar(74, 8, 32, (3.0, 30.0)))
    res = surrogate.compare(arr, u, packed)
    re = res["rate_exact"]
    e_cf = np.abs(res["rate_cf"] - re) / re
    e_sur = np.abs(res["rate_sur"] - re) / re
    assert np.all(res["status_sur"] == 0)
    assert float(np.mean(res["gram_err_sur"])) < float(np.mean(res["gram_err_cf"]))
    assert float(np.mean(e_sur)) < 0.7 * float(np.mean(e_cf)), (np.mean(e_sur), np.mean(e_cf))


def test_trained_surrogate_on_fresnel_base_does_not_lose():
    """With the finite-aperture Fresnel factor as its base, the network
    corrects an already good analytic form: trained briefly, it must stay
    within 10 % of that form's sum-rate error and well below the paper's
    closed form."""
    n, freq, users = inputs.surrogate_trials(75, 600, 32)
    feat, target, _ = surrogate.label_pairs(n, freq, users, base=X.APERTURE_FRESNEL)
    params = dev(inputs.mlp_init_params(76))
    surrogate.Trainer(params, batch=4096, lr=1e-3, seed=77).fit(feat, target, steps=1500)
    packed = X.xlmimo_mlp_pack(params)
    arr = X.array(262144, inputs.wavelength(100e9))
    u = dev(inputs.users_polar(78, 8, 32, (3.0, 30.0)))
    res = surrogate.compare(arr, u, packed, base=X.APERTURE_FRESNEL)
    re = res["rate_exact"]
    e = {k: float(np.mean(np.abs(res["rate_" + k] - re) / re)) for k in ("cf", "fresnel", "sur")}
    assert e["sur"] <= 1.1 * e["fresnel"] and e["sur"] < 0.5 * e["cf"], e


def test_trainer_checkpoint_roundtrip(tmp_path):
    n, freq, users = inputs.surrogate_trials(81, 40, 16)
    feat, target, _ = surrogate.label_pairs(n, freq, users)
    pa = dev(inputs.mlp_init_params(82))
    ta = surrogate.Trainer(pa, batch=1024, seed=83)
    ta.fit(feat, target, steps=6)
    path = str(tmp_path / "ck.npz")
    ta.save(path)
    ta.fit(feat, target, steps=4)
    pb = dev(inputs.mlp_init_params(0))
    tb = surrogate.Trainer(pb, batch=1024, seed=0)
    tb.load(path)
    tb.fit(feat, target, steps=4)
    assert tb.step == ta.step
    assert torch.equal(pa, pb)
