"""Pins of the surrogate's CPU reference: central finite differences of the
loss (FP64) against the backward pass, the Adam update against its closed
form after one step, SiLU's derivative, and the feature / target / correction
definitions on a hand-made pair."""
import math

import numpy as np
import pytest

from oracle import mlp


def make_params(seed, dims):
    g = np.random.Generator(np.random.Philox(key=seed))
    return [(g.normal(0, 1 / math.sqrt(a), (a, b)), g.normal(0, 0.1, b)) for a, b in zip(dims[:-1], dims[1:])]


def test_silu_grad_finite_difference():
    z = np.linspace(-6, 6, 101)
    h = 1e-6
    fd = (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h)
    assert np.allclose(mlp.silu_grad(z), fd, rtol=0, atol=1e-9)


def test_backward_matches_finite_differences():
    dims = [6, 16, 16, 16, 2]
    params = make_params(1, dims)
    g = np.random.Generator(np.random.Philox(key=2))
    X = g.normal(size=(9, 6))
    T = g.normal(size=(9, 2))
    out, cache = mlp.forward(params, X)
    loss, dout = mlp.mse(out, T)
    grads = mlp.backward(params, cache, dout)
    h = 1e-6
    for l in range(len(params)):
        for q in range(2):
            P = params[l][q]
            idx = [tuple(g.integers(0, s) for s in P.shape) for _ in range(5)]
            for ix in idx:
                old = P[ix]
                P[ix] = old + h
                lp, _ = mlp.mse(mlp.forward(params, X)[0], T)
                P[ix] = old - h
                lm, _ = mlp.mse(mlp.forward(params, X)[0], T)
                P[ix] = old
                fd = (lp - lm) / (2 * h)
                assert abs(grads[l][q][ix] - fd) <= 1e-7 * max(1.0, abs(fd))


def test_adam_first_step_closed_form():
    """After one step from zero moments, Adam moves every parameter by
    -lr * g / (|g| + eps) (bias corrections cancel the (1-b) factors)."""
    params = make_params(3, [4, 3])
    grads = make_params(4, [4, 3])
    m = [[np.zeros_like(params[0][0]), np.zeros_like(params[0][1])]]
    v = [[np.zeros_like(params[0][0]), np.zeros_like(params[0][1])]]
    new = mlp.adam(params, grads, m, v, 1, 1e-2)
    for q in range(2):
        gq = grads[0][q]
        assert np.allclose(new[0][q], params[0][q] - 1e-2 * gq / (np.abs(gq) + 1e-8), rtol=1e-12, atol=1e-15)


def test_pair_features_targets_and_correction():
    users = np.array([[[3.0, 4.0], [10.0, -1.0], [2.0, 2.0]]])
    lam = 0.01
    F = mlp.pair_features(users, 4096, lam, lam / 2)
    assert F.shape == (3, 6)
    assert np.allclose(F[0], [(math.log(500.0) - 7.5) / 2, math.atan2(4, 3) / (math.pi / 3),
                              (math.log(math.hypot(10, -1) / lam) - 7.5) / 2, math.atan2(-1, 10) / (math.pi / 3),
                              (12 - 14) / 4, 0.0])
    g = np.random.Generator(np.random.Philox(key=5))
    Gc = g.normal(size=(1, 3, 3)) + 1j * g.normal(size=(1, 3, 3))
    t = g.normal(size=(3, 2)) * 0.1
    G = mlp.apply_correction(Gc, t)
    assert np.allclose(mlp.pair_targets(G, Gc), t, rtol=1e-12, atol=1e-14)
    assert np.allclose(np.diag(G[0]), np.diag(Gc[0]))


def test_bf16_rounding_matches_torch():
    """The BF16 rounding against torch's float32 -> bfloat16 conversion
    (round to nearest even), including ties and values near powers of two."""
    import torch
    g = np.random.Generator(np.random.Philox(key=6))
    x = np.concatenate([g.normal(size=4000).astype(np.float32) * np.float32(10.0) ** g.integers(-8, 8, 4000),
                        np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8), 2.0 - 2.0 ** -9,
                                  0.0, -0.0], np.float32)])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), ref)
    assert mlp.bf16(np.float32(1.0 + 2.0 ** -8)) == 1.0          # tie -> even
    assert mlp.bf16(np.float32(1.0 + 3 * 2.0 ** -8)) == 1.0 + 2.0 ** -6


def test_quantized_backward_is_straight_through():
    """With rounded layers, the gradient equals the exact gradient of the
    network whose weights are the rounded ones, evaluated on rounded inputs:
    checked against finite differences of a network with pre-rounded
    weights, where input rounding is kept fixed by using inputs that are
    already BF16 values (the rounding of a BF16 value is itself)."""
    dims = [6, 16, 16, 2]
    params = make_params(7, dims)
    params = [(mlp.bf16(W), b) for W, b in params]
    g = np.random.Generator(np.random.Philox(key=8))
    X = g.normal(size=(5, 6))
    T = g.normal(size=(5, 2))
    out_q, cache_q = mlp.forward(params, X, qlayers=(1,))
    out_p, cache_p = mlp.forward(params, X)
    # hidden activations are not BF16 values, so layer 1 differs only by input rounding
    assert not np.allclose(out_q, out_p, rtol=0, atol=0)
    _, dq = mlp.mse(out_q, T)
    gq = mlp.backward(params, cache_q, dq, qlayers=(1,))
    # layer 1's weight gradient is bf16(h)^T dz; recompute it from the cache by definition
    h1, z1 = cache_q[1]
    dz1 = (dq @ params[2][0].T) * mlp.silu_grad(z1)
    assert np.allclose(gq[1][0], mlp.bf16(h1).T @ dz1, rtol=1e-13, atol=0)
    assert np.allclose(gq[2][0], cache_q[2][0].T @ dq, rtol=1e-13, atol=0)


def test_weighted_mse_gradient():
    g = np.random.Generator(np.random.Philox(key=9))
    out, T, w = g.normal(size=(7, 2)), g.normal(size=(7, 2)), g.random(7)
    loss, d = mlp.mse(out, T, w)
    h = 1e-6
    for ix in [(0, 0), (3, 1), (6, 0)]:
        o2 = out.copy(); o2[ix] += h
        lp, _ = mlp.mse(o2, T, w)
        o2[ix] -= 2 * h
        lm, _ = mlp.mse(o2, T, w)
        assert abs((lp - lm) / (2 * h) - d[ix]) < 1e-8


def test_flatten_roundtrip_layout():
    theta = np.arange(199682, dtype=np.float64)
    p = mlp.unflatten(theta)
    assert p[0][0][1, 0] == 256 and p[0][1][0] == 6 * 256 and p[4][1][1] == 199681
    assert np.array_equal(mlp.flatten(p), theta)
