"""Plain FP64 NumPy reference of the learned correlation surrogate (test
infrastructure only).  Nothing here is shared with the CUDA library.

The surrogate corrects the closed-form Gram of modified ZF (Sec. V-B,
Eqs. 4 and 6): for a user pair (i < j) it predicts t_ij = G_ij / G~_ij - 1 from
the pair's geometry, so that G~_ij (1 + t_ij) approaches the exact inner
product.  The network is a multilayer perceptron with SiLU activations.

Features of a pair (x = r cos(theta), y = r sin(theta) for each user, r the
distance to the array centre, theta the angle from broadside):
    ((ln(r_i / lambda) - 7.5) / 2, theta_i / (pi/3),
     (ln(r_j / lambda) - 7.5) / 2, theta_j / (pi/3),
     (log2 N - 14) / 4, (spacing / lambda - 0.5) * 4)
Targets: (Re t_ij, Im t_ij).
Parameters: a list of (W, b) per layer, W of shape [in, out]; hidden layers
apply silu(z) = z / (1 + e^{-z}); the last layer is linear.

Mixed precision: the layers listed in `qlayers` multiply the BF16 roundings
(round to nearest, ties to even) of their input and weights, with the sum
itself exact here; the backward pass differentiates that computation with the
rounding taken as the identity (straight-through), i.e. it reuses the rounded
input and weights.
"""
from __future__ import annotations

import math

import numpy as np


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as float64.
    BF16 keeps the upper 16 bits of the binary32 encoding, so rounding adds
    0x7FFF plus the lowest kept bit and truncates the low half."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


def _operands(params, l, h, qlayers):
    W = params[l][0]
    return (bf16(h), bf16(W)) if l in qlayers else (h, W)


def forward(params, X, qlayers=()):
    """Returns (output, cache) with cache = list of (input, pre-activation) per layer."""
    h = np.asarray(X, np.float64)
    cache = []
    for l, (W, b) in enumerate(params):
        hq, Wq = _operands(params, l, h, qlayers)
        z = hq @ Wq + b
        cache.append((h, z))
        h = silu(z) if l < len(params) - 1 else z
    return h, cache


def mse(out, target, weight=None):
    """Loss 0.5/M * sum_m w_m |out_m - target_m|^2 (w = 1 if None), and its gradient."""
    d = out - target
    M = out.shape[0]
    w = np.ones(M) if weight is None else np.asarray(weight, np.float64)
    return 0.5 * float(np.sum(w[:, None] * d * d)) / M, w[:, None] * d / M


def backward(params, cache, dout, qlayers=()):
    """Gradients [(dW, db)] of a scalar loss whose output gradient is dout."""
    grads = [None] * len(params)
    g = dout
    for l in range(len(params) - 1, -1, -1):
        h, z = cache[l]
        if l < len(params) - 1:
            g = g * silu_grad(z)
        hq, Wq = _operands(params, l, h, qlayers)
        grads[l] = (hq.T @ g, g.sum(axis=0))
        g = g @ Wq.T
    return grads


def adam(params, grads, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba): bias-corrected first and second moments."""
    out = []
    for l in range(len(params)):
        new = []
        for q in range(2):
            g = grads[l][q]
            m[l][q] = b1 * m[l][q] + (1 - b1) * g
            v[l][q] = b2 * v[l][q] + (1 - b2) * g * g
            mh = m[l][q] / (1 - b1 ** step)
            vh = v[l][q] / (1 - b2 ** step)
            new.append(params[l][q] - lr * mh / (np.sqrt(vh) + eps))
        out.append(tuple(new))
    return out


def pair_features(users, n_ant, wavelength, spacing):
    """[B * K(K-1)/2][6] features of every pair i < j of every trial, pairs in
    row order (i, then j)."""
    users = np.asarray(users, np.float64)
    B, K, _ = users.shape
    rows = []
    for b in range(B):
        for i in range(K):
            for j in range(i + 1, K):
                f = []
                for k in (i, j):
                    x, y = users[b, k]
                    r = math.hypot(x, y)
                    f += [(math.log(r / wavelength) - 7.5) / 2.0, math.atan2(y, x) / (math.pi / 3)]
                f += [(math.log2(n_ant) - 14.0) / 4.0, (spacing / wavelength - 0.5) * 4.0]
                rows.append(f)
    return np.array(rows, np.float64).reshape(-1, 6)


def pair_weights(Gc):
    """[B * K(K-1)/2] |G~_ij|^2 / (G~_ii G~_jj) for every pair i < j."""
    B, K, _ = Gc.shape
    rows = []
    for b in range(B):
        for i in range(K):
            for j in range(i + 1, K):
                rows.append(abs(Gc[b, i, j]) ** 2 / (Gc[b, i, i].real * Gc[b, j, j].real))
    return np.array(rows, np.float64)


def unflatten(theta, dims=(6, 256, 256, 256, 256, 2)):
    """Parameter list [(W, b)] from the flat layout (per layer W [in][out], then b)."""
    theta = np.asarray(theta, np.float64)
    params, o = [], 0
    for a, b in zip(dims[:-1], dims[1:]):
        W = theta[o:o + a * b].reshape(a, b)
        o += a * b
        params.append((W, theta[o:o + b].copy()))
        o += b
    assert o == theta.size
    return params


def flatten(pairs):
    """Flat vector of [(W, b)] in the same layout."""
    return np.concatenate([np.concatenate([W.reshape(-1), b.reshape(-1)]) for W, b in pairs])


def pair_targets(G, Gc):
    """[B * K(K-1)/2][2] (Re, Im) of G_ij / G~_ij - 1 for every pair i < j."""
    B, K, _ = G.shape
    rows = []
    for b in range(B):
        for i in range(K):
            for j in range(i + 1, K):
                t = G[b, i, j] / Gc[b, i, j] - 1.0
                rows.append([t.real, t.imag])
    return np.array(rows, np.float64).reshape(-1, 2)


def apply_correction(Gc, pred):
    """Surrogate Gram: off-diagonal G~_ij (1 + t_ij) with t from pred (rows in
    pair order), mirrored to keep the matrix Hermitian; diagonal unchanged."""
    B, K, _ = Gc.shape
    out = Gc.copy()
    q = 0
    for b in range(B):
        for i in range(K):
            for j in range(i + 1, K):
                v = Gc[b, i, j] * (1.0 + pred[q, 0] + 1j * pred[q, 1])
                out[b, i, j] = v
                out[b, j, i] = np.conj(v)
                q += 1
    return out
