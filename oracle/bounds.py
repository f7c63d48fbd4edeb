"""Appendix A quantities: the capacity bounds of Hadamard's inequality and of
the Schur-Horn theorem, and the empirical expectation of Fig. 5 (test
infrastructure only: only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg use this module).

For one trial with channel vectors h_1..h_K (Gram G = H^H H) and the receive
SNR of user i, a_i = the i-th diagonal element of (P / sigma_n^2) H^H H
(Appendix A, first equation):

  * the correlation matrix R, r_ij = h_i^H h_j / (|h_i| |h_j|), so that
    (P / sigma_n^2) H^H H = P^{1/2} R P^{1/2} with P = Diag(a_1..a_K);
  * the capacity C = log2 det(I + P^{1/2} R P^{1/2});
  * the Hadamard upper bound U = prod_i (1 + a_i);
  * the lower bound L = det(R) prod_i (1 + a_i)  (Eq. (lower_bound));
  * the normalised gap of Eq. (9) at a_i = 1 (0 dB), the negative empirical
    expectation -E_K[log2 lambda^R] = -(1/K) sum_i log2 lambda_i^R
    = -(1/K) log2 det R, plotted against K in Fig. 5.

Everything is returned in log2 form.  Determinants are LAPACK's (numpy
slogdet on the explicit matrices, no blocking or reordering of ours).
"""
from __future__ import annotations

import math

import numpy as np


def correlation(G):
    """R from the Gram matrices G [B][K][K] (complex128): r_ij = G_ij / sqrt(G_ii G_jj)."""
    G = np.asarray(G, np.complex128)
    d = np.sqrt(np.real(np.einsum("bii->bi", G)))
    return G / (d[:, :, None] * d[:, None, :])


def log2det(A):
    """log2 det of Hermitian positive definite matrices A [B][K][K]."""
    sign, ld = np.linalg.slogdet(A)
    out = ld / math.log(2.0)
    out[np.real(sign) <= 0] = np.nan
    return out


def bounds(G, a):
    """[B][4]: log2 det R, C = log2 det(I + P^1/2 R P^1/2), log2 U, log2 L for
    Gram matrices G [B][K][K] and receive SNRs a (scalar or [B][K], linear)."""
    R = correlation(G)
    B, K, _ = R.shape
    a = np.broadcast_to(np.asarray(a, np.float64), (B, K))
    s = np.sqrt(a)
    M = np.eye(K)[None] + s[:, :, None] * R * s[:, None, :]
    ldr = log2det(R)
    c = log2det(M)
    lu = np.sum(np.log2(1.0 + a), axis=1)
    return np.stack([ldr, c, lu, ldr + lu], axis=1)


def neg_expectation(G):
    """-E_K[log2 lambda^R] = -(1/K) log2 det R per trial (Eq. (9), Fig. 5)."""
    R = correlation(G)
    return -log2det(R) / R.shape[-1]
