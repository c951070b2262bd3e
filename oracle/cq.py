"""Uniform-step convolution quadrature (BDF2) as a scaled DFT over the
frequency circle (oracle, FP64, test infrastructure).

The paper's gCQ (Sec. 2.4, Eqs. (2.17)-(2.21)) reduces for constant time
steps to Lubich's CQ, whose weights are the Taylor coefficients of
K(delta(zeta) / dt), delta(zeta) = (1 - zeta) + (1 - zeta)^2 / 2 for BDF2.
Approximating the Cauchy integral for the weights by the trapezoidal rule on
|zeta| = lam with L = N + 1 points gives, with s_k = delta(zeta_k)/dt,
zeta_k = lam exp(-2 pi i k / L):

    g^_k = sum_{j=0}^{N} lam^j g_j exp(-2 pi i j k / L)
    y^_k = K(s_k) g^_k
    y_n  = lam^{-n} / L  sum_{k=0}^{L-1} y^_k exp(2 pi i n k / L)

lam = (1e-10)^(1 / (2N)) (aliasing ~ lam^L).  Pins: convolution with
K(s) = 1/(s + a) and with a pure delay exp(-s d / c) / (4 pi d) against the
exact time-domain results, second-order error decay
(tests/test_oracle_cq.py).
"""
from __future__ import annotations

import numpy as np


def lam_c(N: int) -> float:
    return (1e-10) ** (1.0 / (2 * N))


def forward(g: np.ndarray, N: int, lam: float | None = None) -> np.ndarray:
    """g (L, ...) time samples g_0..g_N -> g^ (L, ...); lam defaults to lam_c(N)."""
    L = N + 1
    lam = lam_c(N) if lam is None else lam
    j = np.arange(L)
    W = np.exp(-2j * np.pi * np.outer(np.arange(L), j) / L) * lam ** j[None, :]
    return np.tensordot(W, g, axes=(1, 0))


def inverse(yh: np.ndarray, N: int, lam: float | None = None) -> np.ndarray:
    """y^ (L, ...) -> y (L, ...), y_n = lam^-n / L sum_k y^_k e^{2 pi i n k / L}."""
    L = N + 1
    lam = lam_c(N) if lam is None else lam
    n = np.arange(L)
    W = np.exp(2j * np.pi * np.outer(n, np.arange(L)) / L) * (lam ** (-n.astype(float)))[:, None] / L
    return np.tensordot(W, yh, axes=(1, 0))


def convolve(Khat, g: np.ndarray, N: int, dt: float) -> np.ndarray:
    """Discrete convolution y_n ~ (K * g)(t_n) of samples g (L, ...) with the
    operator whose Laplace transform is Khat(s) (scalar function)."""
    from .bem import freqs_bdf2
    s = freqs_bdf2(N, dt)
    gh = forward(g, N)
    yh = np.stack([Khat(sk) * gh[k] for k, sk in enumerate(s)])
    return inverse(yh, N)
