"""Runge-Kutta convolution quadrature with constant steps, 2-stage Radau IIA
(oracle, FP64, test infrastructure).

The paper's time discretisation (Sec. 2.4) is the Runge-Kutta generalised
convolution quadrature with a 2-stage Radau IIA method; with constant steps
it reduces to Runge-Kutta CQ, whose weights are the coefficients of
K(Delta(zeta) / dt) = sum_n W_n zeta^n with the matrix symbol
Delta(zeta) = (A + zeta / (1 - zeta) 1 b^T)^-1 of the Butcher tableau
(A, b, c) (the method's stability function enters through b^T A^-1 =
(0, ..., 1), Sec. 2.4).  For stage data g_j = (g(t_j + c_i dt))_i the
convolution (K * g)(t_n + c_i dt) is approximated by sum_{j <= n} W_{n-j} g_j.
As for BDF2 (oracle/cq.py), the Cauchy integral for the weights is taken by
the trapezoidal rule on |zeta| = lam with L = N + 1 points, which makes the
whole approximation a stage-wise scaled DFT:

    g^_l = sum_j lam^j exp(-2 pi i j l / L) g_j          (each stage)
    y^_l = K(Delta(zeta_l) / dt) g^_l,  zeta_l = lam exp(-2 pi i l / L)
    y_n  = lam^-n / L sum_l exp(2 pi i n l / L) y^_l

and K of the 2 x 2 matrix Delta(zeta_l) / dt is applied through its
eigendecomposition Delta(zeta_l) = P_l diag(mu_l) P_l^-1:
K(Delta / dt) = P_l diag(K(mu_l1 / dt), K(mu_l2 / dt)) P_l^-1.  The
frequencies at which the operator is needed are s_{l, j} = mu_lj / dt,
2 L of them.

Pins (tests/test_oracle_rkcq.py): the tableau's order conditions and
b^T A^-1 = (0, 1); K(s) = 1 reproduces the data; K(s) = 1/s (integration)
is exact for data polynomial of degree <= 2 in t (stage order 2); the
convolution with 1/(s + a) converges to the exact one at third order in dt.
"""
from __future__ import annotations

import numpy as np

from . import cq

# 2-stage Radau IIA
A_RADAU2 = np.array([[5.0 / 12.0, -1.0 / 12.0], [3.0 / 4.0, 1.0 / 4.0]])
B_RADAU2 = np.array([3.0 / 4.0, 1.0 / 4.0])
C_RADAU2 = np.array([1.0 / 3.0, 1.0])


def delta(zeta: complex) -> np.ndarray:
    """Delta(zeta) = (A + zeta / (1 - zeta) 1 b^T)^-1 (2 x 2 complex)."""
    M = A_RADAU2.astype(complex) + (zeta / (1.0 - zeta)) * np.outer(np.ones(2), B_RADAU2)
    return np.linalg.inv(M)


def symbols(N: int, lam: float | None = None):
    """For l = 0 .. L - 1 (L = N + 1): the eigenvalues mu_l (2,) and the
    eigenvector matrices P_l, P_l^-1 of Delta(zeta_l), zeta_l =
    lam exp(-2 pi i l / L), eigenvalues ordered by increasing imaginary part
    then real part."""
    L = N + 1
    lam = cq.lam_c(N) if lam is None else lam
    mus, Ps, Pis = [], [], []
    for l in range(L):
        z = lam * np.exp(-2j * np.pi * l / L)
        w, V = np.linalg.eig(delta(z))
        order = np.lexsort((w.real, w.imag))
        w, V = w[order], V[:, order]
        mus.append(w)
        Ps.append(V)
        Pis.append(np.linalg.inv(V))
    return np.array(mus), np.array(Ps), np.array(Pis)


def freqs_radau2(N: int, dt: float) -> np.ndarray:
    """The 2 L frequencies s_{l, j} = mu_lj / dt, ordered k = 2 l + j."""
    mus, _, _ = symbols(N)
    return (mus / dt).reshape(-1)


def convolve(apply_k, g: np.ndarray, N: int, dt: float, lam: float | None = None) -> np.ndarray:
    """RK-CQ approximation of (K * g) at the stage times: g (L, 2, ...) the
    stage samples g(t_j + c_i dt); apply_k(k, s, x) returns K(s) x for the
    frequency s = s_k (k = 2 l + j) and x of g's trailing shape (the
    result may have another trailing shape).  Returns y (L, 2, ...),
    y[n, i] ~ (K * g)(t_n + c_i dt).  lam (default
    cq.lam_c(N), the radius the CQ path uses) sets the aliasing error
    ~ lam^L against the rounding amplification lam^-N."""
    L = N + 1
    mus, Ps, Pis = symbols(N, lam)
    gh = cq.forward(g.astype(complex), N, lam)      # (L, 2, ...)
    yh = []
    for l in range(L):
        e = np.tensordot(Pis[l], gh[l], axes=(1, 0))          # eigen-coordinates
        f = np.stack([np.asarray(apply_k(2 * l + j, mus[l, j] / dt, e[j])) for j in range(2)])
        yh.append(np.tensordot(Ps[l], f, axes=(1, 0)))
    return cq.inverse(np.stack(yh), N, lam)


def stage_times(N: int, dt: float) -> np.ndarray:
    """t_n + c_i dt for n = 0..N (step n covers (t_n, t_n + dt]), shape (L, 2)."""
    return dt * (np.arange(N + 1)[:, None] + C_RADAU2[None, :])


def dirichlet_traction(xyz, tri, material, u: np.ndarray, N: int, dt: float) -> np.ndarray:
    """The Dirichlet problem of collocation BEM (Sec. 2.3, Eq. (2.15) at the
    element midpoints): V t = (C + K) u in time, by RK-CQ with the dense
    oracle operators at the oracle's frequencies: per frequency
    t^ = V(s)^-1 (C + K)(s) u^.  u: stage data at the nodes (L, 2, n_nodes, 3);
    returns the traction stage data at the elements (L, 2, n_tris, 3)."""
    from . import bem
    s = freqs_radau2(N, dt)
    Vd = bem.Operator(xyz, tri, material, bem.ROWS_CENTROIDS, bem.KERNEL_SL).dense(s)
    Ad = bem.Operator(xyz, tri, material, bem.ROWS_CENTROIDS, bem.KERNEL_DL).dense(s)
    V = [bem.to_matrix(Vd[:, :, k]) for k in range(len(s))]
    A = [bem.to_matrix(Ad[:, :, k]) for k in range(len(s))]
    return convolve(lambda k, sk, x: np.linalg.solve(V[k], A[k] @ x.reshape(-1)).reshape(-1, 3), u, N, dt).real
