"""Pins of oracle/rkcq.py (constant-step Runge-Kutta CQ, 2-stage Radau IIA)
against facts that do not rest on it: the tableau's order conditions and
stiff accuracy; K(s) = 1 reproducing the data; for K(s) = 1/(s + a) the
RK-CQ result is the Radau IIA time stepping of y' = -a y + g, y(0) = 0
(Lubich and Ostermann's identity), written here as a plain stage solve;
integration (a = 0) exact for data of degree <= 1 at both stages and
degree <= 2 at the step point (stage order 2, classical order 3); and
third-order convergence of the convolution with 1/(s + a) against its
closed form.  Radius lam with lam^N = 1e-8 (aliasing lam^L and rounding
amplification lam^-N balanced) unless the default is under test."""
import numpy as np
import pytest

from oracle import rkcq

A, B, C = rkcq.A_RADAU2, rkcq.B_RADAU2, rkcq.C_RADAU2


def _lam(N):
    return (1e-16) ** (1.0 / (2 * N))


def _stage_times(N, dt):
    return dt * (np.arange(N + 1)[:, None] + C[None, :])


def _radau_steps(a, g, dt):
    """Radau IIA stage values of y' = -a y + g, y(0) = 0: per step
    (I + a dt A) Y = y_n 1 + dt A g_n, y_{n+1} = last stage."""
    out = np.zeros_like(g)
    y = 0.0
    M = np.eye(2) + a * dt * A
    for n in range(g.shape[0]):
        Y = np.linalg.solve(M, y * np.ones(2) + dt * A @ g[n])
        out[n] = Y
        y = Y[-1]
    return out


def test_radau_tableau_order_and_stiff_accuracy():
    assert np.allclose(A.sum(1), C)
    for q in range(1, 4):                      # B(3): sum_i b_i c_i^(q-1) = 1/q
        assert abs((B * C ** (q - 1)).sum() - 1.0 / q) < 1e-15
    for q in range(1, 3):                      # C(2): sum_j a_ij c_j^(q-1) = c_i^q / q
        assert np.allclose(A @ C ** (q - 1), C ** q / q)
    assert np.allclose(B @ np.linalg.inv(A), [0.0, 1.0])
    assert np.allclose(A[-1], B)               # stiffly accurate


def test_identity_kernel_reproduces_data_default_radius():
    N, dt = 20, 0.05
    t = _stage_times(N, dt)
    g = np.sin(3 * t) + t ** 2
    y = rkcq.convolve(lambda k, s, x: x, g, N, dt)
    assert np.abs(y - g).max() < 1e-8 * np.abs(g).max()


@pytest.mark.parametrize("a", [0.0, 2.0, 50.0])
@pytest.mark.parametrize("N", [16, 41])
def test_equals_radau_time_stepping(a, N):
    dt = 1.0 / (N + 1)
    t = _stage_times(N, dt)
    g = np.sin(4 * t) + t ** 2 - 0.3
    y = rkcq.convolve(lambda k, s, x: x / (s + a), g, N, dt, _lam(N))
    ref = _radau_steps(a, g, dt)
    assert np.abs(y.imag).max() < 1e-7
    assert np.abs(y.real - ref).max() < 2e-8 * max(1.0, np.abs(ref).max()), np.abs(y.real - ref).max()


@pytest.mark.parametrize("deg", [0, 1, 2])
def test_integration_exact_for_low_degree(deg):
    N, dt = 16, 0.1
    t = _stage_times(N, dt)
    y = rkcq.convolve(lambda k, s, x: x / s, t ** deg, N, dt, _lam(N)).real
    exact = t ** (deg + 1) / (deg + 1)
    tol = 2e-8 * np.abs(exact).max()
    assert np.abs(y[:, 1] - exact[:, 1]).max() < tol            # step points: order 3
    if deg <= 1:                                                # inner stage: stage order 2
        assert np.abs(y[:, 0] - exact[:, 0]).max() < tol
    else:
        assert np.abs(y[:, 0] - exact[:, 0]).max() > 1e3 * tol


def test_third_order_convolution():
    a, errs = 2.0, []
    Ns = (16, 32, 64, 128)
    for N in Ns:
        dt = 1.0 / (N + 1)
        t = _stage_times(N, dt)
        y = rkcq.convolve(lambda k, s, x: x / (s + a), np.sin(4 * t), N, dt, _lam(N)).real
        # e^{-a t} * sin(4 t) in closed form
        exact = (4 * np.exp(-a * t) - 4 * np.cos(4 * t) + a * np.sin(4 * t)) / (a * a + 16)
        errs.append(np.abs(y - exact).max())
    rates = [np.log(errs[i] / errs[i + 1]) / np.log((Ns[i + 1] + 1) / (Ns[i] + 1)) for i in range(len(Ns) - 1)]
    assert min(rates) > 2.7 and rates[-1] > 2.9, (errs, rates)


def test_frequencies_come_in_conjugate_pairs_and_lie_right():
    N, dt = 15, 1e-3
    s = rkcq.freqs_radau2(N, dt)
    assert len(s) == 2 * (N + 1)
    assert (s.real > 0).all()
    for v in s:                                # closed under conjugation (l <-> L - l)
        assert np.abs(s - np.conj(v)).min() < 1e-9 * np.abs(v)


def test_matrix_valued_kernel_equals_radau_system_stepping():
    """The operator case (what the library's RK-CQ computes with a BEM
    operator): K(s) = B (s I + M)^-1 with M non-symmetric, positive real
    eigenvalues, and B rectangular (the output has another trailing shape
    than the input).  RK-CQ equals B times the Radau IIA stage values of
    the system y' = -M y + g, y(0) = 0."""
    rng = np.random.default_rng(5)
    Q = rng.normal(size=(3, 3))
    M = Q @ np.diag([0.5, 2.0, 7.0]) @ np.linalg.inv(Q)
    Bm = rng.normal(size=(2, 3))
    N = 30
    dt = 1.0 / (N + 1)
    t = _stage_times(N, dt)
    g = np.stack([np.sin(3 * t), t ** 2, np.cos(t) - 1.0], axis=-1)          # (L, 2, 3)
    y = rkcq.convolve(lambda k, s, x: Bm @ np.linalg.solve(s * np.eye(3) + M, x), g, N, dt, _lam(N))
    # stage system per step: Y_i = y_n + dt sum_j a_ij (-M Y_j + g_j)
    Y = np.zeros((N + 1, 2, 3))
    yn = np.zeros(3)
    big = np.eye(6) + dt * np.kron(A, M)
    for n in range(N + 1):
        rhs = np.concatenate([yn + dt * (A[0, 0] * g[n, 0] + A[0, 1] * g[n, 1]),
                              yn + dt * (A[1, 0] * g[n, 0] + A[1, 1] * g[n, 1])])
        st = np.linalg.solve(big, rhs).reshape(2, 3)
        Y[n] = st
        yn = st[1]
    ref = Y @ Bm.T
    assert y.shape == (N + 1, 2, 2)
    assert np.abs(y.imag).max() < 1e-7
    assert np.abs(y.real - ref).max() < 2e-8 * np.abs(ref).max(), np.abs(y.real - ref).max()
