"""Pins of the oracle's Laplace-domain kernels: symmetry, Kelvin limit,
Navier residual and traction by finite differences, series/closed form."""
import math

import numpy as np
import pytest

import synthetic as syn
from oracle import kernels as K

MATS = [syn.STEEL, syn.PAPER_CUBE_MATERIAL, (2700.0, 5.1e10, 2.6e10)]


def _speeds(mat):
    return K.wave_speeds(*mat)


def test_wave_speeds_steel():
    c1, c2 = K.wave_speeds(*syn.STEEL)
    assert abs(c1 - 6000.98) < 0.01 and abs(c2 - 3207.66) < 0.01
    c1, c2 = K.wave_speeds(*syn.PAPER_CUBE_MATERIAL)
    assert abs(c1 - 1.0) < 1e-15 and abs(c2 - math.sqrt(0.5)) < 1e-15


@pytest.mark.parametrize("mat", MATS)
@pytest.mark.parametrize("zabs", [0.3, 0.99, 1.01, 4.0, 30.0])
def test_symmetry_and_conjugation(mat, zabs):
    rho, lam, mu = mat
    c1, c2 = _speeds(mat)
    rng = np.random.default_rng(7)
    r = rng.normal(size=(6, 3))
    rr = np.linalg.norm(r, axis=1)
    s = zabs * c2 / rr.mean() * np.exp(0.7j)
    u = K.U(r, s, rho, lam, mu)
    np.testing.assert_allclose(u, np.swapaxes(u, -1, -2), rtol=0, atol=1e-15 * np.abs(u).max())
    np.testing.assert_allclose(K.U(-r, s, rho, lam, mu), u, rtol=1e-14)
    np.testing.assert_allclose(K.U(r, np.conj(s), rho, lam, mu), np.conj(u), rtol=1e-13)
    n = rng.normal(size=(6, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    t = K.T(r, n, s, rho, lam, mu)
    np.testing.assert_allclose(K.T(r, n, np.conj(s), rho, lam, mu), np.conj(t), rtol=1e-12)


@pytest.mark.parametrize("mat", MATS)
def test_kelvin_limit(mat):
    rho, lam, mu = mat
    c1, c2 = _speeds(mat)
    rng = np.random.default_rng(1)
    r = rng.normal(size=(8, 3))
    n = rng.normal(size=(8, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    s = 1e-6 * c2 / np.linalg.norm(r, axis=1).max() * np.exp(0.3j)
    u0 = K.kelvin_U(r, lam, mu)
    np.testing.assert_allclose(K.U(r, s, rho, lam, mu), u0, rtol=0, atol=1e-5 * np.abs(u0).max())
    # U has an O(s) rigid translation term; T starts at O(s^2)
    t0 = K.kelvin_T(r, n, lam, mu)
    np.testing.assert_allclose(K.T(r, n, s, rho, lam, mu), t0, rtol=0, atol=1e-11 * np.abs(t0).max())


def _fd_derivs(f, x, h):
    """4th-order central differences: returns grad (3, ...) and Hessian
    (3, 3, ...) of f at x."""
    e = np.eye(3) * h
    g = []
    for a in range(3):
        g.append((-f(x + 2 * e[a]) + 8 * f(x + e[a]) - 8 * f(x - e[a]) + f(x - 2 * e[a])) / (12 * h))
    H = [[None] * 3 for _ in range(3)]
    for a in range(3):
        for b in range(3):
            if a == b:
                H[a][b] = (-f(x + 2 * e[a]) + 16 * f(x + e[a]) - 30 * f(x) + 16 * f(x - e[a]) - f(x - 2 * e[a])) / (12 * h * h)
            else:
                def fa(y, a=a):
                    return (-f(y + 2 * e[a]) + 8 * f(y + e[a]) - 8 * f(y - e[a]) + f(y - 2 * e[a])) / (12 * h)
                H[a][b] = (-fa(x + 2 * e[b]) + 8 * fa(x + e[b]) - 8 * fa(x - e[b]) + fa(x - 2 * e[b])) / (12 * h)
    return np.array(g), np.array(H)


@pytest.mark.parametrize("mat", MATS)
@pytest.mark.parametrize("zabs", [0.2, 0.9, 1.2, 5.0])
def test_navier_residual(mat, zabs):
    """mu Lap U + (lambda + mu) grad div U - rho s^2 U = 0 away from r = 0."""
    rho, lam, mu = mat
    c1, c2 = _speeds(mat)
    x = np.array([0.31, -0.42, 0.55])
    r = np.linalg.norm(x)
    s = zabs * c2 / r * np.exp(0.4j)
    f = lambda y: K.U(y, s, rho, lam, mu)
    g, H = _fd_derivs(f, x, 1e-3 * r)
    lap = H[0, 0] + H[1, 1] + H[2, 2]                  # (3, 3)
    # (grad div U)_ij = d_i d_k U_kj
    graddiv = np.einsum("ikkj->ij", H)
    res = mu * lap + (lam + mu) * graddiv - rho * s * s * f(x)
    scale = mu * np.abs(lap).max() + rho * abs(s) ** 2 * np.abs(f(x)).max()
    assert np.abs(res).max() < 1e-7 * scale


@pytest.mark.parametrize("mat", MATS)
@pytest.mark.parametrize("zabs", [0.2, 1.5, 6.0])
def test_traction_by_fd_of_U(mat, zabs):
    """T_ij = lambda div(u^j) n_i + mu (d_k u_i + d_i u_k)^j n_k, u^j = U[:, j]."""
    rho, lam, mu = mat
    c1, c2 = _speeds(mat)
    x = np.array([-0.2, 0.37, 0.61])
    n = np.array([0.3, -0.5, 0.81])
    n /= np.linalg.norm(n)
    r = np.linalg.norm(x)
    s = zabs * c2 / r * np.exp(-0.5j)
    g, _ = _fd_derivs(lambda y: K.U(y, s, rho, lam, mu), x, 1e-4 * r)   # g[k][i, j] = d_k U_ij
    div = np.einsum("kkj->j", g)
    T = np.zeros((3, 3), complex)
    for i in range(3):
        for j in range(3):
            T[i, j] = lam * div[j] * n[i] + mu * sum((g[k][i, j] + g[i][k, j]) * n[k] for k in range(3))
    Tk = K.T(x, n, s, rho, lam, mu)
    assert np.abs(T - Tk).max() < 1e-9 * np.abs(Tk).max()


@pytest.mark.parametrize("mat", MATS)
def test_series_matches_closed_form(mat):
    c1, c2 = _speeds(mat)
    r = np.array([0.7, 1.3])
    for arg in [0.0, 0.6, 1.4, -2.0]:
        s = 1.0 * c2 / r * np.exp(1j * arg)
        old = K.SERIES_Z
        try:
            K.SERIES_Z = 0.0
            a = K.coeffs(r, s, c1, c2)
            K.SERIES_Z = 10.0
            b = K.coeffs(r, s, c1, c2)
            K.SERIES_Z = 0.0
            ad = K.coeffs(r, s, c1, c2, dynamic=True)
            K.SERIES_Z = 10.0
            bd = K.coeffs(r, s, c1, c2, dynamic=True)
        finally:
            K.SERIES_Z = old
        for x, y in zip(a + ad, b + bd):
            np.testing.assert_allclose(x, y, rtol=1e-12)


def _speed_perturbed(mat, wave, dc):
    """Material (rho, lam, mu) with one wave speed moved by dc at fixed rho."""
    rho = mat[0]
    c1, c2 = K.wave_speeds(*mat)
    if wave == "p":
        c1 += dc
    else:
        c2 += dc
    return (rho,) + K.lame_from_speeds(rho, c1, c2)


@pytest.mark.parametrize("mat", MATS)
@pytest.mark.parametrize("wave", ["p", "s"])
@pytest.mark.parametrize("zabs", [0.3, 2.5, 30.0])
def test_speed_derivative_by_fd_of_U(mat, wave, zabs):
    """dU/dc_a against 4th-order central differences of U in c_a (rho fixed)."""
    c1, c2 = _speeds(mat)
    rng = np.random.default_rng(11)
    r = rng.normal(size=(6, 3))
    s = zabs * c2 / np.linalg.norm(r, axis=1).mean() * np.exp(0.6j)
    c = c1 if wave == "p" else c2
    h = 1e-4 * c

    def u(dc):
        return K.U(r, s, *_speed_perturbed(mat, wave, dc))
    fd = (-u(2 * h) + 8 * u(h) - 8 * u(-h) + u(-2 * h)) / (12 * h)
    d = K.dU_dc(r, s, *mat, wave)
    np.testing.assert_allclose(d, fd, rtol=0, atol=1e-8 * np.abs(fd).max())
    assert np.abs(d).max() > 0


@pytest.mark.parametrize("mat", MATS)
def test_speed_derivative_kelvin_limit(mat):
    """s -> 0: Kelvin U written in the wave speeds,
    [(1/c1^2 + 1/c2^2) I + (1/c2^2 - 1/c1^2) rh rh^T] / (8 pi rho r), equals
    kelvin_U, and its c-derivatives are [rh rh^T - I] / (4 pi rho r c1^3) and
    -[I + rh rh^T] / (4 pi rho r c2^3)."""
    rho, lam, mu = mat
    c1, c2 = _speeds(mat)
    rng = np.random.default_rng(5)
    r = rng.normal(size=(8, 3))
    rr = np.linalg.norm(r, axis=1)
    rh = r / rr[:, None]
    I = np.eye(3)
    P = rh[:, :, None] * rh[:, None, :]
    uk = ((1 / c1 ** 2 + 1 / c2 ** 2) * I + (1 / c2 ** 2 - 1 / c1 ** 2) * P) / (8 * math.pi * rho * rr[:, None, None])
    np.testing.assert_allclose(uk, K.kelvin_U(r, lam, mu), rtol=1e-13)
    s = 1e-9 * c2 / rr.max() * np.exp(0.4j)
    dp = (P - I) / (4 * math.pi * rho * rr[:, None, None] * c1 ** 3)
    ds = -(I + P) / (4 * math.pi * rho * rr[:, None, None] * c2 ** 3)
    np.testing.assert_allclose(K.dU_dc(r, s, rho, lam, mu, "p"), dp, rtol=0, atol=1e-8 * np.abs(dp).max())
    np.testing.assert_allclose(K.dU_dc(r, s, rho, lam, mu, "s"), ds, rtol=0, atol=1e-8 * np.abs(ds).max())


@pytest.mark.parametrize("mat", MATS)
@pytest.mark.parametrize("wave", ["p", "s"])
@pytest.mark.parametrize("zabs", [0.3, 2.5, 30.0])
def test_traction_speed_derivative_by_fd(mat, wave, zabs):
    """dT/dc_a, d(T - T0)/dc_a and dT0/dc_a against 4th-order central
    differences of T, T - T0 and kelvin_T in c_a (rho fixed)."""
    c1, c2 = _speeds(mat)
    rng = np.random.default_rng(13)
    r = rng.normal(size=(6, 3))
    n = rng.normal(size=(6, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    s = zabs * c2 / np.linalg.norm(r, axis=1).mean() * np.exp(0.6j)
    c = c1 if wave == "p" else c2
    h = 1e-4 * c

    def fd(f):
        return (-f(2 * h) + 8 * f(h) - 8 * f(-h) + f(-2 * h)) / (12 * h)
    m = lambda dc: _speed_perturbed(mat, wave, dc)                  # noqa: E731
    for dyn in (False, True):
        want = fd(lambda dc: K.T(r, n, s, *m(dc), dynamic=dyn))
        got = K.dT_dc(r, n, s, *mat, wave, dynamic=dyn)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-8 * np.abs(want).max())
    want = fd(lambda dc: K.kelvin_T(r, n, *m(dc)[1:]))
    got = K.dkelvin_T_dc(r, n, *mat, wave)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-8 * np.abs(want).max())


@pytest.mark.parametrize("mat", MATS)
@pytest.mark.parametrize("wave", ["p", "s"])
def test_traction_speed_derivative_static_limit(mat, wave):
    """s -> 0: dT/dc_a tends to dT0/dc_a = (dnu/dc_a) dT0/dnu, and the
    dynamic part vanishes."""
    c2 = _speeds(mat)[1]
    rng = np.random.default_rng(17)
    r = rng.normal(size=(8, 3))
    n = rng.normal(size=(8, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    s = 1e-7 * c2 / np.linalg.norm(r, axis=1).max() * np.exp(0.2j)
    d0 = K.dkelvin_T_dc(r, n, *mat, wave)
    np.testing.assert_allclose(K.dT_dc(r, n, s, *mat, wave), d0, rtol=0, atol=1e-6 * np.abs(d0).max())
    assert np.abs(K.dT_dc(r, n, s, *mat, wave, dynamic=True)).max() < 1e-6 * np.abs(d0).max()
