"""Pins of the oracle's quadrature (closed forms, library rules)."""
import math

import numpy as np
import pytest

from oracle import bem, quadrature as quad


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12])
def test_gauss_legendre_matches_library(n):
    x, w = quad.gauss_legendre01(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(x, 0.5 * (xr + 1.0), atol=1e-15)
    np.testing.assert_allclose(w, 0.5 * wr, atol=1e-15)


@pytest.mark.parametrize("n", [3, 5, 8])
def test_triangle_rule_exactness(n):
    xi, eta, w = quad.triangle_rule(n)
    assert abs(w.sum() - 0.5) < 1e-15
    for p in range(2 * n - 1):
        for q in range(2 * n - 1 - p):
            exact = math.factorial(p) * math.factorial(q) / math.factorial(p + q + 2)
            got = (w * xi ** p * eta ** q).sum()
            assert abs(got - exact) < 1e-14 * max(1.0, exact / 1e-3), (p, q)


def _inv_r_apex(A, B, C):
    """int_{ABC} 1/|y - A| dA in closed form: in polar coordinates about A
    the integral is int R(theta) dtheta, R = h / cos(phi) along the edge BC,
    whose primitive is h * asinh(tan(phi)) = h * asinh(t / h)."""
    t = (C - B) / np.linalg.norm(C - B)
    F = B + ((A - B) @ t) * t
    h = np.linalg.norm(F - A)
    tb, tc = (B - F) @ t, (C - F) @ t
    return h * (math.asinh(tc / h) - math.asinh(tb / h))


def test_duffy_inverse_distance_closed_form():
    rng = np.random.default_rng(3)
    base = np.array([[0, 0, 0], [1, 0, 0], [0.5, 0.85, 0]])
    for _ in range(6):
        A, B, C = base + 0.12 * rng.normal(size=(3, 3))
        exact = abs(_inv_r_apex(A, B, C))
        errs = []
        for n in (8, 16):
            y, w = quad.duffy_points(A, B, C, n)
            errs.append(abs((w / np.linalg.norm(y - A, axis=1)).sum() - exact) / exact)
        assert errs[1] < 1e-8 and errs[1] <= errs[0] + 1e-15


def test_duffy_area():
    A, B, C = np.array([0., 0, 0]), np.array([2., 0, 0]), np.array([0.3, 1.5, 0])
    _, w = quad.duffy_points(A, B, C)
    assert abs(w.sum() - 1.5) < 1e-14


def test_cpv_closed_form_vs_polar_quadrature():
    """CPV int_e rh / r^2 dA = int_0^{2 pi} e(theta) ln R(theta) dtheta, the
    right side by brute-force quadrature over theta."""
    xyz = np.array([[0., 0, 0], [1.3, 0.1, 0], [0.2, 0.9, 0]])
    geo = bem.Geometry(xyz, np.array([[0, 1, 2]]))
    x = np.array([0.45, 0.3, 0.0])
    G = geo.cpv_rh_over_r2(0, x)
    # brute force: R(theta) = distance from x to the boundary along e(theta)
    th = (np.arange(200000) + 0.5) * 2 * np.pi / 200000
    d = np.stack([np.cos(th), np.sin(th), 0 * th], 1)
    R = np.full(len(th), np.inf)
    P = xyz
    for a in range(3):
        p0, p1 = P[a], P[(a + 1) % 3]
        e = p1 - p0
        # solve x + R d = p0 + u e
        M = np.stack([d[:, :2], np.broadcast_to(-e[:2], (len(th), 2))], 2)
        rhs = np.broadcast_to((p0 - x)[:2], (len(th), 2))
        sol = np.linalg.solve(M, rhs[..., None])[..., 0]
        ok = (sol[:, 1] >= -1e-12) & (sol[:, 1] <= 1 + 1e-12) & (sol[:, 0] > 0)
        R = np.where(ok, np.minimum(R, sol[:, 0]), R)
    brute = (d * np.log(R)[:, None]).sum(0) * (2 * np.pi / len(th))
    np.testing.assert_allclose(G, brute, atol=1e-8)
