"""Pins of oracle/stokes.py (the analytic field of the unit-cube study,
Sec. 4.1 and Appendix A) against facts that do not rest on its formulas:
Gauss-Legendre quadrature of the integral term; the Navier equation
rho u_tt = (lam + mu) grad div u + mu Lap u by finite differences; the
complex-step gradient against central differences; the Laplace transform
of the field (numerical quadrature in t) against the oracle's own
Laplace-domain kernels U(r, s) and T(r, n, s) times the pulse's
transform; rest at t = 0 on the cube."""
import numpy as np
import pytest

import synthetic as syn
from oracle import kernels, stokes

MAT = syn.PAPER_CUBE_MATERIAL                 # rho 1, c1 1, c2 sqrt(1/2)
SRC = stokes.CUBE_SOURCE
P, D, A_, TC = np.array(SRC["p"]), np.array(SRC["d"]), SRC["a"], SRC["tc"]
PTS = np.array([[0.5, 0.1, -0.2], [-0.5, 0.5, 0.5], [0.0, -0.5, 0.3], [0.2, 0.3, 0.5]])


def _u(x, t):
    return stokes.displacement(x, t, MAT, P, D, A_, TC)


def test_integral_term_vs_quadrature():
    c1, c2 = 1.0, np.sqrt(0.5)
    xg, wg = np.polynomial.legendre.leggauss(80)
    lo, hi = 1.0 / c1, 1.0 / c2
    for r in (0.3, 1.4, 2.5):
        for t in (0.2, 1.7, 2.9, 4.0):
            lam = 0.5 * (hi - lo) * xg + 0.5 * (hi + lo)
            q = 0.5 * (hi - lo) * (wg * lam * stokes.pulse(t - lam * r, A_, TC)).sum()
            assert abs(stokes.integral_term(r, t, c1, c2, A_, TC) - q) <= 1e-13 * max(1.0, abs(q))


def test_navier_equation_by_differences():
    rho, lam, mu = MAT
    h, k = 2e-3, 2e-3
    R, S = [], []
    for x in PTS:
        for t in (1.5, 2.2, 2.8):
            utt = (_u(x, t + k) - 2 * _u(x, t) + _u(x, t - k)) / k ** 2
            lap = np.zeros(3)
            H = np.zeros((3, 3, 3))                       # H[i, a, b] = d2 u_i / dx_a dx_b
            for a_ in range(3):
                for b_ in range(3):
                    ea, eb = np.eye(3)[a_] * h, np.eye(3)[b_] * h
                    H[:, a_, b_] = (_u(x + ea + eb, t) - _u(x + ea - eb, t) - _u(x - ea + eb, t)
                                    + _u(x - ea - eb, t)) / (4 * h * h)
            lap = H[:, 0, 0] + H[:, 1, 1] + H[:, 2, 2]
            graddiv = np.array([H[0, 0, a_] + H[1, 1, a_] + H[2, 2, a_] for a_ in range(3)])
            R.append(rho * utt - (lam + mu) * graddiv - mu * lap)
            S.append(rho * utt)
    assert np.abs(R).max() <= 1e-4 * np.abs(S).max(), (np.abs(R).max(), np.abs(S).max())


def test_complex_step_gradient_vs_differences():
    h = 1e-5
    E, S = [], []
    for x in PTS:
        for t in (1.2, 2.0, 2.6):
            G = stokes.gradient(x, t, MAT, P, D, A_, TC)
            Gd = np.stack([(_u(x + h * e, t) - _u(x - h * e, t)) / (2 * h) for e in np.eye(3)], axis=-1)
            E.append(np.abs(G - Gd).max())
            S.append(np.abs(G).max())
    assert max(E) <= 1e-8 * max(S), (max(E), max(S))


@pytest.mark.parametrize("s", [1.5, 2.0 + 3.0j, 0.8 - 1.5j])
def test_laplace_transform_matches_kernels(s):
    """u^ = U d F^ needs a causal source pulse: delay 1.5 s (F(0) ~ 2e-10)
    instead of the cube's 0.55 s (there the source's pulse, not the field
    on the cube, is already under way at t = 0)."""
    rho, lam, mu = MAT
    tc = 1.5
    t = np.linspace(0.0, 12.0, 24001)
    w = np.full(len(t), t[1] - t[0])
    w[0] = w[-1] = 0.5 * w[0]                                 # trapezoid (integrand smooth, ~0 at both ends)
    es = np.exp(-s * t) * w
    Fh = (es * stokes.pulse(t, A_, tc)).sum()
    n = np.array([0.0, 0.6, 0.8])
    for x in PTS:
        uh = (es[:, None] * stokes.displacement(x, t, MAT, P, D, A_, tc)).sum(0)
        ref = kernels.U(x - P, s, rho, lam, mu) @ D * Fh
        assert np.abs(uh - ref).max() <= 1e-9 * np.abs(ref).max(), (x, uh, ref)
        th = (es[:, None] * stokes.traction(x, n, t, MAT, P, D, A_, tc)).sum(0)
        tref = kernels.T(x - P, n, s, rho, lam, mu) @ D * Fh
        assert np.abs(th - tref).max() <= 1e-9 * np.abs(tref).max(), (x, th, tref)


def test_rest_at_time_zero_on_the_cube():
    xyz, tri = syn.paper_cube(2)
    peak = max(np.abs(_u(xyz, t)).max() for t in np.linspace(0, 3, 31))
    assert np.abs(_u(xyz, 0.0)).max() <= 1e-12 * peak


def test_dirichlet_formulation_converges_in_frequency_domain():
    """Collocation at the element midpoints, V t^ = (C + K) u^ with the exact
    Laplace-domain data u^ = U d, t^ = T d of the cube's source (the
    oracle's kernels, pinned above against the analytic field): solving for
    t^ gets closer to the exact traction from level 1 to level 2 of the
    paper's cube (first order expected for piecewise constant traction)."""
    from oracle import bem
    rho, lam, mu = MAT
    s = 1.5
    errs = []
    for lev in (1, 2):
        xyz, tri = syn.paper_cube(lev)
        V = bem.to_matrix(bem.Operator(xyz, tri, MAT, bem.ROWS_CENTROIDS, bem.KERNEL_SL).dense(np.array([s]))[:, :, 0])
        A = bem.to_matrix(bem.Operator(xyz, tri, MAT, bem.ROWS_CENTROIDS, bem.KERNEL_DL).dense(np.array([s]))[:, :, 0])
        c = xyz[tri].mean(1)
        nrm = np.cross(xyz[tri[:, 1]] - xyz[tri[:, 0]], xyz[tri[:, 2]] - xyz[tri[:, 0]])
        nrm /= np.linalg.norm(nrm, axis=1)[:, None]
        uh = kernels.U(xyz - P, s, rho, lam, mu) @ D
        th = kernels.T(c - P, nrm, s, rho, lam, mu) @ D
        t = np.linalg.solve(V, A @ uh.reshape(-1)).reshape(-1, 3)
        errs.append(np.linalg.norm(t - th) / np.linalg.norm(th))
    assert errs[0] < 0.3 and errs[1] < 0.6 * errs[0], errs
