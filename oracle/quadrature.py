"""Quadrature rules on flat triangles (oracle, FP64, test infrastructure).

The paper fixes no quadrature orders; it names Duffy's transformation for the
weakly singular collocation integrals (Sec. 2.3, last paragraph).  Reading
used on both sides of the parity tests:

* Gauss-Legendre nodes on [0, 1] by Newton's method on P_n (no tables).
* Regular integrals: collapsed (conical product) n x n rule on the reference
  triangle, xi = u, eta = v (1 - u), weight w_u w_v (1 - u); exact for
  polynomials of total degree <= 2n - 2.
* Order by distance: n = 3 if |x - centroid| >= 4 h, n = 5 if >= 2 h,
  n = 8 if >= h, else n = 16, with h the longest edge of the element.  The
  comparisons carry a relative band of 1e-12 (dist >= D h (1 - 1e-12)) so
  that distances lying exactly on a threshold in exact arithmetic (regular
  grids) give the same order whatever the rounding of dist and h.
* Singular (the collocation point lies on the closed element): split the
  element into sub-triangles with apex at the point and use the Duffy map
  y = A + u ((B - A) + v (C - B)), dy = 2 |ABC| u du dv, 16 x 16
  Gauss-Legendre (the v integrand 1/|B - A + v (C - B)| has complex poles
  close to [0, 1] for the flat sub-triangles about a centroid; 8 points
  leave a 1e-4 error there).
"""
from __future__ import annotations

import numpy as np

N_FAR, N_MID, N_NEAR, N_CLOSE, N_SING = 3, 5, 8, 16, 16
D_FAR, D_MID, D_NEAR = 4.0, 2.0, 1.0


def gauss_legendre01(n: int) -> tuple[np.ndarray, np.ndarray]:
    """n-point Gauss-Legendre nodes and weights on [0, 1] (Newton on P_n)."""
    x = np.cos(np.pi * (np.arange(1, n + 1) - 0.25) / (n + 0.5))
    for _ in range(100):
        p0, p1 = np.ones_like(x), x.copy()
        for k in range(2, n + 1):
            p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
        dp = n * (x * p1 - p0) / (x * x - 1.0)
        dx = p1 / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    p0, p1 = np.ones_like(x), x.copy()
    for k in range(2, n + 1):
        p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
    dp = n * (x * p1 - p0) / (x * x - 1.0)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    order = np.argsort(x)
    return 0.5 * (x[order] + 1.0), 0.5 * w[order]


def triangle_rule(n: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Collapsed n x n rule on the reference triangle {xi, eta >= 0,
    xi + eta <= 1}.  Returns (xi, eta, w) with sum(w) = 1/2."""
    g, gw = gauss_legendre01(n)
    u, v = np.meshgrid(g, g, indexing="ij")
    wu, wv = np.meshgrid(gw, gw, indexing="ij")
    xi = u.ravel()
    eta = (v * (1.0 - u)).ravel()
    w = (wu * wv * (1.0 - u)).ravel()
    return xi, eta, w


def order_for(dist: float, h: float) -> int:
    """Regular-rule order n from the distance ratio dist / h."""
    band = 1.0 - 1e-12
    if dist >= D_FAR * h * band:
        return N_FAR
    if dist >= D_MID * h * band:
        return N_MID
    if dist >= D_NEAR * h * band:
        return N_NEAR
    return N_CLOSE


def duffy_points(A, B, C, n: int | None = None):
    """Points and weights of the Duffy rule on triangle (A; B, C) with the
    singular apex A: returns (y (q,3), w (q,)), sum(w) = area(ABC)."""
    A, B, C = (np.asarray(p, dtype=np.float64) for p in (A, B, C))
    n = N_SING if n is None else n
    g, gw = gauss_legendre01(n)
    u, v = np.meshgrid(g, g, indexing="ij")
    wu, wv = np.meshgrid(gw, gw, indexing="ij")
    u, v, wu, wv = u.ravel(), v.ravel(), wu.ravel(), wv.ravel()
    y = A + u[:, None] * ((B - A) + v[:, None] * (C - B))
    area2 = np.linalg.norm(np.cross(B - A, C - A))
    return y, wu * wv * area2 * u
