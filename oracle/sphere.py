"""Closed-form Laplace-domain response of a solid elastic sphere under a
uniform surface pressure (oracle, FP64, test infrastructure).

Physics pin of the assembled operators: the interior Neumann problem of
Eq. (2.12) (rows at nodes) with t = -p n is (C + K) u = V t.  Written from
the Laplace-transformed Navier equation (Eq. (2.1a)): a radial field is
irrotational, u = grad phi with Lap phi = k^2 phi, k = s / c1; regular at
the centre phi = A f(r), f = sinh(k r) / r.  Then u_r = A f'(r),
sigma_rr = A (lambda k^2 f + 2 mu f''), f'' = k^2 f - 2 f' / r, and
sigma_rr(a) = -p fixes A.  Static limit: u_r(a) = -p a / (3 lambda + 2 mu).
"""
from __future__ import annotations

import numpy as np


def radial_displacement(a: float, s: complex, p: complex, rho: float, lam: float, mu: float) -> complex:
    c1 = np.sqrt((lam + 2.0 * mu) / rho)
    k = s / c1
    f = np.sinh(k * a) / a
    df = (k * a * np.cosh(k * a) - np.sinh(k * a)) / a ** 2
    ddf = k * k * f - 2.0 * df / a
    A = -p / (lam * k * k * f + 2.0 * mu * ddf)
    return A * df


def bem_neumann_sphere(op_v, op_k, s: complex, p: complex = 1.0) -> np.ndarray:
    """Solve (C + K) u = V t, t = -p n on every element, by a dense LU
    (numpy.linalg.solve); returns u (n_nodes, 3)."""
    geo = op_v.geo
    t = -p * geo.normal                                        # (E, 3)
    V = op_v.dense(np.array([s]))[:, :, 0]                     # (nN, E, 3, 3)
    CK = op_k.dense(np.array([s]))[:, :, 0]                    # (nN, nN, 3, 3)
    rhs = np.einsum("ieab,eb->ia", V, t).reshape(-1)
    n = CK.shape[0]
    A = CK.transpose(0, 2, 1, 3).reshape(3 * n, 3 * n)
    return np.linalg.solve(A, rhs).reshape(n, 3)
