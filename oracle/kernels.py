"""Laplace-domain elastodynamic fundamental solutions (oracle, FP64).

The paper names the kernels U(r, s) and T(r, s) (Sec. 2.4, after Eq. (2.18);
Sec. 3.1, Eq. (3.9)) but never prints them.  They are written here from the
Laplace-transformed Navier equation (Eq. (2.1a) with d/dt -> s):

    U(r, s) = (1/mu) g2 I + 1/(rho s^2) grad grad (g1 - g2),
    g_a = exp(-s r / c_a) / (4 pi r),   c1, c2 from Eq. (2.2),

which solves mu Lap U + (lambda + mu) grad div U - rho s^2 U = -delta I.
With r = y - x, r = |r|, rh = r / r and h_a = exp(-s r / c_a) / r:

    U_ij = [A delta_ij + B rh_i rh_j] / (4 pi rho)
    A = h2 / c2^2 + (P2 - P1) / s^2,     P_a = (k_a r + 1) e^{-k_a r} / r^3
    B = (Q1 - Q2) / s^2,                 Q_a = (k_a^2 r^2 + 3 k_a r + 3) e^{-k_a r} / r^3

(k_a = s / c_a).  The traction kernel applies the traction operator of
Eq. (2.4) at y with the normal n = n(y) to the columns of U (column j is the
displacement due to a unit load in direction j); sigma from Eq. (2.5):

    4 pi T_ij = c2^2 (A' + B/r)(rh.n delta_ij + rh_i n_j)
              + 2 c2^2 (B' - 2B/r) rh.n rh_i rh_j
              + [(c1^2 - 2 c2^2)(A' + B' + 2B/r) + 2 c2^2 B/r] n_i rh_j

T_ij is traction component i due to the load direction j; the double layer
integrand of Eq. (2.9) is its transpose.  For |s| r / c2 < 1 the closed form
cancels; there the exact power series in z = s r / c2 (rc = c2 / c1) is used:

    A = 1/(r c2^2) sum_m (-z)^m [1/m! + (m+1)(rc^{m+2} - 1)/(m+2)!]
    B = 1/(r c2^2) sum_m (-z)^m (m+1)(m-1)(rc^{m+2} - 1)/(m+2)!

and A', B' follow term by term (d/dr of r^{m-1} = (m-1) r^{m-2}).
Pins: symmetry, conjugate symmetry in s, the static Kelvin limit, the
Navier residual by finite differences, traction by finite differences of U,
series/closed-form agreement (tests/test_oracle_kernels.py).  The wave-speed
derivatives dU/dc1, dU/dc2 (dU_dc) are pinned by finite differences of U in
c1, c2 and by the derivatives of the Kelvin solution written in c1, c2;
dT/dc1, dT/dc2 (dT_dc) and dT0/dc_a by finite differences of T and of
kelvin_T, and by their static limit.
"""
from __future__ import annotations

import math

import numpy as np

SERIES_Z = 1.0      # series branch where |s| r / c2 < SERIES_Z
SERIES_TERMS = 26


def wave_speeds(rho: float, lam: float, mu: float) -> tuple[float, float]:
    """Eq. (2.2): c1 = sqrt((lambda + 2 mu) / rho), c2 = sqrt(mu / rho)."""
    return math.sqrt((lam + 2.0 * mu) / rho), math.sqrt(mu / rho)


def _series_tables(c1: float, c2: float):
    rc = c2 / c1
    m = np.arange(SERIES_TERMS, dtype=np.float64)
    fact_m = np.array([math.factorial(int(k)) for k in m], dtype=np.float64)
    fact_m2 = np.array([math.factorial(int(k) + 2) for k in m], dtype=np.float64)
    pw = rc ** (m + 2.0) - 1.0
    a = 1.0 / fact_m + (m + 1.0) * pw / fact_m2
    b = (m + 1.0) * (m - 1.0) * pw / fact_m2
    return a, b, m


def coeffs(r, s, c1: float, c2: float, dynamic: bool = False):
    """A, B, A', B' of the kernel at distances r and frequencies s (arrays
    that broadcast together).

    With ``dynamic`` the static (s = 0) values are subtracted, giving the
    bounded remainder used next to a singular point."""
    r, s = np.broadcast_arrays(np.asarray(r, dtype=np.float64),
                               np.asarray(s, dtype=np.complex128))
    z = s * r / c2
    A = np.empty(r.shape, dtype=np.complex128)
    B = np.empty_like(A)
    dA = np.empty_like(A)
    dB = np.empty_like(A)
    ser = np.abs(z) < SERIES_Z
    cls = ~ser
    if np.any(ser):
        ta, tb, m = _series_tables(c1, c2)
        zs, rs = z[ser], r[ser]
        mz = np.power.outer(-zs, m)                      # (-z)^m
        start = 1 if dynamic else 0
        sa = (mz[:, start:] * ta[start:]).sum(-1)
        sb = (mz[:, start:] * tb[start:]).sum(-1)
        sda = (mz[:, start:] * (ta * (m - 1.0))[start:]).sum(-1)
        sdb = (mz[:, start:] * (tb * (m - 1.0))[start:]).sum(-1)
        k = 1.0 / (c2 * c2)
        A[ser] = k * sa / rs
        B[ser] = k * sb / rs
        dA[ser] = k * sda / rs ** 2
        dB[ser] = k * sdb / rs ** 2
    if np.any(cls):
        rr, ss = r[cls], s[cls]
        out = []
        for c in (c1, c2):
            kr = ss * rr / c
            e = np.exp(-kr)
            h = e / rr
            P = (kr + 1.0) * e / rr ** 3
            Q = (kr * kr + 3.0 * kr + 3.0) * e / rr ** 3
            R = -(kr ** 3 + 4.0 * kr * kr + 9.0 * kr + 9.0) * e / rr ** 4
            out.append((h, P, Q, R))
        (h1, P1, Q1, R1), (h2, P2, Q2, R2) = out
        Ac = h2 / c2 ** 2 + (P2 - P1) / ss ** 2
        Bc = (Q1 - Q2) / ss ** 2
        dAc = -rr * P2 / c2 ** 2 + Bc / rr
        dBc = (R1 - R2) / ss ** 2
        if dynamic:
            alpha = 0.5 * (1.0 / c1 ** 2 + 1.0 / c2 ** 2)
            beta = 0.5 * (1.0 / c2 ** 2 - 1.0 / c1 ** 2)
            Ac = Ac - alpha / rr
            Bc = Bc - beta / rr
            dAc = dAc + alpha / rr ** 2
            dBc = dBc + beta / rr ** 2
        A[cls], B[cls], dA[cls], dB[cls] = Ac, Bc, dAc, dBc
    return A, B, dA, dB


def U(rvec, s, rho: float, lam: float, mu: float, dynamic=False):
    """Displacement fundamental solution, shape (..., 3, 3), r = y - x; s is
    a scalar or an array broadcasting against rvec.shape[:-1]."""
    c1, c2 = wave_speeds(rho, lam, mu)
    rvec = np.asarray(rvec, dtype=np.float64)
    r = np.linalg.norm(rvec, axis=-1)
    rh = rvec / r[..., None]
    A, B, _, _ = coeffs(r, s, c1, c2, dynamic)
    rh = np.broadcast_to(rh, A.shape + (3,))
    eye = np.eye(3)
    return (A[..., None, None] * eye + B[..., None, None] * rh[..., :, None] * rh[..., None, :]) / (4.0 * math.pi * rho)


def dcoeffs_dc(r, s, c1: float, c2: float, wave: str):
    """dA/dc_a and dB/dc_a at fixed rho, a = 1 (wave "p") or 2 (wave "s").

    The wave speeds (Eq. (2.2)) enter A and B only through k_a = s / c_a in
    h_a, P_a, Q_a and through the explicit 1 / c2^2 of A.  With
    dk_a/dc_a = -k_a / c_a, dP_a/dk_a = -k_a e_a / r,
    dQ_a/dk_a = -k_a (1 + k_a r) e_a / r and k_a^2 / s^2 = 1 / c_a^2
    (e_a = exp(-k_a r)):

        dA/dc1 = -e1 / (r c1^3),            dB/dc1 = (1 + k1 r) e1 / (r c1^3)
        dA/dc2 = (k2 r - 1) e2 / (r c2^3),  dB/dc2 = -(1 + k2 r) e2 / (r c2^3)

    The 1 / s^2 factors cancel, so no series branch is needed at small |s| r."""
    r, s = np.broadcast_arrays(np.asarray(r, dtype=np.float64),
                               np.asarray(s, dtype=np.complex128))
    c = c1 if wave == "p" else c2
    kr = s * r / c
    e = np.exp(-kr) / (r * c ** 3)
    if wave == "p":
        return -e, (1.0 + kr) * e
    return (kr - 1.0) * e, -(1.0 + kr) * e


def dU_dc(rvec, s, rho: float, lam: float, mu: float, wave: str):
    """Derivative of U (shape (..., 3, 3)) with respect to the P-wave speed
    c1 (wave = "p") or the S-wave speed c2 (wave = "s") at fixed density:
    [dA/dc delta_ij + dB/dc rh_i rh_j] / (4 pi rho)."""
    c1, c2 = wave_speeds(rho, lam, mu)
    rvec = np.asarray(rvec, dtype=np.float64)
    r = np.linalg.norm(rvec, axis=-1)
    rh = rvec / r[..., None]
    A, B = dcoeffs_dc(r, s, c1, c2, wave)
    rh = np.broadcast_to(rh, A.shape + (3,))
    eye = np.eye(3)
    return (A[..., None, None] * eye + B[..., None, None] * rh[..., :, None] * rh[..., None, :]) / (4.0 * math.pi * rho)


def dcoeffs2_dc(r, s, c1: float, c2: float, wave: str, dynamic: bool = False):
    """c_a-derivatives (fixed rho) of A, B, A', B' and S3 = A' + B' + 2B/r,
    the coefficients of the traction kernel, from dcoeffs_dc by d/dr
    (e = exp(-k r), k = k_a, x = k r, c = c_a):

        wave p: A = -e/(r c^3),         B = (1 + x) e/(r c^3),
                A' = (1 + x) e/(r^2 c^3),  B' = -(1 + x + x^2) e/(r^2 c^3),
                S3 = (2 + 2x - x^2) e/(r^2 c^3)
        wave s: A = (x - 1) e/(r c^3),  B = -(1 + x) e/(r c^3),
                A' = (1 + x - x^2) e/(r^2 c^3), B' = (1 + x + x^2) e/(r^2 c^3),
                S3 = 0  (S3 depends on c1 only: -(1 + k1 r) e1/(c1^2 r^2)).

    ``dynamic`` subtracts the s = 0 values (the c-derivatives of the static
    coefficients), as coeffs does."""
    r, s = np.broadcast_arrays(np.asarray(r, dtype=np.float64),
                               np.asarray(s, dtype=np.complex128))
    c = c1 if wave == "p" else c2
    x = s * r / c
    e = np.exp(-x)
    em = np.expm1(-x) if dynamic else e       # e - 1 when the static part goes
    f1, f2 = 1.0 / (r * c ** 3), 1.0 / (r * r * c ** 3)
    if wave == "p":
        A = -em * f1
        B = (em + x * e) * f1
        Ap = (em + x * e) * f2
        Bp = -(em + (x + x * x) * e) * f2
        S3 = (2.0 * em + (2.0 * x - x * x) * e) * f2
    else:
        A = (x * e - em) * f1
        B = -(em + x * e) * f1
        Ap = (em + (x - x * x) * e) * f2
        Bp = (em + (x + x * x) * e) * f2
        S3 = np.zeros_like(A)
    return A, B, Ap, Bp, S3


def dT_dc(rvec, n, s, rho: float, lam: float, mu: float, wave: str, dynamic=False):
    """Derivative of T (same layout as T) with respect to c1 (wave "p") or c2
    (wave "s") at fixed density.  T's coefficients f1 = c2^2 (A' + B/r),
    f2 = 2 c2^2 (B' - 2B/r), f3 = (c1^2 - 2 c2^2) S3 + 2 c2^2 B/r are
    differentiated by the product rule, the A, B, A', B', S3 parts by
    dcoeffs2_dc.  ``dynamic``: the derivative of T(s) - T0."""
    c1, c2 = wave_speeds(rho, lam, mu)
    rvec = np.asarray(rvec, dtype=np.float64)
    n = np.broadcast_to(np.asarray(n, dtype=np.float64), rvec.shape)
    r = np.linalg.norm(rvec, axis=-1)
    rh = rvec / r[..., None]
    A, B, dA, dB = coeffs(r, s, c1, c2, dynamic)
    DA, DB, DAp, DBp, DS3 = dcoeffs2_dc(r, s, c1, c2, wave, dynamic)
    r, rh, n = (np.broadcast_to(a, A.shape + a.shape[r.ndim:]) for a in (r, rh, n))
    S3 = dA + dB + 2.0 * B / r
    c1s, c2s = c1 * c1, c2 * c2
    d1s, d2s = (2.0 * c1, 0.0) if wave == "p" else (0.0, 2.0 * c2)
    f1 = d2s * (dA + B / r) + c2s * (DAp + DB / r)
    f2 = 2.0 * d2s * (dB - 2.0 * B / r) + 2.0 * c2s * (DBp - 2.0 * DB / r)
    f3 = (d1s - 2.0 * d2s) * S3 + (c1s - 2.0 * c2s) * DS3 + 2.0 * d2s * B / r + 2.0 * c2s * DB / r
    rn = (rh * n).sum(-1)
    eye = np.eye(3)
    t = (f1[..., None, None] * (rn[..., None, None] * eye + rh[..., :, None] * n[..., None, :])
         + (f2 * rn)[..., None, None] * rh[..., :, None] * rh[..., None, :]
         + f3[..., None, None] * n[..., :, None] * rh[..., None, :])
    return t / (4.0 * math.pi)


def dnu_dc(rho: float, lam: float, mu: float, wave: str) -> float:
    """d nu / d c_a at fixed rho, nu = (c1^2 - 2 c2^2) / (2 (c1^2 - c2^2)):
    c1 c2^2 / (c1^2 - c2^2)^2 (wave p), -c1^2 c2 / (c1^2 - c2^2)^2 (wave s)."""
    c1, c2 = wave_speeds(rho, lam, mu)
    d = (c1 * c1 - c2 * c2) ** 2
    return c1 * c2 * c2 / d if wave == "p" else -c1 * c1 * c2 / d


def dkelvin_T_dnu(rvec, n, lam: float, mu: float):
    """d T0 / d nu: with T0 = -[g P + h Q] / (8 pi r^2), g = (1-2nu)/(1-nu),
    h = 1/(1-nu), P = rh.n I + rh n^T - n rh^T, Q = 3 rh.n rh rh^T:
    -[Q - P] / (8 pi (1-nu)^2 r^2)."""
    nu = lam / (2.0 * (lam + mu))
    rvec = np.asarray(rvec, dtype=np.float64)
    n = np.broadcast_to(np.asarray(n, dtype=np.float64), rvec.shape)
    r = np.linalg.norm(rvec, axis=-1)
    rh = rvec / r[..., None]
    rn = (rh * n).sum(-1)
    P = (rn[..., None, None] * np.eye(3) + rh[..., :, None] * n[..., None, :] - n[..., :, None] * rh[..., None, :])
    Q = 3.0 * rn[..., None, None] * rh[..., :, None] * rh[..., None, :]
    return -(Q - P) / (8.0 * math.pi * (1.0 - nu) ** 2 * (r ** 2)[..., None, None])


def dkelvin_T_dc(rvec, n, rho: float, lam: float, mu: float, wave: str):
    """d T0 / d c_a at fixed rho (T0 depends on the speeds through nu only)."""
    return dnu_dc(rho, lam, mu, wave) * dkelvin_T_dnu(rvec, n, lam, mu)


def lame_from_speeds(rho: float, c1: float, c2: float) -> tuple[float, float]:
    """Inverse of Eq. (2.2): mu = rho c2^2, lambda = rho (c1^2 - 2 c2^2)."""
    return rho * (c1 * c1 - 2.0 * c2 * c2), rho * c2 * c2


def T(rvec, n, s, rho: float, lam: float, mu: float, dynamic=False):
    """Traction fundamental solution T_ij (traction i at y with normal n due
    to a unit load in direction j at x), shape (..., 3, 3), r = y - x."""
    c1, c2 = wave_speeds(rho, lam, mu)
    rvec = np.asarray(rvec, dtype=np.float64)
    n = np.broadcast_to(np.asarray(n, dtype=np.float64), rvec.shape)
    r = np.linalg.norm(rvec, axis=-1)
    rh = rvec / r[..., None]
    A, B, dA, dB = coeffs(r, s, c1, c2, dynamic)
    r, rh, n = (np.broadcast_to(a, A.shape + a.shape[r.ndim:]) for a in (r, rh, n))
    rn = (rh * n).sum(-1)
    c1s, c2s = c1 * c1, c2 * c2
    f1 = c2s * (dA + B / r)
    f2 = 2.0 * c2s * (dB - 2.0 * B / r)
    f3 = (c1s - 2.0 * c2s) * (dA + dB + 2.0 * B / r) + 2.0 * c2s * B / r
    eye = np.eye(3)
    t = (f1[..., None, None] * (rn[..., None, None] * eye + rh[..., :, None] * n[..., None, :])
         + (f2 * rn)[..., None, None] * rh[..., :, None] * rh[..., None, :]
         + f3[..., None, None] * n[..., :, None] * rh[..., None, :])
    return t / (4.0 * math.pi)


def kelvin_U(rvec, lam: float, mu: float):
    """Static Kelvin solution [(3 - 4 nu) I + rh rh^T] / (16 pi mu (1 - nu) r)."""
    nu = lam / (2.0 * (lam + mu))
    rvec = np.asarray(rvec, dtype=np.float64)
    r = np.linalg.norm(rvec, axis=-1)
    rh = rvec / r[..., None]
    out = (3.0 - 4.0 * nu) * np.eye(3) + rh[..., :, None] * rh[..., None, :]
    return out / (16.0 * math.pi * mu * (1.0 - nu) * r[..., None, None])


def kelvin_T(rvec, n, lam: float, mu: float):
    """Static Kelvin traction kernel
    -[rh.n((1-2nu) I + 3 rh rh^T) + (1-2nu)(rh n^T - n rh^T)] / (8 pi (1-nu) r^2)."""
    nu = lam / (2.0 * (lam + mu))
    rvec = np.asarray(rvec, dtype=np.float64)
    n = np.broadcast_to(np.asarray(n, dtype=np.float64), rvec.shape)
    r = np.linalg.norm(rvec, axis=-1)
    rh = rvec / r[..., None]
    rn = (rh * n).sum(-1)
    a = 1.0 - 2.0 * nu
    out = (rn[..., None, None] * (a * np.eye(3) + 3.0 * rh[..., :, None] * rh[..., None, :])
           + a * (rh[..., :, None] * n[..., None, :] - n[..., :, None] * rh[..., None, :]))
    return -out / (8.0 * math.pi * (1.0 - nu) * (r ** 2)[..., None, None])
