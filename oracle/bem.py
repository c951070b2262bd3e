"""Collocation BEM matrices at complex frequencies (oracle, FP64).

Follows the paper's collocation discretisation (Sec. 2.3, Eqs. (2.11)-(2.15)):
flat triangles; P0 traction (columns = elements) for the single layer V and
P1 displacement (columns = nodes) for the double layer K; collocation points
at element midpoints (Dirichlet rows) or at nodes (Neumann rows).  The
Laplace-domain entries replace the time-domain kernels by U(r, s), T(r, s)
(Sec. 2.4, Eq. (2.17) and after):

    V[i, e](s)  = int_e U(y - x_i, s) dy                        (3 x 3)
    K[i, j](s)  = sum_{e ni j} int_e T(x_i, y, s)^T phi_j(y) dy  (3 x 3)

The double-layer operator returned here is C + K (the integral-free term of
Eq. (2.7) included), the matrix that multiplies the displacement in the
Neumann rows of Eq. (2.12).  Readings of what the paper leaves open:

* Index swap in Eq. (2.15) (U*(y_i - x)) read as U(y - x_i): x_i is the
  collocation point, y the integration variable.
* Centroid rows: C = I/2 (smooth point of a flat element), so
  C[i, j] = I/6 for the three vertices j of element i; the strongly singular
  part of the own element is a Cauchy principal value, evaluated in closed
  form from CPV int_e rh / r^2 dA (polar coordinates, x_i inside e).
* Node rows: C(x_i) depends on the solid angle (Sec. 2.2); the static
  diagonal block is fixed by the rigid-body identity
  (C + K_0)[i, i] = -sum_{j != i} K_0[i, j], the frequency-dependent rest
  T(s) - T_0 is bounded and integrated by the Duffy rule.
* T_0 is the static Kelvin traction kernel.

Frequencies: uniform BDF2 convolution quadrature (the configuration's time
grid), s_k = delta(zeta_k) / dt, delta(zeta) = (1 - zeta) + (1 - zeta)^2 / 2,
zeta_k = lam_c exp(-2 pi i k / (N + 1)), lam_c = (1e-10)^(1 / (2N)); the
paper's conjugate-pair property (Sec. 4.1, Fig. circle) holds.
"""
from __future__ import annotations

import math

import numpy as np

from . import kernels, quadrature as quad

ROWS_CENTROIDS, ROWS_NODES = "centroids", "nodes"
KERNEL_SL, KERNEL_DL = "sl", "dl"
# wave-speed derivatives of the single layer at fixed density: dV/dc1 (P
# wave) and dV/dc2 (S wave); integrand dU/dc_a, same columns and quadrature
KERNEL_SL_DCP, KERNEL_SL_DCS = "sl_dcp", "sl_dcs"
SL_KINDS = (KERNEL_SL, KERNEL_SL_DCP, KERNEL_SL_DCS)
# and of the double layer C + K: integrands dT/dc_a, static parts dT0/dc_a,
# the CPV coefficient differentiated through nu, no free term (C = I/2 at a
# smooth point does not depend on the speeds; node rows: rigid-body identity)
KERNEL_DL_DCP, KERNEL_DL_DCS = "dl_dcp", "dl_dcs"
WAVE = {KERNEL_SL_DCP: "p", KERNEL_SL_DCS: "s", KERNEL_DL_DCP: "p", KERNEL_DL_DCS: "s"}


def freqs_bdf2(N: int, dt: float, K: int | None = None) -> np.ndarray:
    """s_k, k = 0..K-1, of BDF2 CQ with L = N + 1 points on the circle."""
    L = N + 1
    K = L if K is None else K
    lam = (1e-10) ** (1.0 / (2 * N))
    k = np.arange(K)
    zeta = lam * np.exp(-2j * np.pi * k / L)
    return ((1.0 - zeta) + 0.5 * (1.0 - zeta) ** 2) / dt


class Geometry:
    """Element geometry of a flat-triangle surface mesh (Eq. (2.10))."""

    def __init__(self, xyz, tri):
        self.xyz = np.asarray(xyz, dtype=np.float64)
        self.tri = np.asarray(tri, dtype=np.int64)
        P = self.xyz[self.tri]                        # (E, 3, 3)
        self.P = P
        cr = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
        nrm = np.linalg.norm(cr, axis=1)
        self.area = 0.5 * nrm
        self.normal = cr / nrm[:, None]
        self.centroid = P.mean(axis=1)
        edges = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 1], P[:, 0] - P[:, 2]], 1)
        self.h = np.linalg.norm(edges, axis=2).max(axis=1)
        self.n_nodes = len(self.xyz)
        self.n_tris = len(self.tri)
        self.node_elems = [[] for _ in range(self.n_nodes)]
        for e, t in enumerate(self.tri):
            for a in t:
                self.node_elems[a].append(e)

    def rows(self, kind):
        return self.centroid if kind == ROWS_CENTROIDS else self.xyz

    def n_cols(self, kernel):
        return self.n_tris if kernel in SL_KINDS else self.n_nodes

    def barycentric(self, e, y):
        """Barycentric coordinates (phi_0, phi_1, phi_2) of points y on e."""
        P0, P1, P2 = self.P[e]
        n = np.cross(P1 - P0, P2 - P0)
        nn = n @ n
        d = y - P0
        l1 = np.cross(d, P2 - P0) @ n / nn
        l2 = np.cross(P1 - P0, d) @ n / nn
        return np.stack([1.0 - l1 - l2, l1, l2], axis=-1)

    def regular_points(self, e, n):
        xi, eta, w = quad.triangle_rule(n)
        P0, P1, P2 = self.P[e]
        y = P0 + xi[:, None] * (P1 - P0) + eta[:, None] * (P2 - P0)
        phi = np.stack([1.0 - xi - eta, xi, eta], axis=-1)
        return y, w * 2.0 * self.area[e], phi

    def singular_points(self, e, x):
        """Duffy points for the collocation point x on the closed element e
        (a vertex of e, or its centroid)."""
        P = self.P[e]
        vert = [a for a in range(3) if np.array_equal(P[a], x)]
        if vert:
            a = vert[0]
            subs = [(P[a], P[(a + 1) % 3], P[(a + 2) % 3])]
        else:
            subs = [(x, P[0], P[1]), (x, P[1], P[2]), (x, P[2], P[0])]
        ys, ws = [], []
        for A, B, C in subs:
            y, w = quad.duffy_points(A, B, C)
            ys.append(y)
            ws.append(w)
        y = np.concatenate(ys)
        return y, np.concatenate(ws), self.barycentric(e, y)

    def cpv_rh_over_r2(self, e, x):
        """CPV int_e rh / r^2 dA for x inside the flat element e: sum over the
        sub-triangles (x; P_a, P_b) of int e(phi) ln R(phi) dphi in closed
        form, phi measured from the foot of the perpendicular on edge ab."""
        P = self.P[e]
        G = np.zeros(3)
        for a in range(3):
            Pa, Pb = P[a], P[(a + 1) % 3]
            t = (Pb - Pa) / np.linalg.norm(Pb - Pa)
            F = Pa + ((x - Pa) @ t) * t                 # foot of perpendicular
            h = np.linalg.norm(F - x)
            e0 = (F - x) / h
            ta, tb = (Pa - F) @ t, (Pb - F) @ t
            Ra, Rb = math.hypot(h, ta), math.hypot(h, tb)

            def prim0(tt, RR):     # int cos(phi) ln(h / cos phi) dphi
                return (tt / RR) * (math.log(RR) + 1.0) - math.asinh(tt / h)

            def prim1(tt, RR):     # int sin(phi) ln(h / cos phi) dphi
                return -(h / RR) * (math.log(RR) + 1.0)

            G += e0 * (prim0(tb, Rb) - prim0(ta, Ra)) + t * (prim1(tb, Rb) - prim1(ta, Ra))
        return G


def _on_element(geo: Geometry, kind, i, e):
    if kind == ROWS_CENTROIDS:
        return i == e
    return i in geo.tri[e]


class Operator:
    """Dense collocation V or C + K at a list of frequencies; with kernel
    KERNEL_SL_DCP / KERNEL_SL_DCS the wave-speed derivative dV/dc1 / dV/dc2
    of the single layer (same quadrature, integrand kernels.dU_dc), with
    KERNEL_DL_DCP / KERNEL_DL_DCS d(C + K)/dc1, d(C + K)/dc2 (integrands
    kernels.dT_dc and dkelvin_T_dc)."""

    def __init__(self, xyz, tri, material, rows=ROWS_NODES, kernel=KERNEL_SL):
        self.geo = Geometry(xyz, tri)
        self.rho, self.lam, self.mu = material
        self.rows_kind, self.kernel = rows, kernel
        self.x = self.geo.rows(rows)
        self.n_rows = len(self.x)
        self.n_cols = self.geo.n_cols(kernel)

    # ---- integrands ------------------------------------------------------
    def _U(self, r, s, dynamic=False):
        if self.kernel == KERNEL_SL_DCP:
            return kernels.dU_dc(r, s, self.rho, self.lam, self.mu, "p")
        if self.kernel == KERNEL_SL_DCS:
            return kernels.dU_dc(r, s, self.rho, self.lam, self.mu, "s")
        return kernels.U(r, s, self.rho, self.lam, self.mu, dynamic)

    def _TT(self, r, n, s, dynamic=False):
        """Transposed traction kernel T^T (double-layer integrand)."""
        if self.kernel in (KERNEL_DL_DCP, KERNEL_DL_DCS):
            t = kernels.dT_dc(r, n, s, self.rho, self.lam, self.mu, WAVE[self.kernel], dynamic)
        else:
            t = kernels.T(r, n, s, self.rho, self.lam, self.mu, dynamic)
        return np.swapaxes(t, -1, -2)

    def _T0T(self, r, n):
        if self.kernel in (KERNEL_DL_DCP, KERNEL_DL_DCS):
            t = kernels.dkelvin_T_dc(r, n, self.rho, self.lam, self.mu, WAVE[self.kernel])
        else:
            t = kernels.kelvin_T(r, n, self.lam, self.mu)
        return np.swapaxes(t, -1, -2)

    # ---- element integrals -------------------------------------------------
    def _elem_points(self, i, e):
        x = self.x[i]
        if _on_element(self.geo, self.rows_kind, i, e):
            return True, self.geo.singular_points(e, x)
        n = quad.order_for(float(np.linalg.norm(x - self.geo.centroid[e])), float(self.geo.h[e]))
        return False, self.geo.regular_points(e, n)

    def v_elem(self, i, e, s):
        """V[i, e] at frequencies s (K,) -> (K, 3, 3)."""
        _, (y, w, _) = self._elem_points(i, e)
        r = y - self.x[i]
        Uq = self._U(r[None], np.asarray(s)[:, None])            # (K, q, 3, 3)
        return np.einsum("q,kqab->kab", w, Uq)

    def k_elem(self, i, e, s):
        """Contributions of element e to the C + K row i at frequencies s:
        (K, 3 local vertices, 3, 3).  For node rows the static part of the
        diagonal (local vertex == i) is left out (rigid-body fix-up)."""
        s = np.asarray(s)
        geo, x = self.geo, self.x[i]
        sing, (y, w, phi) = self._elem_points(i, e)
        r = y - x
        n = geo.normal[e]
        out = np.zeros((len(s), 3, 3, 3), dtype=np.complex128)
        if not sing:
            Tq = self._TT(r[None], n, s[:, None])                 # (K, q, 3, 3)
            return np.einsum("q,qa,kqbc->kabc", w, phi, Tq)
        Tdyn = self._TT(r[None], n, s[:, None], dynamic=True)    # T(s) - T0
        T0 = self._T0T(r, n)                                      # (q, 3, 3)
        if self.rows_kind == ROWS_NODES:
            for a in range(3):
                if geo.tri[e, a] == i:
                    out[:, a] = np.einsum("q,q,kqbc->kbc", w, phi[:, a], Tdyn)
                else:
                    out[:, a] = np.einsum("q,q,kqbc->kbc", w, phi[:, a], Tdyn) \
                        + np.einsum("q,q,qbc->bc", w, phi[:, a], T0)[None]
            return out
        # centroid row on its own element: free term + CPV + Duffy remainders
        nu = self.lam / (2.0 * (self.lam + self.mu))
        G = geo.cpv_rh_over_r2(e, x)
        # CPV int T0^T: T0^T_bc = -(1-2nu)(rh_c n_b - n_c rh_b) / (8 pi (1-nu) r^2)
        cpv = -(1.0 - 2.0 * nu) * (np.outer(n, G) - np.outer(G, n)) / (8.0 * math.pi * (1.0 - nu))
        free = np.eye(3) / 6.0
        if self.kernel in (KERNEL_DL_DCP, KERNEL_DL_DCS):
            # d/dnu of -(1-2nu)/(1-nu) is 1/(1-nu)^2; the free term I/2 is fixed
            dnu = kernels.dnu_dc(self.rho, self.lam, self.mu, WAVE[self.kernel])
            cpv = dnu * (np.outer(n, G) - np.outer(G, n)) / (8.0 * math.pi * (1.0 - nu) ** 2)
            free = np.zeros((3, 3))
        for a in range(3):
            out[:, a] = (np.einsum("q,q,kqbc->kbc", w, phi[:, a], Tdyn)
                         + np.einsum("q,q,qbc->bc", w, phi[:, a] - 1.0 / 3.0, T0)[None]
                         + (cpv / 3.0 + free)[None])
        return out

    def _regular_groups(self, i, elems):
        """Regular (non-singular) elements of row i grouped by rule order:
        yields (elems, y (E, q, 3), w (E, q), phi (q, 3))."""
        geo, x = self.geo, self.x[i]
        elems = np.asarray(elems, dtype=np.int64)
        if len(elems) == 0:
            return
        dist = np.linalg.norm(geo.centroid[elems] - x, axis=1)
        order = np.array([quad.order_for(float(d), float(h)) for d, h in zip(dist, geo.h[elems])])
        for n in sorted(set(order.tolist())):
            es = elems[order == n]
            xi, eta, w = quad.triangle_rule(n)
            P = geo.P[es]
            y = P[:, None, 0] + xi[None, :, None] * (P[:, None, 1] - P[:, None, 0]) \
                + eta[None, :, None] * (P[:, None, 2] - P[:, None, 0])
            ww = w[None, :] * 2.0 * geo.area[es][:, None]
            phi = np.stack([1.0 - xi - eta, xi, eta], axis=-1)
            yield es, y, ww, phi

    def rigid_body_diag(self, i):
        """-sum_{j != i} K_0[i, j] for a node row i (static Kelvin kernel)."""
        geo, x = self.geo, self.x[i]
        acc = np.zeros((3, 3))
        sing = [e for e in geo.node_elems[i]]
        for e in sing:
            y, w, phi = geo.singular_points(e, x)
            a = int(np.nonzero(geo.tri[e] == i)[0][0])
            acc += np.einsum("q,qbc->bc", w * (1.0 - phi[:, a]), self._T0T(y - x, geo.normal[e]))
        rest = np.setdiff1d(np.arange(geo.n_tris), sing)
        for es, y, w, _ in self._regular_groups(i, rest):
            T0 = self._T0T(y - x, geo.normal[es][:, None, :])
            acc += np.einsum("eq,eqbc->bc", w, T0)
        return -acc

    # ---- blocks ------------------------------------------------------------
    def block(self, rows, cols, s):
        """Dense sub-tensor C[rows, cols, s] -> (m, n, K, 3, 3) complex128."""
        rows, cols = np.asarray(rows), np.asarray(cols)
        s = np.atleast_1d(np.asarray(s, dtype=np.complex128))
        K = len(s)
        out = np.zeros((len(rows), len(cols), K, 3, 3), dtype=np.complex128)
        geo = self.geo
        if self.kernel in SL_KINDS:
            for a, i in enumerate(rows):
                i = int(i)
                sing = [b for b, e in enumerate(cols) if _on_element(geo, self.rows_kind, i, int(e))]
                for b in sing:
                    out[a, b] = self.v_elem(i, int(cols[b]), s)
                regb = np.setdiff1d(np.arange(len(cols)), sing)
                pos = {int(cols[b]): b for b in regb}
                for es, y, w, _ in self._regular_groups(i, cols[regb]):
                    Uq = self._U((y - self.x[i])[None], s[:, None, None])     # (K, E, q, 3, 3)
                    val = np.einsum("eq,keqab->ekab", w, Uq)
                    out[a, [pos[int(e)] for e in es]] = val
            return out
        colpos = {int(j): b for b, j in enumerate(cols)}
        elems = np.array(sorted({e for j in cols for e in geo.node_elems[int(j)]}), dtype=np.int64)
        for a, i in enumerate(rows):
            i = int(i)
            sing = [int(e) for e in elems if _on_element(geo, self.rows_kind, i, int(e))]
            for e in sing:
                contrib = self.k_elem(i, e, s)
                for loc in range(3):
                    b = colpos.get(int(geo.tri[e, loc]))
                    if b is not None:
                        out[a, b] += contrib[:, loc]
            rest = np.setdiff1d(elems, sing)
            for es, y, w, phi in self._regular_groups(i, rest):
                Tq = self._TT((y - self.x[i])[None], geo.normal[es][None, :, None, :], s[:, None, None])
                val = np.einsum("eq,qa,keqbc->keabc", w, phi, Tq)           # (K, E, 3, 3, 3)
                for loc in range(3):
                    for ei, e in enumerate(es):
                        b = colpos.get(int(geo.tri[e, loc]))
                        if b is not None:
                            out[a, b] += val[:, ei, loc]
            if self.rows_kind == ROWS_NODES and i in colpos:
                out[a, colpos[i]] += self.rigid_body_diag(i)[None]
        return out

    def dense(self, s):
        return self.block(np.arange(self.n_rows), np.arange(self.n_cols), s)


def to_matrix(blk):
    """(m, n, 3, 3) block array -> (3m, 3n) matrix (node-major xyz)."""
    m, n = blk.shape[:2]
    return blk.transpose(0, 2, 1, 3).reshape(3 * m, 3 * n)


def from_matrix(M):
    m, n = M.shape[0] // 3, M.shape[1] // 3
    return M.reshape(m, 3, n, 3).transpose(0, 2, 1, 3)
