"""Pins of the oracle's matrices: frequency set, meshes of Table 1, rigid-body
identity, singular V against a closed form, conjugate symmetry, and the
closed-form response of a sphere under uniform pressure."""
import math
import os

import numpy as np
import pytest

import synthetic as syn
from oracle import bem, kernels, quadrature as quad, sphere

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_paper_cube_meshes_table1():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "paper_table1_mesh.txt"))
            if l.strip() and not l.startswith("#")]
    for lvl, nodes, elems in rows[:3]:
        xyz, tri = syn.paper_cube(int(lvl))
        assert (len(xyz), len(tri)) == (int(nodes), int(elems))
        geo = bem.Geometry(xyz, tri)
        assert abs(geo.area.sum() - 6.0) < 1e-12


def test_mesh_sizes_of_workloads():
    xyz, tri = syn.cube_grid(4)
    assert (len(xyz), len(tri)) == (98, 192)
    xyz, tri = syn.icosphere(4)
    assert (len(xyz), len(tri)) == (2562, 5120)
    geo = bem.Geometry(xyz, tri)
    # outward normals: sum n.(centroid) area = 3 volume > 0
    vol = (geo.normal * geo.centroid).sum(1) @ geo.area / 3
    assert abs(vol - 4 * math.pi / 3) < 0.02


def test_bdf2_frequencies():
    N, dt = 64, 2e-5
    s = bem.freqs_bdf2(N, dt)
    L = N + 1
    for k in range(1, L):
        assert abs(s[L - k] - np.conj(s[k])) < 1e-9 * abs(s[k])
    assert abs(s[0].imag) == 0.0
    # BDF2 generating polynomial delta(zeta) = 3/2 - 2 zeta + zeta^2 / 2
    lam = 1e-10 ** (1 / (2 * N))
    z = lam * np.exp(-2j * np.pi * np.arange(L) / L)
    np.testing.assert_allclose(s * dt, 1.5 - 2 * z + 0.5 * z * z, rtol=1e-14)
    assert 8.8e3 < abs(s).min() < 9.0e3 and 1.75e5 < abs(s).max() < 1.77e5


def test_rigid_body_centroid_rows():
    """sum_j (C + K)(s -> 0)[i, j] = 0 (rigid translation), quadrature-limited."""
    xyz, tri = syn.cube_grid(2)
    op = bem.Operator(xyz, tri, syn.STEEL, rows=bem.ROWS_CENTROIDS, kernel=bem.KERNEL_DL)
    D = op.dense(np.array([1e-2]))
    assert np.abs(D[:, :, 0].sum(1)).max() < 1e-6     # quadrature rule of the module
    old = quad.N_NEAR, quad.N_CLOSE
    try:
        quad.N_NEAR, quad.N_CLOSE = 24, 24
        D = op.dense(np.array([1e-2]))
    finally:
        quad.N_NEAR, quad.N_CLOSE = old
    assert np.abs(D[:, :, 0].sum(1)).max() < 1e-8


def test_rigid_body_node_rows_dynamic_part_small():
    xyz, tri = syn.icosphere(1)
    op = bem.Operator(xyz, tri, syn.STEEL, rows=bem.ROWS_NODES, kernel=bem.KERNEL_DL)
    D = op.dense(np.array([1e-2]))
    assert np.abs(D[:, :, 0].sum(1)).max() < 1e-10


def test_singular_single_layer_trace_closed_form():
    """Static V on the own element: tr U0 = (3(3-4nu)+1) / (16 pi mu (1-nu) r),
    int_e 1/r dA in closed form (sum over sub-triangles about the centroid)."""
    rho, lam, mu = syn.STEEL
    nu = lam / (2 * (lam + mu))
    xyz = np.array([[0., 0, 0], [1., 0, 0], [0.4, 0.8, 0.1]])
    tri = np.array([[0, 1, 2]])
    op = bem.Operator(xyz, tri, syn.STEEL, rows=bem.ROWS_CENTROIDS, kernel=bem.KERNEL_SL)
    V = op.v_elem(0, 0, np.array([1e-9]))[0]
    x = xyz.mean(0)
    inv_r = 0.0
    for a in range(3):
        B, C = xyz[a], xyz[(a + 1) % 3]
        t = (C - B) / np.linalg.norm(C - B)
        F = B + ((x - B) @ t) * t
        h = np.linalg.norm(F - x)
        inv_r += h * (math.asinh(((C - F) @ t) / h) - math.asinh(((B - F) @ t) / h))
    tr = (3 * (3 - 4 * nu) + 1) / (16 * math.pi * mu * (1 - nu)) * inv_r
    assert abs(np.trace(V).real - tr) < 1e-8 * tr


def test_operator_conjugate_symmetry():
    xyz, tri = syn.cube_grid(1)
    s = np.array([3e3 + 4e3j])
    for rows, kern in [(bem.ROWS_CENTROIDS, bem.KERNEL_SL), (bem.ROWS_NODES, bem.KERNEL_DL)]:
        op = bem.Operator(xyz, tri, syn.STEEL, rows=rows, kernel=kern)
        a = op.dense(s)
        b = op.dense(np.conj(s))
        np.testing.assert_allclose(b, np.conj(a), rtol=0, atol=1e-13 * np.abs(a).max())


@pytest.mark.slow
def test_sphere_uniform_pressure_closed_form():
    """Neumann rows at nodes: (C + K) u = V t, t = -p n; the radial
    displacement converges to the closed form on refining the icosphere."""
    rho, lam, mu = syn.STEEL
    s0 = bem.freqs_bdf2(64, 2e-5, 1)[0]
    errs = []
    for lvl in (1, 2):
        xyz, tri = syn.icosphere(lvl)
        ov = bem.Operator(xyz, tri, syn.STEEL, rows=bem.ROWS_NODES, kernel=bem.KERNEL_SL)
        ok = bem.Operator(xyz, tri, syn.STEEL, rows=bem.ROWS_NODES, kernel=bem.KERNEL_DL)
        u = sphere.bem_neumann_sphere(ov, ok, s0)
        ur = (u * xyz).sum(1)
        ex = sphere.radial_displacement(1.0, s0, 1.0, rho, lam, mu)
        errs.append(np.abs(ur - ex).max() / abs(ex))
    assert errs[0] < 0.025 and errs[1] < 0.008 and errs[1] < errs[0] / 2.5


def test_sphere_closed_form_static_limit():
    rho, lam, mu = syn.STEEL
    c1 = math.sqrt((lam + 2 * mu) / rho)
    u = sphere.radial_displacement(1.0, 1e-3 * c1, 1.0, rho, lam, mu)   # k a = 1e-3
    assert abs(u - (-1.0 / (3 * lam + 2 * mu))) < 1e-5 * abs(u)


@pytest.mark.parametrize("rows", [bem.ROWS_CENTROIDS, bem.ROWS_NODES])
@pytest.mark.parametrize("kern,wave", [(bem.KERNEL_SL_DCP, "p"), (bem.KERNEL_SL_DCS, "s")])
def test_speed_derivative_operator_by_fd(rows, kern, wave):
    """dV/dc_a (singular, near and far element integrals) against central
    differences of the single layer V in c_a at fixed density."""
    xyz, tri = syn.icosphere(1)
    s = bem.freqs_bdf2(16, 2e-5, 16)[[0, 9]]
    rho = syn.STEEL[0]
    c1, c2 = kernels.wave_speeds(*syn.STEEL)
    c = c1 if wave == "p" else c2
    h = 1e-4 * c
    rws = np.array([0, 5, 17])

    def v(dc):
        cc1, cc2 = (c1 + dc, c2) if wave == "p" else (c1, c2 + dc)
        mat = (rho,) + kernels.lame_from_speeds(rho, cc1, cc2)
        op = bem.Operator(xyz, tri, mat, rows=rows, kernel=bem.KERNEL_SL)
        return op.block(rws, np.arange(op.n_cols), s)
    fd = (-v(2 * h) + 8 * v(h) - 8 * v(-h) + v(-2 * h)) / (12 * h)
    op = bem.Operator(xyz, tri, syn.STEEL, rows=rows, kernel=kern)
    d = op.block(rws, np.arange(op.n_cols), s)
    assert op.n_cols == len(tri)
    np.testing.assert_allclose(d, fd, rtol=0, atol=1e-7 * np.abs(fd).max())


@pytest.mark.parametrize("rows", [bem.ROWS_CENTROIDS, bem.ROWS_NODES])
@pytest.mark.parametrize("kern,wave", [(bem.KERNEL_DL_DCP, "p"), (bem.KERNEL_DL_DCS, "s")])
def test_dl_speed_derivative_operator_by_fd(rows, kern, wave):
    """d(C + K)/dc_a (rigid-body diagonal or CPV + free term, Duffy
    remainders, near and far elements) against central differences of the
    double layer in c_a at fixed density."""
    xyz, tri = syn.icosphere(1)
    s = bem.freqs_bdf2(16, 2e-5, 16)[[0, 9]]
    rho = syn.STEEL[0]
    c1, c2 = kernels.wave_speeds(*syn.STEEL)
    c = c1 if wave == "p" else c2
    h = 1e-4 * c
    rws = np.array([0, 5, 17])

    def k(dc):
        cc1, cc2 = (c1 + dc, c2) if wave == "p" else (c1, c2 + dc)
        mat = (rho,) + kernels.lame_from_speeds(rho, cc1, cc2)
        op = bem.Operator(xyz, tri, mat, rows=rows, kernel=bem.KERNEL_DL)
        return op.block(rws, np.arange(op.n_cols), s)
    fd = (-k(2 * h) + 8 * k(h) - 8 * k(-h) + k(-2 * h)) / (12 * h)
    op = bem.Operator(xyz, tri, syn.STEEL, rows=rows, kernel=kern)
    d = op.block(rws, np.arange(op.n_cols), s)
    assert op.n_cols == len(xyz)
    np.testing.assert_allclose(d, fd, rtol=0, atol=1e-7 * np.abs(fd).max())
