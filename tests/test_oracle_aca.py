"""Pins of the oracle's 3D-ACA (Algorithm 1) and face ACA: exact recovery
of separable tensors, interpolation at the pivots, the norm recursion, the
dense fallback, and the error bound against dense BEM tensors."""
import numpy as np
import pytest

import synthetic as syn
from oracle import aca, bem, hmatrix, pipeline


def _rand(seed, shape):
    return syn.complex_normal(seed, shape)


def test_separable_tensor_recovered():
    m, n, K, r = 7, 5, 11, 3
    faces = [_rand(10 + t, (m, n, 3, 3)) for t in range(r)]
    fibres = [_rand(20 + t, (K, 3, 3)) for t in range(r)]
    C = sum(aca.face_fibre(H, f) for H, f in zip(faces, fibres))
    res = aca.aca3d(C, 1e-12)
    assert res.kind == "aca" and res.rank == r
    assert np.linalg.norm(res.tensor() - C) < 1e-10 * np.linalg.norm(C)


def test_norm_recursion_equals_explicit():
    faces = [_rand(30 + t, (4, 6, 3, 3)) for t in range(4)]
    fibres = [_rand(40 + t, (9, 3, 3)) for t in range(4)]
    C = sum(aca.face_fibre(H, f) for H, f in zip(faces, fibres))
    assert abs(aca.norm2_recursive(faces, fibres) - np.linalg.norm(C) ** 2) < 1e-10 * np.linalg.norm(C) ** 2


def _cube_tensor(kern):
    xyz, tri = syn.cube_grid(1)
    s = bem.freqs_bdf2(16, 1e-4, 16)
    op = bem.Operator(xyz, tri, syn.STEEL, rows=bem.ROWS_CENTROIDS, kernel=kern)
    return op.dense(s)


@pytest.mark.parametrize("kern", [bem.KERNEL_SL, bem.KERNEL_DL])
def test_interpolation_property(kern):
    C = _cube_tensor(kern)
    res = aca.aca3d(C, 1e-8)
    assert res.kind == "aca"
    T = res.tensor()
    scale = np.abs(C).max()
    for k in res.ks:                       # faces exact at the pivot frequencies
        assert np.abs(T[:, :, k] - C[:, :, k]).max() < 1e-12 * scale
    for (i, j) in res.pivots:              # fibres exact along the pivot positions
        assert np.abs(T[i, j] - C[i, j]).max() < 1e-12 * scale


@pytest.mark.parametrize("eps", [1e-3, 1e-6])
@pytest.mark.parametrize("kern", [bem.KERNEL_SL, bem.KERNEL_DL])
def test_error_bound_dense_bem(eps, kern):
    C = _cube_tensor(kern)
    res = aca.aca3d(C, eps)
    err = np.linalg.norm(res.tensor() - C) / np.linalg.norm(C)
    assert err < 5 * eps
    assert res.rank < C.shape[2]


def test_dense_fallback_rank_deficient_blocks():
    """Every 3 x 3 entry of rank 2 (the coplanar double-layer situation of
    Sec. 4.1): no regular pivot exists -> dense."""
    m, n, K = 4, 3, 6
    a = _rand(5, (m, n, K, 3, 2))
    b = _rand(6, (m, n, K, 2, 3))
    C = np.einsum("ijkab,ijkbc->ijkac", a, b)
    assert aca.aca3d(C, 1e-6).kind == "dense"
    assert aca.aca3d(np.zeros((2, 2, 3, 3, 3), complex), 1e-6).kind == "rank0"


def test_face_aca_recovers_low_rank_and_smooth_faces():
    m, n = 20, 15
    u = _rand(1, (m, 3, 6))
    v = _rand(2, (n, 6, 3))
    H = np.einsum("iar,jrb->ijab", u, v)          # block rank 6 (2 block pairs)
    lr = aca.aca_matrix(H, 1e-10)
    M = bem.to_matrix(H)
    assert np.linalg.norm(lr.matrix() - M) < 1e-9 * np.linalg.norm(M)
    assert lr.U.shape[1] <= 6
    # a far-field single-layer face: smooth kernel, fast decay of ranks
    xyz, tri = syn.icosphere(2)
    op = bem.Operator(xyz, tri, syn.STEEL, rows=bem.ROWS_NODES, kernel=bem.KERNEL_SL)
    rows = np.nonzero(xyz[:, 2] > 0.8)[0]
    cols = np.nonzero(op.geo.centroid[:, 2] < -0.8)[0]
    F = op.block(rows, cols, np.array([9e3]))[:, :, 0]
    for eps in (1e-4, 1e-8):
        lr = aca.aca_matrix(F, eps)
        M = bem.to_matrix(F)
        assert np.linalg.norm(lr.matrix() - M) < 20 * eps * np.linalg.norm(M)
        if eps == 1e-4:
            assert lr.U.shape[1] < 0.6 * min(M.shape)


def test_compressed_apply_matches_dense():
    xyz, tri = syn.icosphere(1)
    s = bem.freqs_bdf2(16, 1e-4, 8)
    op = bem.Operator(xyz, tri, syn.STEEL, rows=bem.ROWS_NODES, kernel=bem.KERNEL_SL)
    D = op.dense(s)
    X = syn.complex_normal(1, (op.n_cols, 3, len(s)))
    blocks = pipeline.compress(op, s, 1e-6, leaf=8, dense_tensor=D)
    Y = aca.apply_batched(blocks, X, op.n_rows)
    Yd = aca.apply_dense(D, X)
    assert np.linalg.norm(Y - Yd) < 5e-6 * np.linalg.norm(Yd)
    y = aca.apply_contracted(blocks, X, op.n_rows)
    assert np.linalg.norm(y - Yd.sum(2)) < 5e-6 * np.linalg.norm(Yd.sum(2))
    # every index pair covered exactly once by the block partition
    cover = np.zeros((op.n_rows, op.n_cols), int)
    for b in blocks:
        cover[np.ix_(b.rows, b.cols)] += 1
    assert (cover == 1).all()
    assert any(b.far for b in blocks)


def test_adjoint_apply_pins():
    """Conjugate-transpose apply: against the conjugate transpose of the
    explicit 3M x 3N matrix of each frequency (numpy) and by the inner-product
    identity <C x, y> = <x, C^H y> with the forward apply."""
    xyz, tri = syn.cube_grid(1)
    s = bem.freqs_bdf2(16, 1e-4, 4)
    op = bem.Operator(xyz, tri, syn.STEEL, rows=bem.ROWS_NODES, kernel=bem.KERNEL_DL)
    D = op.dense(s)
    M, N, K = D.shape[:3]
    X = syn.complex_normal(2, (N, 3, K))
    Y = syn.complex_normal(3, (M, 3, K))
    XA = aca.apply_adjoint_dense(D, Y)
    assert XA.shape == (N, 3, K)
    for k in range(K):
        A = bem.to_matrix(D[:, :, k])                     # (3M, 3N)
        ref = A.conj().T @ Y[:, :, k].reshape(-1)
        assert np.allclose(XA[:, :, k].reshape(-1), ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
    lhs = np.vdot(Y, aca.apply_dense(D, X))               # <y, C x>
    rhs = np.vdot(XA, X)                                  # <C^H y, x>
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("kern,dkern", [(bem.KERNEL_SL, {"p": bem.KERNEL_SL_DCP, "s": bem.KERNEL_SL_DCS}),
                                        (bem.KERNEL_DL, {"p": bem.KERNEL_DL_DCP, "s": bem.KERNEL_DL_DCS})])
def test_receiver_energy_speed_gradient_by_fd(kern, dkern):
    """The wave-speed gradient of a receiver response from the derivative
    operators against central differences of the response in c_a (rho
    fixed), single and double layer, node rows."""
    from oracle import kernels
    xyz, tri = syn.icosphere(1)
    s = bem.freqs_bdf2(16, 1e-4, 16)[[0, 5]]
    rho = syn.STEEL[0]
    c1, c2 = kernels.wave_speeds(*syn.STEEL)
    op = bem.Operator(xyz, tri, syn.STEEL, rows=bem.ROWS_NODES, kernel=kern)
    C = op.dense(s)
    X = syn.complex_normal(9, (op.n_cols, 3, len(s)))
    w = (syn.uniform01(9, op.n_rows) < 0.4).astype(np.float64)
    for wave, c in (("p", c1), ("s", c2)):
        dC = bem.Operator(xyz, tri, syn.STEEL, rows=bem.ROWS_NODES, kernel=dkern[wave]).dense(s)
        g = aca.receiver_energy_speed_gradient(C, dC, X, w)
        h = 1e-4 * c

        def J(dc):
            cc1, cc2 = (c1 + dc, c2) if wave == "p" else (c1, c2 + dc)
            mat = (rho,) + kernels.lame_from_speeds(rho, cc1, cc2)
            return aca.receiver_energy(bem.Operator(xyz, tri, mat, rows=bem.ROWS_NODES, kernel=kern).dense(s), X, w)
        fd = (-J(2 * h) + 8 * J(h) - 8 * J(-h) + J(-2 * h)) / (12 * h)
        assert abs(g - fd) <= 1e-7 * abs(fd), (wave, g, fd)
