"""Adjoint (conjugate-transpose) apply of the compressed operator through the
C ABI, against the FP64 oracle's conjugate-transpose apply of the dense
tensor, plus the inner-product identity <C x, y> = <x, C^H y> on the
compressed operator itself (dense faces, low-rank faces, dense fallback
blocks; batched and contracted)."""
import numpy as np
import pytest

import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2607_15292_b300 as g
from oracle import aca, bem  # noqa: E402

EPS = 1e-6
ROWS = {"nodes": 1, "centroids": 0}
KERN = {"sl": 0, "dl": 1}


def _two_spheres(level, offset, seed):
    xyz, tri = syn.icosphere(level)
    rng = np.random.default_rng(seed)
    a = xyz * (1 + 0.05 * rng.normal(size=(len(xyz), 1)))
    b = xyz * (1 + 0.05 * rng.normal(size=(len(xyz), 1))) + np.array([offset, 0.3, -0.2])
    return np.concatenate([a, b]), np.concatenate([tri, tri + len(xyz)]).astype(np.int32)


CASES = {
    # name: (mesh, rows, kernel, leaf, column sample or None for all)
    "cube2-centroids-sl": (lambda: syn.cube_grid(2), "centroids", "sl", 8, None),
    "ico2-nodes-dl": (lambda: syn.icosphere(2), "nodes", "dl", 16, None),
    "spheres-nodes-sl": (lambda: _two_spheres(2, 8.0, 7), "nodes", "sl", 64, 48),   # low-rank faces
}
_ORACLE = {}


def _oracle_cols(name, s):
    """Oracle tensor restricted to sampled columns: (M, |J|, K, 3, 3), J."""
    if name not in _ORACLE:
        mesh, rows, kern, leaf, ns = CASES[name]
        xyz, tri = mesh()
        op = bem.Operator(xyz, tri, syn.STEEL, rows=rows, kernel=kern)
        J = np.arange(op.n_cols) if ns is None else np.sort(
            np.random.default_rng(2).choice(op.n_cols, ns, replace=False))
        _ORACLE[name] = (op.block(np.arange(op.n_rows), J, s), J)
    return _ORACLE[name]


def _compress(name, precision, s):
    mesh, rows, kern, leaf, _ = CASES[name]
    xyz, tri = mesh()
    ctx = g.Context(eps=EPS, precision=precision, leaf=leaf)
    ctx.material(*syn.STEEL)
    ctx.freqs(s)
    t = ctx.mesh(xyz, tri).tree(ROWS[rows], KERN[kern])
    return t, t.compress()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_apply_matches_oracle(name, precision):
    s = bem.freqs_bdf2(16, 1e-4, 16)
    K = len(s)
    D, J = _oracle_cols(name, s)
    t, op = _compress(name, precision, s)
    if name.startswith("spheres"):
        assert op.stats().n_faces_lowrank > 0
    cdt = torch.complex128 if precision == 0 else torch.complex64
    Y = syn.complex_normal(8, (K, t.n_rows, 3))
    Yt = torch.tensor(Y, dtype=cdt, device="cuda")
    Xt = torch.empty((K, t.n_cols, 3), dtype=cdt, device="cuda")
    op.apply_adjoint(Yt, Xt, g.BEM_APPLY_BATCHED)
    Xo = aca.apply_adjoint_dense(D, Y.transpose(1, 2, 0))          # (|J|, 3, K)
    X = Xt.cpu().numpy().astype(np.complex128)[:, J].transpose(1, 2, 0)
    assert _rel(X, Xo) < EPS, _rel(X, Xo)
    # contracted adjoint: out_k = C_k^H y for every k
    y = syn.complex_normal(9, (t.n_rows, 3))
    yt = torch.tensor(y, dtype=cdt, device="cuda")
    op.apply_adjoint(yt, Xt, g.BEM_APPLY_CONTRACTED)
    Xc = Xt.cpu().numpy().astype(np.complex128)[:, J].transpose(1, 2, 0)
    Xco = aca.apply_adjoint_dense(D, np.repeat(y[:, :, None], K, axis=2))
    assert _rel(Xc, Xco) < EPS, _rel(Xc, Xco)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_inner_product_identity(name, precision):
    """<y, C x> = <C^H y, x> on the compressed operator: the adjoint is the
    exact conjugate transpose of what the forward apply applies."""
    s = bem.freqs_bdf2(16, 1e-4, 16)
    K = len(s)
    t, op = _compress(name, precision, s)
    cdt = torch.complex128 if precision == 0 else torch.complex64
    X = torch.tensor(syn.complex_normal(4, (K, t.n_cols, 3)), dtype=cdt, device="cuda")
    Y = torch.tensor(syn.complex_normal(5, (K, t.n_rows, 3)), dtype=cdt, device="cuda")
    CX = torch.empty((K, t.n_rows, 3), dtype=cdt, device="cuda")
    CHY = torch.empty((K, t.n_cols, 3), dtype=cdt, device="cuda")
    op.apply(X, CX)
    op.apply_adjoint(Y, CHY)
    tol = 1e-12 if precision == 0 else 2e-6
    for k in range(K):
        lhs = torch.vdot(Y[k].flatten().to(torch.complex128), CX[k].flatten().to(torch.complex128)).item()
        rhs = torch.vdot(CHY[k].flatten().to(torch.complex128), X[k].flatten().to(torch.complex128)).item()
        scale = (torch.linalg.norm(Y[k].to(torch.complex128)) * torch.linalg.norm(CX[k].to(torch.complex128))).item()
        assert abs(lhs - rhs) <= tol * scale, (k, lhs, rhs)
    # contracted: <y, sum_k C_k x_k> = sum_k <C_k^H y, x_k>
    y = torch.tensor(syn.complex_normal(6, (t.n_rows, 3)), dtype=cdt, device="cuda")
    cx = torch.empty((t.n_rows, 3), dtype=cdt, device="cuda")
    op.apply(X, cx, g.BEM_APPLY_CONTRACTED)
    op.apply_adjoint(y, CHY, g.BEM_APPLY_CONTRACTED)
    lhs = torch.vdot(y.flatten().to(torch.complex128), cx.flatten().to(torch.complex128)).item()
    rhs = torch.vdot(CHY.flatten().to(torch.complex128), X.flatten().to(torch.complex128)).item()
    scale = (torch.linalg.norm(y.to(torch.complex128)) * torch.linalg.norm(cx.to(torch.complex128))).item()
    assert abs(lhs - rhs) <= tol * scale * np.sqrt(K)


def test_autograd_function_gradcheck_fp64():
    """torch.autograd.gradcheck of the differentiable apply (FP64, small
    operator): the backward is the exact vector-Jacobian product."""
    from paper_2607_15292_b300 import autograd as ga
    xyz, tri = syn.cube_grid(1)
    s = bem.freqs_bdf2(8, 1e-4, 2)
    ctx = g.Context(eps=EPS, precision=0, leaf=4)
    ctx.material(*syn.STEEL)
    ctx.freqs(s)
    op = ctx.mesh(xyz, tri).tree(g.BEM_ROWS_NODES, g.BEM_SL).compress()
    X = torch.tensor(syn.complex_normal(1, (len(s), len(tri), 3)), dtype=torch.complex128, device="cuda",
                     requires_grad=True)
    for mode in (g.BEM_APPLY_BATCHED, g.BEM_APPLY_CONTRACTED):
        assert torch.autograd.gradcheck(lambda x: ga.apply(op, x, mode), (X,), eps=1e-6, atol=1e-9, rtol=1e-6)


@pytest.mark.parametrize("precision", [0, 1])
def test_receiver_energy_gradient_matches_oracle(precision):
    """Gradient of a receiver energy L = sum_k sum_{i in R} |(C_k x_k)_i|^2
    with respect to the traction loads x (single layer, node rows): autograd
    through the compressed operator against C^H of the oracle's dense tensor
    applied to the receiver residual (same convention, dL/dx*)."""
    from paper_2607_15292_b300 import autograd as ga
    s = bem.freqs_bdf2(16, 1e-4, 16)
    K = len(s)
    xyz, tri = syn.icosphere(2)
    opo = bem.Operator(xyz, tri, syn.STEEL, rows="nodes", kernel="sl")
    D = opo.dense(s)                                         # (M, N, K, 3, 3)
    ctx = g.Context(eps=EPS, precision=precision, leaf=16)
    ctx.material(*syn.STEEL)
    ctx.freqs(s)
    op = ctx.mesh(xyz, tri).tree(g.BEM_ROWS_NODES, g.BEM_SL).compress()
    rec = np.sort(np.random.default_rng(4).choice(len(xyz), 16, replace=False))
    cdt = torch.complex128 if precision == 0 else torch.complex64
    x0 = syn.complex_normal(2, (K, len(tri), 3))
    X = torch.tensor(x0, dtype=cdt, device="cuda", requires_grad=True)
    Y = ga.apply(op, X)
    L = (Y[:, torch.tensor(rec, device="cuda")].abs() ** 2).sum()
    L.backward()
    # the same loss on the oracle's output, differentiated by autograd with respect to Y only
    Yo = torch.tensor(np.einsum("ijkab,kjb->kia", D, x0), dtype=torch.complex128, requires_grad=True)
    (Yo[:, torch.tensor(rec)].abs() ** 2).sum().backward()
    gY = Yo.grad.numpy()                                     # (K, M, 3)
    gX = aca.apply_adjoint_dense(D, gY.transpose(1, 2, 0)).transpose(2, 0, 1)
    got = X.grad.cpu().numpy().astype(np.complex128)
    assert _rel(got, gX) < EPS, _rel(got, gX)
