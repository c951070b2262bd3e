"""Wave-speed derivatives at fixed density of the single layer (dV/dc_p,
dV/dc_s: kernels BEM_SL_DCP, BEM_SL_DCS) and of the double layer
(d(C + K)/dc_p, d(C + K)/dc_s: BEM_DL_DCP, BEM_DL_DCS), through the C ABI.

Entries (singular, near and far rules) element by element against the
oracle (FP64 within 1e-10 per 3x3 block, MIXED within the entry tolerance);
the 3D-ACA compression of the derivative operators and their apply against
the oracle's dense tensors; the wave-speed gradient of a receiver functional
J = sum_k sum_i w_i |(C(c) x)_k[i]|^2 (C = V or C + K) by the adjoint
method (autograd through bem_op_inner) against central differences of J
built from the library's exact entries at perturbed wave speeds."""
import numpy as np
import pytest

import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2607_15292_b300 as g
    from paper_2607_15292_b300 import autograd as ga
from oracle import bem, kernels  # noqa: E402

ROWS = {"nodes": 1, "centroids": 0}
DK = {("sl", "p"): (2, bem.KERNEL_SL_DCP), ("sl", "s"): (3, bem.KERNEL_SL_DCS),
      ("dl", "p"): (4, bem.KERNEL_DL_DCP), ("dl", "s"): (5, bem.KERNEL_DL_DCS)}


def _ctx(s, precision=0, eps=1e-6, leaf=16, material=syn.STEEL):
    ctx = g.Context(eps=eps, precision=precision, leaf=leaf)
    ctx.material(*material)
    ctx.freqs(s)
    return ctx


def _entries(mesh, rows, kern, req, precision):
    req_t = torch.tensor(np.asarray(req, dtype=np.int32), device="cuda")
    dt = torch.complex128 if precision == 0 else torch.complex64
    out = torch.empty((len(req), 3, 3), dtype=dt, device="cuda")
    mesh.entries(rows, kern, req_t, out)
    return out.cpu().numpy().astype(np.complex128)


def _block_err(a, b, floor):
    num = np.linalg.norm((a - b).reshape(len(a), -1), axis=1)
    den = np.linalg.norm(b.reshape(len(b), -1), axis=1) + floor
    return (num / den).max()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("rows", ["nodes", "centroids"])
@pytest.mark.parametrize("layer", ["sl", "dl"])
@pytest.mark.parametrize("wave", ["p", "s"])
def test_speed_derivative_entries_vs_oracle(precision, rows, layer, wave):
    xyz, tri = syn.icosphere(1)
    s = bem.freqs_bdf2(16, 1e-4, 16)
    ks = [0, 7, 15]
    kid, okern = DK[(layer, wave)]
    mesh = _ctx(s, precision).mesh(xyz, tri)
    D = bem.Operator(xyz, tri, syn.STEEL, rows=rows, kernel=okern).dense(s[ks])
    m, n = D.shape[:2]
    assert n == (len(tri) if layer == "sl" else len(xyz))
    req = [(i, j, k) for i in range(m) for j in range(n) for k in ks]
    got = _entries(mesh, ROWS[rows], kid, req, precision)
    want = np.stack([D[i, j, ks.index(k)] for i, j, k in req])
    if precision == 0:
        assert _block_err(got, want, 1e-12 * np.abs(want).max()) < 1e-10
    else:
        assert np.linalg.norm(got - want) <= 1e-6 * np.linalg.norm(want)
        assert _block_err(got, want, 1e-6 * np.abs(want).max()) < 2e-5


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("layer", ["sl", "dl"])
@pytest.mark.parametrize("wave", ["p", "s"])
def test_speed_derivative_operator_compressed(precision, layer, wave):
    """3D-ACA of the derivative operator on the level-2 icosphere (node
    rows, far blocks present): dense reconstruction and batched apply within
    10 eps."""
    eps = 1e-6
    xyz, tri = syn.icosphere(2)
    s = bem.freqs_bdf2(16, 1e-4, 16)
    kid, okern = DK[(layer, wave)]
    D = bem.Operator(xyz, tri, syn.STEEL, rows="nodes", kernel=okern).dense(s)
    ctx = _ctx(s, precision, eps=eps)
    t = ctx.mesh(xyz, tri).tree(g.BEM_ROWS_NODES, kid)
    op = t.compress()
    nc = len(tri) if layer == "sl" else len(xyz)
    assert t.n_cols == nc and t.n_far > 0
    cdt = torch.complex128 if precision == 0 else torch.complex64
    out = torch.empty(D.shape, dtype=cdt, device="cuda")
    op.dense(out)
    C = out.cpu().numpy().astype(np.complex128)
    e0 = np.linalg.norm(C - D) / np.linalg.norm(D)
    assert e0 < eps, e0
    K = len(s)
    X = syn.complex_normal(3, (K, nc, 3))
    Xt = torch.tensor(X, dtype=cdt, device="cuda")
    Yt = torch.empty((K, len(xyz), 3), dtype=cdt, device="cuda")
    op.apply(Xt, Yt)
    Yd = np.einsum("ijkab,kjb->kia", D, X)
    e1 = np.linalg.norm(Yt.cpu().numpy() - Yd) / np.linalg.norm(Yd)
    assert e1 < eps, e1
    # <G, dV X> through bem_op_inner against the oracle's dense product
    G = syn.complex_normal(4, (K, len(xyz), 3))
    Gt = torch.tensor(G, dtype=cdt, device="cuda")
    ip = op.inner(Gt, Xt)
    want = np.vdot(G, Yd)
    e2 = abs(ip - want) / (np.linalg.norm(G) * np.linalg.norm(Yd))
    assert e2 < eps, e2


def _receiver_functional(V, t, w):
    """J = sum_k sum_i w_i |(V_k t_k)[i]|^2 from a dense (m, n, K, 3, 3) V."""
    Y = np.einsum("ijkab,kjb->kia", V, t)
    return float((w[None, :, None] * np.abs(Y) ** 2).sum())


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("layer", ["sl", "dl"])
def test_wave_speed_gradient_adjoint_vs_fd(precision, layer):
    xyz, tri = syn.icosphere(1)
    s = bem.freqs_bdf2(16, 1e-4, 8)
    K = len(s)
    rho = syn.STEEL[0]
    c1, c2 = kernels.wave_speeds(*syn.STEEL)
    rng = np.random.default_rng(21)
    base = g.BEM_SL if layer == "sl" else g.BEM_DL
    nc = len(tri) if layer == "sl" else len(xyz)
    t = syn.complex_normal(5, (K, nc, 3))
    w = (rng.random(len(xyz)) < 0.3).astype(np.float64)      # receivers
    # adjoint gradient through the compressed operators
    ctx = _ctx(s, precision, eps=1e-8 if precision == 0 else 1e-6, leaf=8)
    mesh = ctx.mesh(xyz, tri)
    op = mesh.tree(g.BEM_ROWS_NODES, base).compress()
    dops = [mesh.tree(g.BEM_ROWS_NODES, DK[(layer, wv)][0]).compress() for wv in ("p", "s")]
    cdt = torch.complex128 if precision == 0 else torch.complex64
    T = torch.tensor(t, dtype=cdt, device="cuda", requires_grad=True)
    c = torch.tensor([c1, c2], dtype=torch.float64, device="cuda", requires_grad=True)
    W = torch.tensor(w, dtype=torch.float64, device="cuda")
    Y = ga.apply_speeds(op, dops, T, c)
    J = (W[None, :, None] * Y.abs().to(torch.float64) ** 2).sum()
    J.backward()
    grad = c.grad.cpu().numpy()
    # the traction gradient equals the plain adjoint apply's
    gX = torch.empty_like(T)
    Yc = Y.detach()
    op.apply_adjoint((2 * W[None, :, None] * Yc).to(cdt), gX)
    assert torch.linalg.norm(T.grad - gX) <= 1e-5 * torch.linalg.norm(gX)
    # central differences of J from exact FP64 entries at perturbed speeds
    req = [(i, j, k) for i in range(len(xyz)) for j in range(nc) for k in range(K)]

    def J_at(cc1, cc2):
        mat = (rho,) + kernels.lame_from_speeds(rho, cc1, cc2)
        mh = _ctx(s, 0, material=mat).mesh(xyz, tri)
        E = _entries(mh, 1, base, req, 0).reshape(len(xyz), nc, K, 3, 3)
        return _receiver_functional(E, t, w)
    for a, (cc, name) in enumerate(((c1, "p"), (c2, "s"))):
        h = 1e-4 * cc
        if name == "p":
            fd = (-J_at(c1 + 2 * h, c2) + 8 * J_at(c1 + h, c2) - 8 * J_at(c1 - h, c2) + J_at(c1 - 2 * h, c2)) / (12 * h)
        else:
            fd = (-J_at(c1, c2 + 2 * h) + 8 * J_at(c1, c2 + h) - 8 * J_at(c1, c2 - h) + J_at(c1, c2 - 2 * h)) / (12 * h)
        tol = 1e-6 if precision == 0 else 2e-5
        assert abs(grad[a] - fd) <= tol * abs(fd), (name, grad[a], fd)
