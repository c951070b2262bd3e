"""K-frequency BiCGstab solve (bem_op_solve, Sec. 5) on the compressed
operator: the Neumann problem of a sphere under uniform pressure,
(C + K)(s_k) u_k = V(s_k) t with t = -p n, node rows, for 16 frequencies of
the sphere workload's set.  Against the oracle's direct dense solve
(numpy.linalg.solve of the assembled matrices) per frequency, the closed-form
radial displacement (discretisation error of the level-2 icosphere), and the
true residual through the library's own apply."""
import numpy as np
import pytest

import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2607_15292_b300 as g
from oracle import bem, sphere  # noqa: E402

EPS = 1e-6


@pytest.mark.parametrize("precision", [0, 1])
def test_sphere_pressure_solve(precision):
    xyz, tri = syn.icosphere(2)
    s = bem.freqs_bdf2(64, 2e-5, 16)
    K = len(s)
    ctx = g.Context(eps=EPS, precision=precision, leaf=16)
    ctx.material(*syn.STEEL)
    ctx.freqs(s)
    mesh = ctx.mesh(xyz, tri)
    opV = mesh.tree(g.BEM_ROWS_NODES, g.BEM_SL).compress()
    opK = mesh.tree(g.BEM_ROWS_NODES, g.BEM_DL).compress()
    cdt = torch.complex128 if precision == 0 else torch.complex64
    ov = bem.Operator(xyz, tri, syn.STEEL, rows=bem.ROWS_NODES, kernel=bem.KERNEL_SL)
    ok = bem.Operator(xyz, tri, syn.STEEL, rows=bem.ROWS_NODES, kernel=bem.KERNEL_DL)
    t = -ov.geo.normal                                              # p = 1 on every element
    T = torch.tensor(np.broadcast_to(t, (K,) + t.shape).copy(), dtype=cdt, device="cuda")
    B = torch.empty((K, len(xyz), 3), dtype=cdt, device="cuda")
    opV.apply(T, B)
    U = torch.empty_like(B)
    tol = 1e-9 if precision == 0 else 2e-6
    it, rr = opK.solve(B, U, tol=tol, max_iter=300)
    assert (it > 0).all() and (rr <= tol).all()
    # true residual through the library's apply
    R = torch.empty_like(B)
    opK.apply(U, R)
    res = (torch.linalg.norm((R - B).to(torch.complex128)) / torch.linalg.norm(B.to(torch.complex128))).item()
    assert res < (1e-8 if precision == 0 else 2e-5), res
    u = U.cpu().numpy().astype(np.complex128)
    rho, lam, mu = syn.STEEL
    for k in (0, 7, 15):
        uo = sphere.bem_neumann_sphere(ov, ok, s[k])                 # dense direct solve, FP64
        err = np.linalg.norm(u[k] - uo) / np.linalg.norm(uo)
        # perturbation bound of a linear system: operator and right-hand side
        # within EPS of the oracle's (compressed tensor and apply, MIXED
        # entries), residual within tol -> ||du|| / ||u|| <= kappa (2 EPS + tol)
        A = bem.to_matrix(ok.dense(s[k:k + 1])[:, :, 0])
        kappa = np.linalg.cond(A)
        assert err < kappa * (2 * EPS + tol), (k, err, kappa)
        # closed form: discretisation error of the level-2 icosphere (oracle
        # direct solve: 0.65 %, 5.7 %, 4.4 % at k = 0, 7, 15)
        ur = (u[k] * xyz).sum(1)
        ex = sphere.radial_displacement(1.0, s[k], 1.0, rho, lam, mu)
        assert np.abs(ur - ex).max() / abs(ex) < (0.01 if k == 0 else 0.08), k
