"""The receiver energy of a traction-driven Neumann problem through CQ and
its adjoint gradient (bem_receiver_energy_grad: half-set CQ transforms,
K-batched forward and adjoint BiCGstab on the compressed operators, the
wave-speed terms through the compressed derivative operators) against the
oracle's dense-matrix pipeline (oracle/adjoint.py, itself pinned by central
differences) on a small box; the adjoint solve on its own against dense
solves; argument refusals."""
import numpy as np
import pytest

import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2607_15292_b300 as g
from oracle import adjoint, bem  # noqa: E402

N, DT = 11, 4e-5
KERNS = (bem.KERNEL_SL, bem.KERNEL_DL, bem.KERNEL_SL_DCP, bem.KERNEL_SL_DCS, bem.KERNEL_DL_DCP, bem.KERNEL_DL_DCS)


@pytest.fixture(scope="module")
def case():
    xyz, tri = syn.box(2.0, 1.0, 1.0, 0.5)
    s = bem.freqs_bdf2(N, DT, adjoint.half_count(N))
    ops = adjoint.operators(xyz, tri, syn.STEEL, s, KERNS)
    gt = syn.box_traction(xyz, tri, N, DT, width=0.5, t0=1.5e-4, tw=6e-5)
    rec = syn.box_receivers(xyz, 6)
    J, dg, dc = adjoint.receiver_energy_grad(ops["sl"], ops["dl"], [ops["sl_dcp"], ops["sl_dcs"]],
                                             [ops["dl_dcp"], ops["dl_dcs"]], gt, rec, N, DT)
    return dict(xyz=xyz, tri=tri, s=s, ops=ops, g=gt, rec=rec, J=J, dg=dg, dc=dc)


def _lib_ops(c, precision, eps):
    ctx = g.Context(eps=eps, precision=precision, leaf=12, eta=2.0)
    ctx.material(*syn.STEEL)
    ctx.freqs(c["s"])
    mesh = ctx.mesh(c["xyz"], c["tri"])
    kinds = (g.BEM_SL, g.BEM_DL, g.BEM_SL_DCP, g.BEM_SL_DCS, g.BEM_DL_DCP, g.BEM_DL_DCS)
    return ctx, [mesh.tree(g.BEM_ROWS_NODES, k).compress() for k in kinds]


# MIXED keeps the frequency-domain vectors (g^, u^, G^, W) in complex64: their
# rounding, 2^-24 and uncorrelated across frequencies, comes back from the
# inverse transform multiplied by lam^-n, up to lam^-N = 1e5 at the last
# level (lam = (1e-10)^(1/(2N))): about 6e-3 of the largest value at worst
# for single samples (the traction gradient), less for sums over the time
# levels (J, the wave-speed gradients).  FP64: 1e5 x 1e-16 plus the
# compression and solve tolerances.
@pytest.mark.parametrize("precision,eps,tol_j,tol_g,tol_c", [(0, 1e-10, 1e-7, 1e-7, 1e-6),
                                                              (1, 1e-6, 1e-4, 6e-3, 1e-3)])
def test_receiver_energy_gradient_vs_oracle(case, record, precision, eps, tol_j, tol_g, tol_c):
    c = case
    ctx, (V, A, dVp, dVs, dAp, dAs) = _lib_ops(c, precision, eps)
    gt = torch.tensor(c["g"], dtype=torch.float64, device="cuda")
    J, dg, dc, it = g.receiver_energy_grad(V, A, gt, c["rec"], N, DT, dV=(dVp, dVs), dA=(dAp, dAs),
                                           tol=1e-11 if precision == 0 else 1e-7, max_iter=300)
    ej = abs(J - c["J"]) / c["J"]
    eg = np.abs(dg.cpu().numpy() - c["dg"]).max() / np.abs(c["dg"]).max()
    ec = max(abs(a - b) / abs(b) for a, b in zip(dc, c["dc"]))
    record("J_rel_err", ej)
    record("dJdg_rel_err", eg)
    record("dJdc_rel_err", ec)
    assert ej < tol_j and eg < tol_g and ec < tol_c, (ej, eg, ec)
    assert it.min() >= 1
    # J alone (no gradient requested) is the same number
    J2, dg2, dc2, _ = g.receiver_energy_grad(V, A, gt, c["rec"], N, DT, grad_g=False,
                                             tol=1e-11 if precision == 0 else 1e-7, max_iter=300)
    assert dg2 is None and dc2 == [] and abs(J2 - J) <= 1e-12 * J


@pytest.mark.parametrize("precision", [0, 1])
def test_adjoint_solve_vs_dense(case, precision):
    c = case
    ctx, ops = _lib_ops(c, precision, 1e-10 if precision == 0 else 1e-6)
    A = ops[1]
    K = len(c["s"])
    cdt = torch.complex128 if precision == 0 else torch.complex64
    B = torch.tensor(syn.complex_normal(21, (K, A.tree.n_rows, 3)), dtype=cdt, device="cuda")
    X = torch.empty_like(B)
    it, rr = A.solve(B, X, tol=1e-10 if precision == 0 else 1e-6, max_iter=300, adjoint=True)
    Bn = B.cpu().numpy().astype(np.complex128)
    Xn = X.cpu().numpy().astype(np.complex128)
    for k in range(K):
        Ak = c["ops"]["dl"][k]
        ref = np.linalg.solve(Ak.conj().T, Bn[k].reshape(-1))
        err = np.linalg.norm(Xn[k].reshape(-1) - ref) / np.linalg.norm(ref)
        assert err < (1e-8 if precision == 0 else 2e-4), (k, err)


def test_receiver_energy_refusals(case):
    c = case
    ctx, (V, A, dVp, dVs, dAp, dAs) = _lib_ops(c, 0, 1e-8)
    gt = torch.tensor(c["g"], dtype=torch.float64, device="cuda")
    with pytest.raises(g.BemError):        # receivers repeated
        g.receiver_energy_grad(V, A, gt, [1, 1], N, DT)
    with pytest.raises(g.BemError):        # receiver out of range
        g.receiver_energy_grad(V, A, gt, [10 ** 6], N, DT)
    with pytest.raises(g.BemError):        # V and A swapped
        g.receiver_energy_grad(A, V, torch.zeros((N + 1, A.tree.n_cols, 3), dtype=torch.float64, device="cuda"),
                               c["rec"], N, DT)
    with pytest.raises(g.BemError):        # frequencies of another dt
        g.receiver_energy_grad(V, A, gt, c["rec"], N, 2 * DT)
    with pytest.raises(g.BemError):        # derivative operators of the wrong kinds
        g.receiver_energy_grad(V, A, gt, c["rec"], N, DT, dV=(dVs,), dA=(dAs,))
    with pytest.raises(ValueError):        # traction of the wrong shape
        g.receiver_energy_grad(V, A, gt[:-1], c["rec"], N, DT)


def test_receiver_energy_autograd_and_traction_differences(case):
    """torch.autograd through ReceiverEnergy gives the library's gradients;
    central differences of the library's J match them (FP64): in single
    traction samples (J is quadratic in g: exact for any step; 1e-3 of the
    largest sample keeps the solves' tolerance out of the quotient) and in
    each wave speed (relative step 1e-6, operators recompressed at the
    perturbed speeds)."""
    from paper_2607_15292_b300 import autograd as ga
    c = case
    ctx, (V, A, dVp, dVs, dAp, dAs) = _lib_ops(c, 0, 1e-10)
    gt = torch.tensor(c["g"], dtype=torch.float64, device="cuda", requires_grad=True)
    cs = torch.zeros(2, dtype=torch.float64, requires_grad=True)
    J = ga.receiver_energy(gt, cs, V, A, (dVp, dVs), (dAp, dAs), c["rec"], N, DT, tol=1e-12, max_iter=300)
    J.backward()
    J0, dg, dc, _ = g.receiver_energy_grad(V, A, gt.detach(), c["rec"], N, DT, dV=(dVp, dVs), dA=(dAp, dAs),
                                           tol=1e-12, max_iter=300)
    assert torch.equal(gt.grad, dg) and np.allclose(cs.grad.numpy(), dc, rtol=0, atol=0)
    h = 1e-3 * float(np.abs(c["g"]).max())
    top = int(np.argmax(np.abs(c["g"][:, :, 2]).max(axis=0)))
    for n, e, a in ((3, top, 2), (6, top, 0), (N, 0, 1)):
        Js = []
        for sg in (1.0, -1.0):
            gp = gt.detach().clone()
            gp[n, e, a] += sg * h
            Js.append(g.receiver_energy_grad(V, A, gp, c["rec"], N, DT, grad_g=False, tol=1e-12, max_iter=300)[0])
        fd = (Js[0] - Js[1]) / (2 * h)
        assert abs(fd - dg[n, e, a].item()) <= 1e-6 * dg.abs().max().item(), (n, e, a, fd, dg[n, e, a].item())
    rho, lam, mu = syn.STEEL
    cp, cs0 = np.sqrt((lam + 2 * mu) / rho), np.sqrt(mu / rho)
    for a in range(2):
        Js = []
        for sg in (1.0, -1.0):
            p, q = (cp * (1 + sg * 1e-6), cs0) if a == 0 else (cp, cs0 * (1 + sg * 1e-6))
            ctx2 = g.Context(eps=1e-10, precision=0, leaf=12, eta=2.0)
            ctx2.material(rho, rho * p * p - 2 * rho * q * q, rho * q * q)
            ctx2.freqs(c["s"])
            m2 = ctx2.mesh(c["xyz"], c["tri"])
            V2, A2 = (m2.tree(g.BEM_ROWS_NODES, k).compress() for k in (g.BEM_SL, g.BEM_DL))
            Js.append(g.receiver_energy_grad(V2, A2, gt.detach(), c["rec"], N, DT, grad_g=False, tol=1e-12,
                                             max_iter=300)[0])
        fd = (Js[0] - Js[1]) / (2e-6 * (cp if a == 0 else cs0))
        assert abs(fd - dc[a]) <= 1e-3 * abs(dc[a]), (a, fd, dc[a])
