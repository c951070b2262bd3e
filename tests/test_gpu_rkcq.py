"""Runge-Kutta CQ (2-stage Radau IIA, constant steps) of the compressed
single layer through bem_rkcq_apply (stage-wise scaled DFT fused with the
eigen-mixing of Delta(zeta_l), the batched apply at the 2L frequencies,
mixing back, inverse DFT) against the oracle's RK-CQ (oracle/rkcq.py,
pinned by the Radau IIA time-stepping identity and its order) with dense
oracle matrices at the oracle's own frequencies; argument refusals."""
import numpy as np
import pytest

import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2607_15292_b300 as g
from oracle import adjoint, bem, rkcq  # noqa: E402

N, DT = 15, 4e-5


@pytest.fixture(scope="module")
def case():
    xyz, tri = syn.box(2.0, 1.0, 1.0, 0.5)
    V = adjoint.operators(xyz, tri, syn.STEEL, rkcq.freqs_radau2(N, DT), (bem.KERNEL_SL,))[bem.KERNEL_SL]
    gs = syn.box_traction(xyz, tri, N, DT, width=0.5, t0=2.5e-4, tw=8e-5, offsets=rkcq.C_RADAU2)
    y = rkcq.convolve(lambda k, s, x: (V[k] @ x.reshape(-1)).reshape(-1, 3), gs, N, DT)
    return dict(xyz=xyz, tri=tri, g=gs, y=y.real)


def _op(c, precision, eps, freqs=None, half=False):
    ctx = g.Context(eps=eps, precision=precision, leaf=12, eta=2.0)
    ctx.material(*syn.STEEL)
    ctx.freqs(g.freqs_radau2(N, DT, half)[0] if freqs is None else freqs)
    mesh = ctx.mesh(c["xyz"], c["tri"])
    return ctx, mesh.tree(g.BEM_ROWS_NODES, g.BEM_SL).compress()


# The inverse transform multiplies each frequency's rounding by up to
# lam^-N = 1e5 (lam = (1e-10)^(1/(2N))) at the last level: FP64 (compression
# eps 1e-10) keeps 1e-7 of the largest value; MIXED carries complex64
# frequency-domain vectors (2^-24 ~ 6e-8, times 1e5) and eps 1e-6 entries.
@pytest.mark.parametrize("half", [False, True])
@pytest.mark.parametrize("precision,eps,tol", [(0, 1e-10, 1e-7), (1, 1e-6, 6e-3)])
def test_rkcq_apply_vs_oracle(case, record, precision, eps, tol, half):
    """Full set (2L frequencies) and half set (2 (floor(L/2) + 1)): the same
    result, the half set through the conjugate pairs."""
    c = case
    ctx, V = _op(c, precision, eps, half=half)
    assert V.K == (2 * (N + 1) if not half else 2 * ((N + 1) // 2 + 1))
    gt = torch.tensor(c["g"], dtype=torch.float64, device="cuda")
    y = torch.full((N + 1, 2, V.tree.n_rows, 3), float("nan"), dtype=torch.float64, device="cuda")
    g.rkcq_apply(V, gt, y, N, DT)
    err = np.abs(y.cpu().numpy() - c["y"]).max() / np.abs(c["y"]).max()
    record("rkcq_rel_err", err)
    assert err < tol, err
    y2 = torch.empty_like(y)
    g.rkcq_apply(V, gt, y2, N, DT)
    assert torch.equal(y, y2)                      # deterministic


def test_rkcq_refusals(case):
    c = case
    ctx, V = _op(c, 0, 1e-8, freqs=bem.freqs_bdf2(2 * N + 1, DT, 2 * (N + 1)))
    gt = torch.zeros((N + 1, 2, V.tree.n_cols, 3), dtype=torch.float64, device="cuda")
    y = torch.empty((N + 1, 2, V.tree.n_rows, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(g.BemError):                # BDF2 frequencies, not Radau IIA
        g.rkcq_apply(V, gt, y, N, DT)
    ctx, V = _op(c, 0, 1e-8)
    with pytest.raises(g.BemError):                # another dt
        g.rkcq_apply(V, gt, y, N, 2 * DT)
    ctx, V = _op(c, 0, 1e-8, freqs=g.freqs_radau2(N, DT)[0][:2 * ((N + 1) // 2)])
    with pytest.raises(g.BemError):                # neither the full nor the half set
        g.rkcq_apply(V, gt, y, N, DT)
    with pytest.raises(ValueError):                # stage data of the wrong shape
        g.rkcq_apply(V, gt[:, :1], y, N, DT)
