"""FP64 applies are reproducible bit for bit: each block writes its
contribution to its own rows (columns in the adjoint) into a slot of a
partial buffer, and one kernel sums the blocks of every row in increasing
block order, so the result does not depend on which CTA finishes first.
Checked for the batched, contracted and adjoint applies, on an operator with
dense, 3D-ACA and low-rank-face blocks, over repeated calls and against the
oracle's dense tensor (Eq. (3.15))."""
import numpy as np
import pytest

import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2607_15292_b300 as g
from oracle import bem  # noqa: E402


def _op(kern):
    xyz, tri = syn.icosphere(2)
    s = bem.freqs_bdf2(24, 5e-5, 24)
    ctx = g.Context(eps=1e-8, precision=g.BEM_FP64, leaf=16, eta=2.0)
    ctx.material(*syn.STEEL)
    ctx.freqs(s)
    t = ctx.mesh(xyz, tri).tree(g.BEM_ROWS_NODES, kern)
    return t, t.compress(), len(s)


@pytest.mark.parametrize("kern", [0, 1])
def test_fp64_applies_bitwise_reproducible(kern):
    t, op, K = _op(kern)
    st = op.stats()
    assert st.n_aca > 0
    X = torch.tensor(syn.complex_normal(3, (K, t.n_cols, 3)), dtype=torch.complex128, device="cuda")
    Yin = torch.tensor(syn.complex_normal(4, (K, t.n_rows, 3)), dtype=torch.complex128, device="cuda")
    outs = []
    for _ in range(4):
        Y = torch.empty((K, t.n_rows, 3), dtype=torch.complex128, device="cuda")
        y = torch.empty((t.n_rows, 3), dtype=torch.complex128, device="cuda")
        XA = torch.empty((K, t.n_cols, 3), dtype=torch.complex128, device="cuda")
        op.apply(X, Y)
        op.apply(X, y, g.BEM_APPLY_CONTRACTED)
        op.apply_adjoint(Yin, XA)
        torch.cuda.synchronize()
        outs.append((Y, y, XA))
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert torch.equal(a, b)
    # and the fixed order sums the same operator: against the dense tensor
    Dn = torch.empty((t.n_rows, t.n_cols, K, 3, 3), dtype=torch.complex128, device="cuda")
    op.dense(Dn)
    D = Dn.permute(2, 0, 3, 1, 4).reshape(K, 3 * t.n_rows, 3 * t.n_cols)
    Xf = X.reshape(K, -1, 1)
    Yr = torch.bmm(D, Xf).reshape(K, t.n_rows, 3)
    Y, y, XA = outs[0]
    assert (torch.linalg.norm(Y - Yr) / torch.linalg.norm(Yr)).item() < 1e-12
    assert (torch.linalg.norm(y - Yr.sum(0)) / torch.linalg.norm(Yr.sum(0))).item() < 1e-12
    XAr = torch.bmm(D.conj().transpose(1, 2), Yin.reshape(K, -1, 1)).reshape(K, t.n_cols, 3)
    assert (torch.linalg.norm(XA - XAr) / torch.linalg.norm(XAr)).item() < 1e-12
