"""Frequency tile of the batched apply (16, 32 or 64 frequencies per CTA)
and its autotune (bem_op_autotune): every tile gives the same apply (each
frequency's arithmetic is the same; only the FP64 atomics across blocks
may add in another order), the default follows K, and the autotune times
all three on the operator, keeps the fastest, and the apply stays within
the 3D-ACA tolerance of the oracle's dense product."""
import numpy as np
import pytest

import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2607_15292_b300 as g
from oracle import bem  # noqa: E402


@pytest.mark.parametrize("precision", [0, 1])
def test_apply_tiles_agree_and_autotune(precision):
    xyz, tri = syn.icosphere(2)
    s = bem.freqs_bdf2(16, 1e-4, 16)
    K = len(s)
    ctx = g.Context(eps=1e-6, precision=precision, leaf=16)
    ctx.material(*syn.STEEL)
    ctx.freqs(s)
    op = ctx.mesh(xyz, tri).tree(g.BEM_ROWS_NODES, g.BEM_SL).compress()
    assert op.stats().apply_bk == 16            # smallest tile >= K
    cdt = torch.complex128 if precision == 0 else torch.complex64
    X = torch.tensor(syn.complex_normal(2, (K, len(tri), 3)), dtype=cdt, device="cuda")
    outs = {}
    for bk in (16, 32, 64):
        op.set_apply_tile(bk)
        Y = torch.empty((K, len(xyz), 3), dtype=cdt, device="cuda")
        op.apply(X, Y)
        outs[bk] = Y.cpu().numpy().astype(np.complex128)
    tol = 1e-13 if precision == 0 else 1e-6
    for bk in (32, 64):
        assert np.linalg.norm(outs[bk] - outs[16]) <= tol * np.linalg.norm(outs[16]), bk
    with pytest.raises(g.BemError) as e:
        op.set_apply_tile(48)
    assert e.value.status == g.BEM_ERR_ARG
    best = op.autotune()
    st = op.stats()
    assert best in (16, 32, 64) and st.apply_bk == best
    assert all(t > 0 for t in st.apply_tune_ms)
    assert st.apply_tune_ms[(16, 32, 64).index(best)] == min(st.apply_tune_ms)
    Y = torch.empty((K, len(xyz), 3), dtype=cdt, device="cuda")
    op.apply(X, Y)
    D = bem.Operator(xyz, tri, syn.STEEL, rows=bem.ROWS_NODES, kernel=bem.KERNEL_SL).dense(s)
    Yd = np.einsum("ijkab,kjb->kia", D, X.cpu().numpy().astype(np.complex128))
    assert np.linalg.norm(Y.cpu().numpy() - Yd) / np.linalg.norm(Yd) < 1e-5
