"""CUDA-graph capture of the apply: bem_op_apply issues only stream-ordered
work (kernel launches and memsets on the given stream; no allocation, no host
synchronisation), so a caller can capture a sequence of applies once and
replay it with new vector contents.  Checked: replays of a captured batched
apply, contracted apply and adjoint apply equal direct calls, for new inputs
written into the captured buffers between replays (bitwise in FP64, whose
apply sums the blocks of every row in a fixed order)."""
import numpy as np
import pytest

import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2607_15292_b300 as g
from oracle import bem  # noqa: E402


@pytest.mark.parametrize("precision", [0, 1])
def test_apply_captured_in_cuda_graph(precision):
    xyz, tri = syn.icosphere(2)
    s = bem.freqs_bdf2(16, 1e-4, 16)
    K = len(s)
    ctx = g.Context(eps=1e-6, precision=precision, leaf=16)
    ctx.material(*syn.STEEL)
    ctx.freqs(s)
    t = ctx.mesh(xyz, tri).tree(g.BEM_ROWS_NODES, g.BEM_DL)
    op = t.compress()
    cdt = torch.complex128 if precision == 0 else torch.complex64
    X = torch.zeros((K, t.n_cols, 3), dtype=cdt, device="cuda")
    Yin = torch.zeros((K, t.n_rows, 3), dtype=cdt, device="cuda")
    Y = torch.empty((K, t.n_rows, 3), dtype=cdt, device="cuda")
    y = torch.empty((t.n_rows, 3), dtype=cdt, device="cuda")
    XA = torch.empty((K, t.n_cols, 3), dtype=cdt, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):          # warm-up outside the capture
        op.apply(X, Y)
        op.apply(X, y, g.BEM_APPLY_CONTRACTED)
        op.apply_adjoint(Yin, XA)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        op.apply(X, Y)
        op.apply(X, y, g.BEM_APPLY_CONTRACTED)
        op.apply_adjoint(Yin, XA)
    for seed in (1, 2):
        X.copy_(torch.tensor(syn.complex_normal(seed, X.shape), dtype=cdt))
        Yin.copy_(torch.tensor(syn.complex_normal(seed + 10, Yin.shape), dtype=cdt))
        graph.replay()
        torch.cuda.synchronize()
        Yd = torch.empty_like(Y)
        yd = torch.empty_like(y)
        XAd = torch.empty_like(XA)
        op.apply(X, Yd)
        op.apply(X, yd, g.BEM_APPLY_CONTRACTED)
        op.apply_adjoint(Yin, XAd)
        torch.cuda.synchronize()
        # the same kernels on the same data: FP64 sums the blocks of a row in a
        # fixed order (bitwise equal); MIXED adds them with FP64 atomics
        for a, b in ((Y, Yd), (y, yd), (XA, XAd)):
            if precision == 0:
                assert torch.equal(a, b), seed
            else:
                err = (torch.linalg.norm((a - b).to(torch.complex128)) /
                       torch.linalg.norm(b.to(torch.complex128))).item()
                assert err < 1e-6, (seed, err)
        assert np.isfinite(Y.cpu().numpy()).all()
