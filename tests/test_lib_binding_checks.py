"""The Python binding refuses buffers the C ABI would misread, before any
library call: the library reads and writes device buffers by pointer and
size only, so a CPU tensor, another complex type, another shape, a strided
view or a tensor on another device would make it read or write outside the
buffer.  Runs without a GPU: a host-only context (device -1) and stand-in
tensor objects that describe a CUDA buffer without owning one."""
import numpy as np
import pytest

import synthetic as syn
import paper_2607_15292_b300 as g

torch = pytest.importorskip("torch")


class FakeCuda:
    """Describes a CUDA tensor (shape, dtype, device, layout) with no
    storage: the validation reads only these attributes, and a refused call
    never reaches the library."""

    def __init__(self, shape, dtype, device=0, contiguous=True, ptr=1 << 20):
        self.shape = tuple(shape)
        self.dtype = dtype
        self.is_cuda = True
        self.device = torch.device("cuda", device)
        self._contig = contiguous
        self._ptr = ptr

    def is_contiguous(self):
        return self._contig

    def data_ptr(self):
        return self._ptr

    def numel(self):
        return int(np.prod(self.shape))


@pytest.fixture()
def mesh():
    ctx = g.Context(device=-1, precision=g.BEM_FP64)
    ctx.material(*syn.STEEL)
    ctx.freqs([1e3 + 10j, 2e3 + 30j])
    xyz, tri = syn.cube_grid(1)
    return ctx.mesh(xyz, tri)


def test_entries_refuses_cpu_and_non_tensor_buffers(mesh):
    req = torch.zeros((4, 3), dtype=torch.int32)
    out = torch.zeros((4, 3, 3), dtype=torch.complex128)
    for call in (mesh.entries, mesh.entries_noalloc):
        with pytest.raises(ValueError, match="CUDA"):
            call(0, 0, req, out)
        with pytest.raises(ValueError):
            call(0, 0, np.zeros((4, 3), np.int32), out)


def test_entries_refuses_wrong_dtype_shape_layout_device(mesh):
    ctx = mesh.ctx
    ctx.device = 0          # describe the context as living on cuda:0 for the stand-ins
    good_req = FakeCuda((4, 3), torch.int32)
    cases = [
        (FakeCuda((4, 3), torch.int64), FakeCuda((4, 3, 3), torch.complex128), "dtype"),
        (FakeCuda((4, 2), torch.int32), FakeCuda((4, 3, 3), torch.complex128), "shape"),
        (good_req, FakeCuda((4, 3, 3), torch.complex64), "dtype"),      # c64 output in FP64: half the bytes
        (good_req, FakeCuda((5, 3, 3), torch.complex128), "shape"),
        (good_req, FakeCuda((4, 3, 3), torch.complex128, contiguous=False), "contiguous"),
        (good_req, FakeCuda((4, 3, 3), torch.complex128, device=1), "cuda:1"),
        (good_req, FakeCuda((4, 3, 3), torch.complex128, ptr=(1 << 20) + 8), "aligned"),
    ]
    for req, out, what in cases:
        for call in (mesh.entries, mesh.entries_noalloc):
            with pytest.raises(ValueError, match=what):
                call(0, 0, req, out)


def test_apply_and_solve_refuse_wrong_buffers(mesh):
    """Operator-level checks (shapes of both apply modes and of the adjoint)
    on an operator object that is never compressed: the refusal comes first."""
    tree = mesh.tree(g.BEM_ROWS_NODES, g.BEM_SL)      # 8 node rows x 12 element columns
    op = g.Operator.__new__(g.Operator)
    op.tree, op.ctx, op.K, op._p = tree, mesh.ctx, mesh.ctx.K, None
    mesh.ctx.device = 0
    K, nr, nc = op.K, tree.n_rows, tree.n_cols
    c = torch.complex128
    with pytest.raises(ValueError, match="shape"):
        op.apply(FakeCuda((K, nc, 3), c), FakeCuda((nr, 3), c))                  # batched output shape
    with pytest.raises(ValueError, match="shape"):
        op.apply(FakeCuda((K, nc, 3), c), FakeCuda((K, nr, 3), c), g.BEM_APPLY_CONTRACTED)
    with pytest.raises(ValueError, match="shape"):
        op.apply(FakeCuda((K, nc, 3), c), FakeCuda((K, nc, 3), c), transpose=1)   # adjoint takes rows in
    with pytest.raises(ValueError, match="dtype"):
        op.apply(FakeCuda((K, nc, 3), torch.complex64), FakeCuda((K, nr, 3), c))
    with pytest.raises(ValueError, match="mode"):
        op.apply(FakeCuda((K, nc, 3), c), FakeCuda((K, nr, 3), c), 7)
    with pytest.raises(ValueError, match="square"):
        op.solve(FakeCuda((K, nr, 3), c), FakeCuda((K, nr, 3), c))
    sq = mesh.tree(g.BEM_ROWS_NODES, g.BEM_DL)
    op.tree = sq
    with pytest.raises(ValueError, match="shape"):
        op.solve(FakeCuda((K, sq.n_rows + 1, 3), c), FakeCuda((K, sq.n_rows, 3), c))
    op.tree = tree
    with pytest.raises(ValueError, match="shape"):
        op.dense(FakeCuda((nr, nc, K, 3), c))


def test_cq_refuses_wrong_buffers():
    N, nvec = 8, 5
    with pytest.raises(ValueError, match="dtype"):
        g.cq_forward(N, nvec, FakeCuda((N + 1, nvec), torch.complex64), FakeCuda((N + 1, nvec), torch.complex128))
    with pytest.raises(ValueError, match="shape"):
        g.cq_inverse(N, nvec, FakeCuda((N, nvec), torch.complex128), FakeCuda((N + 1, nvec), torch.complex128))
    x = FakeCuda((N + 1, nvec), torch.complex128)
    with pytest.raises(ValueError, match="overlap"):
        g.cq_forward(N, nvec, x, x)


def test_rkcq_refuses_wrong_buffers(mesh):
    """RK-CQ apply and solve: stage buffers of the wrong dtype, shape or
    level count, and a solve on a non-square operator, are refused before
    the library is called; the C entry points refuse NULL handles."""
    tree = mesh.tree(g.BEM_ROWS_NODES, g.BEM_SL)      # 8 node rows x 12 element columns
    op = g.Operator.__new__(g.Operator)
    op.tree, op.ctx, op.K, op._p = tree, mesh.ctx, mesh.ctx.K, None
    mesh.ctx.device = 0
    N, nr, nc = 3, tree.n_rows, tree.n_cols
    f = torch.float64
    with pytest.raises(ValueError, match="dtype"):
        g.rkcq_apply(op, FakeCuda((N + 1, 2, nc, 3), torch.float32), FakeCuda((N + 1, 2, nr, 3), f), N, 1e-3)
    with pytest.raises(ValueError, match="shape"):
        g.rkcq_apply(op, FakeCuda((N + 1, 2, nr, 3), f), FakeCuda((N + 1, 2, nr, 3), f), N, 1e-3)   # rows in
    with pytest.raises(ValueError, match="shape"):
        g.rkcq_apply(op, FakeCuda((N, 2, nc, 3), f), FakeCuda((N + 1, 2, nr, 3), f), N, 1e-3)       # one level short
    with pytest.raises(ValueError, match="shape"):
        g.rkcq_apply(op, FakeCuda((N + 1, 1, nc, 3), f), FakeCuda((N + 1, 2, nr, 3), f), N, 1e-3)   # one stage
    with pytest.raises(ValueError, match="square"):
        g.rkcq_solve(op, FakeCuda((N + 1, 2, nr, 3), f), FakeCuda((N + 1, 2, nr, 3), f), N, 1e-3)
    assert g._lib.bem_rkcq_apply(None, N, 1e-3, None, None, None) == g.BEM_ERR_ARG
    it = np.zeros(8, dtype=np.int32)
    rr = np.zeros(8)
    assert g._lib.bem_rkcq_solve(None, N, 1e-3, None, None, 1e-8, 10, it.ctypes.data_as(g._P(g._i32)),
                                 rr.ctypes.data_as(g._P(g._dbl)), None) == g.BEM_ERR_ARG
    assert g._lib.bem_op_pivot_freqs(None, it.ctypes.data_as(g._P(g._i32))) == g.BEM_ERR_ARG
