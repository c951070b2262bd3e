"""Failure detection without a GPU fault.

The faults are made on the host side: bem_debug_set makes the 3D-ACA face
kernel treat its staged face copies as not landed (after they have landed,
so nothing is left in flight) or caps the compression's device allocations;
bad inputs are NaN values in the solve's right-hand side or the apply's
input.  Each case checks the status the library returns and that the
context stays usable: the next call on it gives the normal result."""
import numpy as np
import pytest

import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2607_15292_b300 as g
from oracle import bem  # noqa: E402


def _tree(precision=0, K=16, level=1, kernel=0):
    ctx = g.Context(eps=1e-6, precision=precision, leaf=8)
    ctx.material(*syn.STEEL)
    ctx.freqs(bem.freqs_bdf2(16, 1e-4, K))
    xyz, tri = syn.icosphere(level)
    return ctx.mesh(xyz, tri).tree(g.BEM_ROWS_NODES, kernel)


def _dense(op):
    t = op.tree
    cdt = torch.complex128 if op.ctx.precision == 0 else torch.complex64
    out = torch.empty((t.n_rows, t.n_cols, op.K, 3, 3), dtype=cdt, device="cuda")
    op.dense(out)
    return out.cpu().numpy()


@pytest.mark.parametrize("precision", [0, 1])
def test_face_copy_timeout_path_returns_error_and_context_recovers(precision):
    t = _tree(precision)
    ref = _dense(t.compress())
    g.debug_set(g.BEM_DEBUG_FACE_WAIT_FAIL, 1)
    try:
        with pytest.raises(g.BemError) as e:
            t.compress()
        assert e.value.status == g.BEM_ERR_CUDA and "did not complete" in str(e.value)
    finally:
        g.debug_set(g.BEM_DEBUG_FACE_WAIT_FAIL, 0)
    torch.cuda.synchronize()
    again = _dense(t.compress())
    assert np.array_equal(again, ref)     # same work, same order: bitwise the same operator


def test_allocation_cap_gives_oom_and_context_recovers():
    t = _tree(0)
    ref = _dense(t.compress())
    free0 = torch.cuda.mem_get_info()[0]
    g.debug_set(g.BEM_DEBUG_ALLOC_CAP, 64 * 1024)
    try:
        with pytest.raises(g.BemError) as e:
            t.compress()
        assert e.value.status == g.BEM_ERR_OOM
    finally:
        g.debug_set(g.BEM_DEBUG_ALLOC_CAP, 0)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (4 << 20)    # what the failed call held is released
    assert np.array_equal(_dense(t.compress()), ref)
    with pytest.raises(g.BemError) as e:
        g.debug_set(g.BEM_DEBUG_ALLOC_CAP, -1)
    assert e.value.status == g.BEM_ERR_ARG
    with pytest.raises(g.BemError):
        g.debug_set(99, 1)


def test_solve_refuses_nan_right_hand_side():
    t = _tree(0, K=8, kernel=g.BEM_DL)       # C + K on node rows: square
    op = t.compress()
    K, n = op.K, t.n_rows
    B = torch.tensor(syn.complex_normal(3, (K, n, 3)), dtype=torch.complex128, device="cuda")
    X = torch.empty_like(B)
    B[2, 5, 1] = complex(float("nan"), 0.0)
    with pytest.raises(g.BemError) as e:
        op.solve(B, X, tol=1e-8)
    assert e.value.status == g.BEM_ERR_ARG
    B[2, 5, 1] = 0.0
    it, rr = op.solve(B, X, tol=1e-8)
    assert (rr <= 1e-8).all()


@pytest.mark.parametrize("precision", [0, 1])
def test_apply_propagates_nan_only_into_its_frequency(precision):
    t = _tree(precision, K=8)
    op = t.compress()
    K = op.K
    cdt = torch.complex128 if precision == 0 else torch.complex64
    X = torch.tensor(syn.complex_normal(4, (K, t.n_cols, 3)), dtype=cdt, device="cuda")
    X[3, 7, 0] = complex(float("nan"), 0.0)
    Y = torch.empty((K, t.n_rows, 3), dtype=cdt, device="cuda")
    op.apply(X, Y)
    y = Y.cpu().numpy()
    assert np.isnan(y[3]).any()                                  # not hidden
    assert np.isfinite(np.delete(y, 3, axis=0)).all()            # and not spread to other frequencies
