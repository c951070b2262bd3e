"""Checkpoint of a compressed operator (bem_op_save / bem_op_load): the
loaded operator has the same block outcomes, face ranks and statistics
counts and applies exactly as the saved one (batched, contracted and
adjoint; dense reconstruction bit for bit); files of another tree or
precision, truncated files and files with a flipped payload byte are
rejected with BEM_ERR_ARG."""
import os

import numpy as np
import pytest

import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2607_15292_b300 as g
from oracle import bem  # noqa: E402


def _ctx(s, precision, leaf=16):
    ctx = g.Context(eps=1e-6, precision=precision, leaf=leaf)
    ctx.material(*syn.STEEL)
    ctx.freqs(s)
    return ctx


def _two_spheres(level, offset, seed):
    """Two perturbed icospheres `offset` apart: far blocks large enough for
    low-rank faces (the factor pairs of the file format)."""
    xyz, tri = syn.icosphere(level)
    rng = np.random.default_rng(seed)
    a = xyz * (1 + 0.05 * rng.normal(size=(len(xyz), 1)))
    b = xyz * (1 + 0.05 * rng.normal(size=(len(xyz), 1))) + np.array([offset, 0.3, -0.2])
    return np.concatenate([a, b]), np.concatenate([tri, tri + len(xyz)]).astype(np.int32)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kern,geom", [(0, "sphere"), (1, "sphere"), (0, "two")])
def test_save_load_roundtrip(tmp_path, precision, kern, geom):
    xyz, tri = syn.icosphere(2) if geom == "sphere" else _two_spheres(2, 8.0, 7)
    s = bem.freqs_bdf2(16, 1e-4, 16)
    K = len(s)
    ctx = _ctx(s, precision, leaf=16 if geom == "sphere" else 64)
    mesh = ctx.mesh(xyz, tri)
    t = mesh.tree(g.BEM_ROWS_NODES, kern)
    op = t.compress()
    if geom == "two":
        assert op.stats().n_faces_lowrank > 0        # factor pairs are in the file
    path = str(tmp_path / "op.bin")
    op.save(path)
    op2 = g.Operator.load(t, path)
    sa, sb = op.stats(), op2.stats()
    for f in ("n_blocks", "n_aca", "n_dense", "n_rank0", "rank_max", "rank_mean", "stored_bytes", "n_faces",
              "n_faces_lowrank", "apply_bytes", "apply_bk"):
        assert getattr(sa, f) == getattr(sb, f), f
    assert np.array_equal(op.blocks(), op2.blocks())
    assert np.array_equal(op.face_ranks(), op2.face_ranks())
    cdt = torch.complex128 if precision == 0 else torch.complex64
    da = torch.empty((t.n_rows, t.n_cols, K, 3, 3), dtype=cdt, device="cuda")
    db = torch.empty_like(da)
    op.dense(da)
    op2.dense(db)
    assert torch.equal(da, db)
    X = torch.tensor(syn.complex_normal(3, (K, t.n_cols, 3)), dtype=cdt, device="cuda")
    tol = 1e-13 if precision == 0 else 1e-6       # FP64 atomics across blocks in any order
    for mode, shape in ((g.BEM_APPLY_BATCHED, (K, t.n_rows, 3)), (g.BEM_APPLY_CONTRACTED, (t.n_rows, 3))):
        ya = torch.empty(shape, dtype=cdt, device="cuda")
        yb = torch.empty_like(ya)
        op.apply(X, ya, mode)
        op2.apply(X, yb, mode)
        assert (torch.linalg.norm((ya - yb).to(torch.complex128)) <= tol * torch.linalg.norm(ya.to(torch.complex128)))
    Yin = torch.tensor(syn.complex_normal(4, (K, t.n_rows, 3)), dtype=cdt, device="cuda")
    xa = torch.empty((K, t.n_cols, 3), dtype=cdt, device="cuda")
    xb = torch.empty_like(xa)
    op.apply_adjoint(Yin, xa)
    op2.apply_adjoint(Yin, xb)
    assert torch.linalg.norm((xa - xb).to(torch.complex128)) <= tol * torch.linalg.norm(xa.to(torch.complex128))


def test_load_rejects_mismatch_and_corruption(tmp_path):
    xyz, tri = syn.icosphere(2)
    s = bem.freqs_bdf2(16, 1e-4, 16)
    ctx = _ctx(s, 0)
    mesh = ctx.mesh(xyz, tri)
    t = mesh.tree(g.BEM_ROWS_NODES, g.BEM_SL)
    path = str(tmp_path / "op.bin")
    t.compress().save(path)
    bad = [mesh.tree(g.BEM_ROWS_NODES, g.BEM_DL),                       # another kernel
           _ctx(s, 1).mesh(xyz, tri).tree(g.BEM_ROWS_NODES, g.BEM_SL),  # another precision
           _ctx(s[:8], 0).mesh(xyz, tri).tree(g.BEM_ROWS_NODES, g.BEM_SL)]   # another K
    for tb in bad:
        with pytest.raises(g.BemError) as e:
            g.Operator.load(tb, path)
        assert e.value.status == g.BEM_ERR_ARG
    raw = open(path, "rb").read()
    trunc = str(tmp_path / "trunc.bin")
    open(trunc, "wb").write(raw[: len(raw) // 2])
    flip = str(tmp_path / "flip.bin")
    b = bytearray(raw)
    b[len(b) - 100] ^= 0x01
    open(flip, "wb").write(bytes(b))
    for p in (trunc, flip, str(tmp_path / "absent.bin")):
        with pytest.raises(g.BemError) as e:
            g.Operator.load(t, p)
        assert e.value.status == g.BEM_ERR_ARG
    assert os.path.getsize(path) > 0
    g.Operator.load(t, path)                       # the intact file still loads
