"""Multi-operator work list (bem_op_compress_batch) on the device: several
meshes of the multi-mesh workload, each with its own frequency count, plus a
single and a double layer sharing one mesh (the rigid-body diagonal is built
before the workers start), compressed from one work list on three streams.
Every operator equals the one bem_op_compress builds alone (dense
reconstruction and rank statistics), and the apply of a batched operator is
within the 3D-ACA tolerance of the oracle's dense product."""
import numpy as np
import pytest

import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2607_15292_b300 as g
from oracle import bem, kernels  # noqa: E402


def _freqs(xyz, tri, K):
    """N = K, dt = 0.6 h / c1 with h the mean edge length."""
    e = np.concatenate([xyz[tri[:, 1]] - xyz[tri[:, 0]], xyz[tri[:, 2]] - xyz[tri[:, 1]]])
    h = np.linalg.norm(e, axis=1).mean()
    c1 = kernels.wave_speeds(*syn.STEEL)[0]
    return bem.freqs_bdf2(K, 0.6 * h / c1, K)


def _setup(precision):
    jobs = []
    for name, xyz, tri, K in syn.batch_meshes(5, n_max=5):
        ctx = g.Context(eps=1e-6, precision=precision, leaf=16)
        ctx.material(*syn.STEEL)
        ctx.freqs(_freqs(xyz, tri, K))
        mesh = ctx.mesh(xyz, tri)
        jobs.append((name, xyz, tri, mesh.tree(g.BEM_ROWS_NODES, g.BEM_SL)))
    name, xyz, tri, t = jobs[0]
    jobs.append((name + "-dl", xyz, tri, t.mesh.tree(g.BEM_ROWS_NODES, g.BEM_DL)))
    return jobs


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_sequential(precision):
    seq = [(n, x, tr, t.compress()) for n, x, tr, t in _setup(precision)]
    jobs = _setup(precision)
    ops = g.compress_batch([t for *_, t in jobs], n_streams=3)
    cdt = torch.complex128 if precision == 0 else torch.complex64
    for (name, xyz, tri, a), b in zip(seq, ops):
        ta, tb = a.tree, b.tree
        assert (ta.n_rows, ta.n_cols, a.K) == (tb.n_rows, tb.n_cols, b.K), name
        sa, sb = a.stats(), b.stats()
        assert (sa.n_aca, sa.n_dense, sa.n_rank0, sa.rank_max) == (sb.n_aca, sb.n_dense, sb.n_rank0, sb.rank_max), name
        assert (sa.rank_mean, sa.stored_bytes, sa.n_faces_lowrank) == (sb.rank_mean, sb.stored_bytes, sb.n_faces_lowrank), name
        da = torch.empty((ta.n_rows, ta.n_cols, a.K, 3, 3), dtype=cdt, device="cuda")
        db = torch.empty_like(da)
        a.dense(da)
        b.dense(db)
        assert torch.equal(da, db), name


def test_batch_apply_against_oracle():
    jobs = _setup(0)
    ops = g.compress_batch([t for *_, t in jobs], n_streams=4)
    name, xyz, tri, t = jobs[3]
    op = ops[3]
    s = _freqs(xyz, tri, op.K)
    D = bem.Operator(xyz, tri, syn.STEEL, rows=bem.ROWS_NODES, kernel=bem.KERNEL_SL).dense(s)
    X = syn.complex_normal(7, (op.K, len(tri), 3))
    Y = torch.empty((op.K, len(xyz), 3), dtype=torch.complex128, device="cuda")
    op.apply(torch.tensor(X, device="cuda"), Y)
    Yd = np.einsum("ijkab,kjb->kia", D, X)
    assert np.linalg.norm(Y.cpu().numpy() - Yd) / np.linalg.norm(Yd) < 1e-5, name
