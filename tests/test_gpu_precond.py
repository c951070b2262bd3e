"""Block-Jacobi preconditioning of the K-batched solves (bem_op_set_precond,
an addition beyond the paper's unpreconditioned BiCGstab): the solutions of
C_k x_k = b_k and C_k^H x_k = b_k with and without the preconditioner agree
with the oracle's dense direct solves, on the two square operators
(single layer with centroid rows, double layer with node rows), in both
precisions; the iteration counts are recorded; refusals."""
import numpy as np
import pytest

import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2607_15292_b300 as g
from oracle import bem  # noqa: E402

S = bem.freqs_bdf2(16, 5e-5, 8)
CASES = [("sl", "centroids"), ("dl", "nodes")]


def _dense(kern, rows):
    xyz, tri = syn.icosphere(1)
    op = bem.Operator(xyz, tri, syn.STEEL, rows=rows, kernel=bem.KERNEL_SL if kern == "sl" else bem.KERNEL_DL)
    C = op.dense(S)                    # (n, n, K, 3, 3)
    return [bem.to_matrix(C[:, :, k]) for k in range(len(S))]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kern,rows", CASES)
def test_block_jacobi_solves_match_dense(kern, rows, precision, record):
    xyz, tri = syn.icosphere(1)
    ctx = g.Context(eps=1e-10 if precision == 0 else 1e-6, precision=precision, leaf=8)
    ctx.material(*syn.STEEL)
    ctx.freqs(S)
    t = ctx.mesh(xyz, tri).tree(g.BEM_ROWS_CENTROIDS if rows == "centroids" else g.BEM_ROWS_NODES,
                                g.BEM_SL if kern == "sl" else g.BEM_DL)
    op = t.compress()
    K, n = len(S), t.n_rows
    cdt = torch.complex128 if precision == 0 else torch.complex64
    B = torch.tensor(syn.complex_normal(31, (K, n, 3)), dtype=cdt, device="cuda")
    Cs = _dense(kern, rows)
    Bn = B.cpu().numpy().astype(np.complex128)
    tol = 1e-10 if precision == 0 else 1e-6
    bound = 1e-8 if precision == 0 else 3e-4
    its = {}
    for pc in (0, 1):
        op.set_precond(pc)
        for adj in (False, True):
            X = torch.empty_like(B)
            it, rr = op.solve(B, X, tol=tol, max_iter=400, adjoint=adj)
            its[(pc, adj)] = int(it.max())
            Xn = X.cpu().numpy().astype(np.complex128)
            for k in range(K):
                A = Cs[k].conj().T if adj else Cs[k]
                ref = np.linalg.solve(A, Bn[k].reshape(-1))
                err = np.linalg.norm(Xn[k].reshape(-1) - ref) / np.linalg.norm(ref)
                assert err < bound, (pc, adj, k, err)
    for (pc, adj), v in its.items():
        record(f"iters_pc{pc}_adj{int(adj)}", v)


def test_block_jacobi_refusals():
    xyz, tri = syn.icosphere(1)
    ctx = g.Context(eps=1e-6, precision=0, leaf=8)
    ctx.material(*syn.STEEL)
    ctx.freqs(S)
    op = ctx.mesh(xyz, tri).tree(g.BEM_ROWS_NODES, g.BEM_SL).compress()   # rows nodes, columns elements
    with pytest.raises(g.BemError):
        op.set_precond(1)
    with pytest.raises(g.BemError):
        op.set_precond(2)
    op.set_precond(0)
