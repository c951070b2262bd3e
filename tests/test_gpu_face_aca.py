"""Face ACA + QR/SVD recompression (Sec. 3.1, Eq. (3.12)) through the C ABI,
against the FP64 oracle.

Single faces (bem_face_compress, the step bem_op_compress applies to every
face of a far block): an exactly separable face is recovered at its rank,
a Laplace-domain single-layer face between two separated spheres matches
the oracle's aca_matrix + recompress in rank and error, and a full-rank
face stays dense.  Operator level: two separated spheres, whose coupling
blocks are large enough for low-rank faces to be smaller than dense ones;
sampled rows of the compressed tensor and of both applies against the
oracle, the apply against the operator's own dense reconstruction, and the
face compression turned off."""
import numpy as np
import pytest

import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2607_15292_b300 as g
from oracle import aca, bem  # noqa: E402

N_C1, DT_C1, K_C1 = 16, 1e-4, 16
EPS = 1e-6


def _two_spheres(level, offset, seed):
    """Two perturbed unit icospheres with centres `offset` apart.  Blocks
    coupling them are far and hold hundreds of points, so low-rank faces are
    smaller than dense ones; the perturbation (generic geometry, no
    symmetric ties in the PCA splits) keeps the trees deterministic."""
    xyz, tri = syn.icosphere(level)
    rng = np.random.default_rng(seed)
    a = xyz * (1 + 0.05 * rng.normal(size=(len(xyz), 1)))
    b = xyz * (1 + 0.05 * rng.normal(size=(len(xyz), 1))) + np.array([offset, 0.3, -0.2])
    return np.concatenate([a, b]), np.concatenate([tri, tri + len(xyz)]).astype(np.int32)


def _ctx(precision, s=None, **kw):
    ctx = g.Context(eps=EPS, precision=precision, **kw)
    ctx.material(*syn.STEEL)
    ctx.freqs(bem.freqs_bdf2(N_C1, DT_C1, K_C1) if s is None else s)
    return ctx


def _gpu_face(ctx, H, eps_face, precision):
    m, n = H.shape[:2]
    Ht = torch.tensor(H, dtype=torch.complex128, device="cuda")
    cdt = torch.complex128 if precision == 0 else torch.complex64
    out = torch.zeros(9 * m * n, dtype=cdt, device="cuda")
    k = ctx.face_compress(Ht, eps_face, out)
    if k < 0:
        return k, None
    f = out.cpu().numpy().astype(np.complex128)
    U = f[:3 * m * k].reshape(k, 3 * m).T
    W = f[3 * m * k:3 * (m + n) * k].reshape(k, 3 * n).T
    M = U @ W.T                                    # 3m x 3n, rows (i, a), columns (j, b)
    return k, M.reshape(m, 3, n, 3).transpose(0, 2, 1, 3)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("precision", [0, 1])
def test_face_compress_separable_face_exact_rank(precision):
    m, n, r = 40, 56, 4
    A = syn.complex_normal(11, (r, m, 3, 3))
    B = syn.complex_normal(12, (r, n, 3, 3))
    H = np.einsum("tiac,tjcb->ijab", A, B)        # sum_t A_t[i] B_t[j]: rank 3 r as a 3m x 3n matrix
    lr = aca.aca_matrix(H, 1e-8)
    assert lr is not None and lr.U.shape[1] == 3 * r
    k, Hg = _gpu_face(_ctx(precision), H, 1e-8, precision)
    assert k == 3 * r
    assert _rel(Hg, H) < (1e-12 if precision == 0 else 2e-6)


@pytest.mark.parametrize("precision", [0, 1])
def test_face_compress_kernel_face_matches_oracle(precision):
    """Single-layer face V(s_0) between the two spheres (162 nodes x 320
    elements): rank and accuracy of the GPU against the oracle's ACA."""
    xyz, tri = _two_spheres(2, 8.0, 7)
    s = bem.freqs_bdf2(N_C1, DT_C1, K_C1)
    op = bem.Operator(xyz, tri, syn.STEEL, rows="nodes", kernel="sl")
    H = op.block(np.arange(162), np.arange(320, 640), s[:1])[:, :, 0]
    eps_face = 1e-8 if precision == 0 else 1e-6
    lr = aca.aca_matrix(H, eps_face)
    ko = lr.U.shape[1]
    eo = _rel(lr.matrix().reshape(162, 3, 320, 3).transpose(0, 2, 1, 3), H)
    assert ko * (162 + 320) < 3 * 162 * 320 and eo < 3 * eps_face
    k, Hg = _gpu_face(_ctx(precision), H, eps_face, precision)
    assert k >= 0
    eg = _rel(Hg, H)
    if precision == 0:
        # the GPU stops on the face's own norm, the oracle on the norm of the
        # partial sum: the two may stop one ACA step (3 ranks) apart
        assert abs(k - ko) <= max(3, ko // 20), (k, ko)
        assert eg < 3 * eps_face, eg
    else:
        assert abs(k - ko) <= max(3, ko // 10), (k, ko)
        assert eg < 4 * eps_face, eg


@pytest.mark.parametrize("precision", [0, 1])
def test_face_compress_full_rank_face_stays_dense(precision):
    H = syn.complex_normal(5, (6, 7, 3, 3))
    k, _ = _gpu_face(_ctx(precision), H, 1e-8, precision)
    assert k == -1


_ROWS = {}


def _oracle_rows(kern, rows_idx):
    key = (kern, tuple(rows_idx))
    if key not in _ROWS:
        xyz, tri = _two_spheres(2, 8.0, 7)
        s = bem.freqs_bdf2(N_C1, DT_C1, K_C1)
        op = bem.Operator(xyz, tri, syn.STEEL, rows="nodes", kernel=kern)
        ncol = len(tri) if kern == "sl" else len(xyz)
        _ROWS[key] = op.block(np.asarray(rows_idx), np.arange(ncol), s)      # (r, n, K, 3, 3)
    return _ROWS[key]


def _operator(precision, kern, compress_faces=1):
    xyz, tri = _two_spheres(2, 8.0, 7)
    ctx = _ctx(precision, leaf=64, compress_faces=compress_faces)
    t = ctx.mesh(xyz, tri).tree(g.BEM_ROWS_NODES, g.BEM_SL if kern == "sl" else g.BEM_DL)
    return ctx, t, t.compress()


def _gpu_dense(op, t, precision):
    cdt = torch.complex128 if precision == 0 else torch.complex64
    out = torch.empty((t.n_rows, t.n_cols, K_C1, 3, 3), dtype=cdt, device="cuda")
    op.dense(out)
    return out


ROWS_SAMPLE = sorted(set(np.random.default_rng(3).choice(324, 40, replace=False).tolist()) | {0, 161, 162, 323})


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kern", ["sl", "dl"])
def test_operator_with_low_rank_faces(kern, precision):
    ctx, t, op = _operator(precision, kern)
    st = op.stats()
    fr = op.face_ranks()
    assert fr.shape == (K_C1, t.n_blocks)
    assert st.n_faces == (fr >= -1).sum() and st.n_faces_lowrank == (fr >= 0).sum()
    assert st.n_faces_lowrank > 0, "no face stored low rank"
    assert (op.blocks()[:, 3] == (fr >= 0).sum(0)).all()
    _, _, tb = t.export()
    for b in np.nonzero((fr >= 0).any(0))[0]:
        m, n = tb[b, 1], tb[b, 3]
        assert tb[b, 4] == 1 and (fr[:, b][fr[:, b] >= 0] * (m + n) < 3 * m * n).all()
    R = _oracle_rows(kern, ROWS_SAMPLE)
    C = _gpu_dense(op, t, precision)[ROWS_SAMPLE].cpu().numpy().astype(np.complex128)
    assert _rel(C, R) < EPS, _rel(C, R)
    K = K_C1
    cdt = torch.complex128 if precision == 0 else torch.complex64
    X = syn.complex_normal(3, (K, t.n_cols, 3))
    Xt = torch.tensor(X, dtype=cdt, device="cuda")
    Yt = torch.empty((K, t.n_rows, 3), dtype=cdt, device="cuda")
    op.apply(Xt, Yt, g.BEM_APPLY_BATCHED)
    Y = Yt.cpu().numpy()[:, ROWS_SAMPLE]
    Yo = np.einsum("ijkab,kjb->kia", R, X)
    assert _rel(Y, Yo) < EPS, _rel(Y, Yo)
    Yc = np.einsum("ijkab,kjb->kia", C, X)       # the operator's own reconstruction
    assert _rel(Y, Yc) < (1e-12 if precision == 0 else 1e-5)
    yt = torch.empty((t.n_rows, 3), dtype=cdt, device="cuda")
    op.apply(Xt, yt, g.BEM_APPLY_CONTRACTED)
    ec = _rel(yt.cpu().numpy()[ROWS_SAMPLE], Yo.sum(0))
    assert ec < EPS, ec


def test_face_compression_off_stores_dense_faces():
    _, t, op0 = _operator(0, "sl", compress_faces=0)
    _, _, op1 = _operator(0, "sl", compress_faces=1)
    fr0, fr1 = op0.face_ranks(), op1.face_ranks()
    assert (fr0 <= -1).all() and (fr0 == -1).sum() == (fr1 >= -1).sum()
    s0, s1 = op0.stats(), op1.stats()
    assert s0.n_faces_lowrank == 0 and s1.n_faces_lowrank > 0 and s1.stored_bytes < s0.stored_bytes
    C0 = _gpu_dense(op0, t, 0)
    C1 = _gpu_dense(op1, t, 0)
    # face ACA error: eps_aca = eps / 100 per face, relative to that face
    assert (torch.linalg.norm(C1 - C0) / torch.linalg.norm(C0)).item() < EPS
