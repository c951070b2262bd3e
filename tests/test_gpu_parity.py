"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Entries (A4/A5): element by element, FP64 within 1e-10 relative per 3x3
block, MIXED within the stated tolerance.  3D-ACA (A7) and apply (A8/A9):
the compressed tensor and the applied vectors against the oracle's dense
tensor within the 3D-ACA tolerance (pivots may differ on near-ties, so
factors are not compared).  Sizes span several tiles and ragged tails."""
import numpy as np
import pytest

import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2607_15292_b300 as g
from oracle import aca, bem  # noqa: E402

ROWS = {"nodes": 1, "centroids": 0}
KERN = {"sl": 0, "dl": 1}
N_C1, DT_C1, K_C1 = 16, 1e-4, 16
# per-block relative error bound of the MIXED (FP32) entries: u = 2^-24 times
# the cancellation of the kernel formulas (series below |s| r / c2 = 2,
# closed form above: at most e^2 < 2^3), of the quadrature sum over an
# element whose phase varies by |s| h / c2 (at most 2^2 on these meshes), and
# 2^3 for the 3 x 3 products and the float-float phase reduction
MIXED_BLOCK_TOL = 2.0 ** -16


def _ctx(s, precision=0, eps=1e-6, leaf=32, eta=2.0, material=syn.STEEL):
    ctx = g.Context(eps=eps, precision=precision, leaf=leaf, eta=eta)
    ctx.material(*material)
    ctx.freqs(s)
    return ctx


def _gpu_entries(mesh, rows, kern, req, precision):
    req_t = torch.tensor(np.asarray(req, dtype=np.int32), device="cuda")
    dt = torch.complex128 if precision == 0 else torch.complex64
    out = torch.empty((len(req), 3, 3), dtype=dt, device="cuda")
    mesh.entries(ROWS[rows], KERN[kern], req_t, out)
    return out.cpu().numpy().astype(np.complex128)


def _block_err(a, b, floor):
    num = np.linalg.norm((a - b).reshape(len(a), -1), axis=1)
    den = np.linalg.norm(b.reshape(len(b), -1), axis=1) + floor
    return (num / den).max()


CASES = [("cube2", "centroids", "sl"), ("cube2", "centroids", "dl"),
         ("ico1", "nodes", "sl"), ("ico1", "nodes", "dl"),
         ("cube2", "nodes", "dl"), ("ico1", "centroids", "sl")]


def _mesh(name):
    return syn.cube_grid(2) if name == "cube2" else syn.icosphere(1)


@pytest.mark.parametrize("name,rows,kern", CASES)
def test_entries_fp64_all_pairs(name, rows, kern):
    xyz, tri = _mesh(name)
    s = bem.freqs_bdf2(N_C1, DT_C1, K_C1)
    ctx = _ctx(s)
    mesh = ctx.mesh(xyz, tri)
    op = bem.Operator(xyz, tri, syn.STEEL, rows=rows, kernel=kern)
    ks = [0, 5, 15]
    D = op.dense(s[ks])                                        # (m, n, 3, 3, 3)
    m, n = D.shape[:2]
    req = [(i, j, k) for i in range(m) for j in range(n) for k in ks]
    got = _gpu_entries(mesh, rows, kern, req, 0)
    want = np.stack([D[i, j, ks.index(k)] for i, j, k in req])
    floor = 1e-12 * np.abs(want).max()
    assert _block_err(got, want, floor) < 1e-10


@pytest.mark.parametrize("rows,kern", [("centroids", "sl"), ("nodes", "dl")])
def test_entries_static_kernel(rows, kern):
    """k = -1 requests the s = 0 (Kelvin) kernels."""
    xyz, tri = syn.cube_grid(2)
    ctx = _ctx(bem.freqs_bdf2(N_C1, DT_C1, 4))
    mesh = ctx.mesh(xyz, tri)
    op = bem.Operator(xyz, tri, syn.STEEL, rows=rows, kernel=kern)
    D = op.dense(np.array([1e-30 + 0j]))[:, :, 0]
    req = [(i, j, -1) for i in range(D.shape[0]) for j in range(D.shape[1])]
    got = _gpu_entries(mesh, rows, kern, req, 0)
    want = np.stack([D[i, j] for i, j, _ in req])
    assert _block_err(got, want, 1e-12 * np.abs(want).max()) < 1e-10


@pytest.mark.parametrize("name,rows,kern", CASES[:4])
def test_entries_mixed(name, rows, kern, record):
    xyz, tri = _mesh(name)
    s = bem.freqs_bdf2(N_C1, DT_C1, K_C1)
    ctx = _ctx(s, precision=1)
    mesh = ctx.mesh(xyz, tri)
    op = bem.Operator(xyz, tri, syn.STEEL, rows=rows, kernel=kern)
    ks = [0, 7, 15]
    D = op.dense(s[ks])
    m, n = D.shape[:2]
    req = [(i, j, k) for i in range(m) for j in range(n) for k in ks]
    got = _gpu_entries(mesh, rows, kern, req, 1)
    want = np.stack([D[i, j, ks.index(k)] for i, j, k in req])
    eg = np.linalg.norm(got - want) / np.linalg.norm(want)
    eb = _block_err(got, want, 1e-6 * np.abs(want).max())
    record("mixed_entries_global", eg)
    record("mixed_entries_block_max", eb)
    assert eg <= 1e-6, eg
    assert eb < MIXED_BLOCK_TOL, eb


def test_entries_out_of_range_request_reports_error():
    xyz, tri = syn.cube_grid(1)
    ctx = _ctx(bem.freqs_bdf2(N_C1, DT_C1, 2))
    mesh = ctx.mesh(xyz, tri)
    req_t = torch.tensor([[0, 0, 0], [0, 999, 0], [0, 0, 7]], dtype=torch.int32, device="cuda")
    out = torch.zeros((3, 3, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(g.BemError) as e:
        mesh.entries(0, 0, req_t, out)
    assert e.value.status == g.BEM_ERR_ARG
    o = out.cpu().numpy()
    assert np.isfinite(o[0]).all() and np.isnan(o[1]).all() and np.isnan(o[2]).all()


# --------------------------------------------------------------------------
# 3D-ACA + apply
# --------------------------------------------------------------------------
_DENSE_CACHE = {}


def _oracle_dense(name, rows, kern, s):
    key = (name, rows, kern, len(s))
    if key not in _DENSE_CACHE:
        xyz, tri = _mesh(name) if name in ("cube2", "ico1") else (syn.cube_grid(4) if name == "cube4" else syn.icosphere(2))
        op = bem.Operator(xyz, tri, syn.STEEL, rows=rows, kernel=kern)
        _DENSE_CACHE[key] = op.dense(s)
    return _DENSE_CACHE[key]


def _meshx(name):
    return {"cube2": syn.cube_grid(2), "ico1": syn.icosphere(1), "cube4": syn.cube_grid(4),
            "ico2": syn.icosphere(2)}[name]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name,rows,kern,leaf", [("cube2", "centroids", "sl", 8), ("cube2", "centroids", "dl", 8),
                                                 ("ico2", "nodes", "sl", 16), ("ico2", "nodes", "dl", 16)])
def test_aca3d_tensor_and_apply(name, rows, kern, leaf, precision, record):
    eps = 1e-6
    s = bem.freqs_bdf2(N_C1, DT_C1, K_C1)
    xyz, tri = _meshx(name)
    D = _oracle_dense(name, rows, kern, s)                    # (m, n, K, 3, 3)
    ctx = _ctx(s, precision=precision, eps=eps, leaf=leaf)
    t = ctx.mesh(xyz, tri).tree(ROWS[rows], KERN[kern])
    op = t.compress()
    st = op.stats()
    assert st.n_blocks == t.n_blocks and st.n_aca + st.n_dense + st.n_rank0 == st.n_blocks
    cdt = torch.complex128 if precision == 0 else torch.complex64
    out = torch.empty(D.shape, dtype=cdt, device="cuda")
    op.dense(out)
    C = out.cpu().numpy().astype(np.complex128)
    err = np.linalg.norm(C - D) / np.linalg.norm(D)
    record("tensor_vs_dense", err)
    assert err < eps, err
    # batched apply Y_k = C_k X_k
    K = len(s)
    X = syn.complex_normal(1, (K, D.shape[1], 3))
    Xt = torch.tensor(X, dtype=cdt, device="cuda")
    Yt = torch.empty((K, D.shape[0], 3), dtype=cdt, device="cuda")
    op.apply(Xt, Yt, g.BEM_APPLY_BATCHED)
    Y = Yt.cpu().numpy()
    Yd = np.einsum("ijkab,kjb->kia", D, X)
    ea = np.linalg.norm(Y - Yd) / np.linalg.norm(Yd)
    record("apply_vs_dense", ea)
    assert ea < eps, ea
    # contracted apply y = sum_k C_k X_k
    yt = torch.empty((D.shape[0], 3), dtype=cdt, device="cuda")
    op.apply(Xt, yt, g.BEM_APPLY_CONTRACTED)
    y = yt.cpu().numpy()
    ec = np.linalg.norm(y - Yd.sum(0)) / np.linalg.norm(Yd.sum(0))
    record("contracted_vs_dense", ec)
    assert ec < eps, ec
    if precision == 0 and name == "ico2":
        assert st.n_far > 0


def test_aca3d_against_oracle_compression_config1(record):
    """Cube 4x4 squares per face (192 triangles), centroid rows, K = 16:
    GPU and oracle compressed tensors both within eps of the dense tensor."""
    eps = 1e-6
    s = bem.freqs_bdf2(N_C1, DT_C1, K_C1)
    xyz, tri = syn.cube_grid(4)
    op = bem.Operator(xyz, tri, syn.STEEL, rows="centroids", kernel="sl")
    D = _oracle_dense("cube4", "centroids", "sl", s)
    ctx = _ctx(s, eps=eps)
    gop = ctx.mesh(xyz, tri).tree(0, 0).compress()
    out = torch.empty(D.shape, dtype=torch.complex128, device="cuda")
    gop.dense(out)
    C = out.cpu().numpy()
    from oracle import pipeline
    blocks = pipeline.compress(op, s, eps, dense_tensor=D)
    Co = np.zeros_like(D)
    for b in blocks:
        Co[np.ix_(b.rows, b.cols)] = aca.block_tensor(b, len(s))
    nD = np.linalg.norm(D)
    eg, eo = np.linalg.norm(C - D) / nD, np.linalg.norm(Co - D) / nD
    record("config1_gpu_vs_dense", eg)
    record("config1_oracle_vs_dense", eo)
    assert eg < eps and eo < eps, (eg, eo)
    assert np.linalg.norm(C - Co) / nD < 2 * eps


# --------------------------------------------------------------------------
# CQ transforms (scaled DFT over the frequency circle)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("N,nvec", [(16, 7), (64, 1000), (128, 33)])
def test_cq_transforms_match_oracle(N, nvec):
    from oracle import cq
    L = N + 1
    g_host = syn.complex_normal(5, (L, nvec))
    gin = torch.tensor(g_host, dtype=torch.complex128, device="cuda")
    gh = torch.empty_like(gin)
    g.cq_forward(N, nvec, gin, gh)
    want = cq.forward(g_host, N)
    got = gh.cpu().numpy()
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    back = torch.empty_like(gin)
    g.cq_inverse(N, nvec, gh, back)
    # the inverse scales level n by lam^-n (up to 1e5): rounding grows with it
    scale = (cq.lam_c(N) ** -np.arange(L))[:, None] * np.abs(want).max() / L
    err = np.abs(back.cpu().numpy() - cq.inverse(want, N))
    assert (err <= 1e-12 * scale).all()
    assert (np.abs(back.cpu().numpy() - g_host) <= 1e-12 * scale + 1e-13 * np.abs(g_host).max()).all()


# --------------------------------------------------------------------------
# accuracy of the compressed operator against exact rows, both precisions
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kern", ["sl", "dl"])
def test_compressed_apply_within_eps_of_exact_rows(kern, record):
    """Icosphere level 3 (1,280 triangles, 642 nodes), node rows, K = 64
    frequencies of N = 64, dt = 2e-5 (the sphere workload's frequency set),
    eps = 1e-6: the batched apply of the compressed operator, FP64 and MIXED,
    against exact rows (FP64 entries, element-wise parity-checked against the
    oracle above) on 32 seeded rows, all columns and frequencies: within eps."""
    eps = 1e-6
    xyz, tri = syn.icosphere(3)
    s = bem.freqs_bdf2(64, 2e-5, 64)
    K = len(s)
    kk = KERN[kern]
    ncol = len(tri) if kern == "sl" else len(xyz)
    rows = np.sort(np.random.default_rng(9).choice(len(xyz), 32, replace=False))
    X = syn.complex_normal(4, (K, ncol, 3))
    ctxE = _ctx(s)
    r_, c_, k_ = np.meshgrid(rows, np.arange(ncol), np.arange(K), indexing="ij")
    req = np.stack([r_.ravel(), c_.ravel(), k_.ravel()], 1)
    E = _gpu_entries(ctxE.mesh(xyz, tri), "nodes", kern, req, 0).reshape(len(rows), ncol, K, 3, 3)
    Yex = np.einsum("ijkab,kjb->kia", E, X)
    for precision in (0, 1):
        ctx = _ctx(s, precision=precision, eps=eps)
        op = ctx.mesh(xyz, tri).tree(ROWS["nodes"], kk).compress()
        cdt = torch.complex128 if precision == 0 else torch.complex64
        Yt = torch.empty((K, len(xyz), 3), dtype=cdt, device="cuda")
        op.apply(torch.tensor(X, dtype=cdt, device="cuda"), Yt, g.BEM_APPLY_BATCHED)
        Y = Yt.cpu().numpy().astype(np.complex128)[:, rows]
        err = np.linalg.norm(Y - Yex) / np.linalg.norm(Yex)
        record(f"exact_rows_p{precision}", err)
        assert err < eps, (precision, err)


def test_material_change_rebuilds_rigid_body_diagonal():
    """The rigid-body diagonal of node rows depends on Poisson's ratio: after
    bem_material_set changes the material, double-layer entries and the
    compressed operator follow the new material (against the oracle)."""
    xyz, tri = syn.cube_grid(2)
    s = bem.freqs_bdf2(N_C1, DT_C1, 4)
    ctx = _ctx(s)
    mesh = ctx.mesh(xyz, tri)
    ks = [0, 3]
    req = [(i, j, k) for i in range(len(xyz)) for j in range(len(xyz)) for k in ks]
    _gpu_entries(mesh, "nodes", "dl", req, 0)            # builds the diagonal for steel
    alu = (2700.0,) + syn.lame_from_young(7.0e10, 0.33)
    ctx.material(*alu)
    got = _gpu_entries(mesh, "nodes", "dl", req, 0)
    D = bem.Operator(xyz, tri, alu, rows="nodes", kernel="dl").dense(s[ks])
    want = np.stack([D[i, j, ks.index(k)] for i, j, k in req])
    assert _block_err(got, want, 1e-12 * np.abs(want).max()) < 1e-10
    t = mesh.tree(ROWS["nodes"], KERN["dl"])
    op = t.compress()
    out = torch.empty((len(xyz), len(xyz), len(s), 3, 3), dtype=torch.complex128, device="cuda")
    op.dense(out)
    Dall = bem.Operator(xyz, tri, alu, rows="nodes", kernel="dl").dense(s)
    assert np.linalg.norm(out.cpu().numpy() - Dall) / np.linalg.norm(Dall) < 1e-6
