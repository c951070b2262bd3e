"""The tensor-core batched apply (tcgen05, kind::tf32 with split operands) of
MIXED operators, through the C ABI.

* The operand layout itself: one CTA computes D = A B^T through the same
  shared-memory planes, descriptors, MMA issue and tensor-memory read-out
  (bem_tc_selftest) against an FP64 product.
* The apply of compressed operators (dense and low-rank faces, ragged row
  tiles, every frequency tile 16/32/64, K from 16 to 128): against the
  oracle's dense tensor (within eps, like the SIMT kernel) and against the
  SIMT kernel on the same operator (the two differ by FP32 rounding only)."""
import numpy as np
import pytest

import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2607_15292_b300 as g
from oracle import bem  # noqa: E402


def _tf32(x):
    """Round float32 values to TF32 (10 explicit mantissa bits), nearest."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return b.view(np.float32)


def _hw_read(plane_vals, R, KD, swapped):
    """The (R x KD) matrix the tensor core reads from a plane written with
    the layout plane_off(r, k) = (r/8) SBO + (k/4) LBO + (r%8) 16 + (k%4) 4,
    LBO = 128, SBO = KD/4 * 128, if it interpreted the descriptor with LBO and
    SBO exchanged (diagnostic for a failing self-test)."""
    lbo, sbo = 128, KD // 4 * 128
    mem = {}
    for r in range(R):
        for k in range(KD):
            mem[(r // 8) * sbo + (k // 4) * lbo + (r % 8) * 16 + (k % 4) * 4] = plane_vals[r, k]
    out = np.zeros((R, KD), np.float32)
    for r in range(R):
        for k in range(KD):
            a = (r // 8) * (lbo if swapped else sbo) + (k // 4) * (sbo if swapped else lbo) + (r % 8) * 16 + (k % 4) * 4
            out[r, k] = mem.get(a, np.nan)
    return out


@pytest.mark.parametrize("negate", [False, True])
def test_tc_selftest_matches_fp64_product(negate, record):
    rng = np.random.default_rng(5)
    A = _tf32(rng.standard_normal((128, 32)))
    B = _tf32(rng.standard_normal((64, 32)))
    D = g.tc_selftest(A, B, negate=negate)
    want = (-1.0 if negate else 1.0) * (A.astype(np.float64) @ B.astype(np.float64).T)
    err = np.abs(D - want).max() / np.abs(want).max()
    record("tc_selftest_err", err)
    if not err < 1e-6:
        alt = _hw_read(A, 128, 32, True).astype(np.float64) @ _hw_read(B, 64, 32, True).astype(np.float64).T
        alt_err = np.nanmax(np.abs(D - alt)) / np.abs(want).max()
        pytest.fail(f"tensor-core self-test: rel err {err:.3e}; with LBO/SBO exchanged {alt_err:.3e}; "
                    f"D[0,:4]={D[0, :4]}, want {want[0, :4]}")


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


CASES = [
    # mesh, rows, kernel, leaf, N, K: ragged row tiles, several frequency tiles
    ("ico2", "nodes", "sl", 16, 16, 16),
    ("ico2", "nodes", "dl", 16, 64, 40),
    ("cube4", "centroids", "sl", 32, 64, 64),
    ("cube4", "centroids", "dl", 32, 128, 100),
]


def _mesh(name):
    return {"ico2": syn.icosphere(2), "cube4": syn.cube_grid(4)}[name]


@pytest.mark.parametrize("name,rows,kern,leaf,N,K", CASES)
def test_tc_apply_matches_oracle_and_simt(name, rows, kern, leaf, N, K, record):
    eps = 1e-6
    xyz, tri = _mesh(name)
    s = bem.freqs_bdf2(N, 1e-4 if name == "cube4" else 2e-5, K)
    ctx = g.Context(eps=eps, leaf=leaf, precision=g.BEM_MIXED)
    ctx.material(*syn.STEEL)
    ctx.freqs(s)
    t = ctx.mesh(xyz, tri).tree(1 if rows == "nodes" else 0, 0 if kern == "sl" else 1)
    op = t.compress()
    assert op.stats().apply_kernel == 1
    D = bem.Operator(xyz, tri, syn.STEEL, rows=rows, kernel=kern).dense(s)
    X = syn.complex_normal(17, (K, t.n_cols, 3))
    Xt = torch.tensor(X, dtype=torch.complex64, device="cuda")
    Yd = np.einsum("ijkab,kjb->kia", D, X)
    out = {}
    for bk in (16, 32, 64):
        op.set_apply_tile(bk)
        for kind in (1, 0):
            op.set_apply_kernel(kind)
            Y = torch.empty((K, t.n_rows, 3), dtype=torch.complex64, device="cuda")
            op.apply(Xt, Y)
            out[(bk, kind)] = Y.cpu().numpy().astype(np.complex128)
        e_tc, e_simt = _rel(out[(bk, 1)], Yd), _rel(out[(bk, 0)], Yd)
        d = _rel(out[(bk, 1)], out[(bk, 0)])
        record(f"tc_vs_oracle_bk{bk}", e_tc)
        record(f"simt_vs_oracle_bk{bk}", e_simt)
        record(f"tc_vs_simt_bk{bk}", d)
        # both within eps of the oracle's tensor; apart by FP32 rounding only
        assert e_tc < eps, (bk, e_tc, e_simt)
        assert d < eps, (bk, d)
    assert op.stats().apply_errors == 0


def test_tc_apply_with_low_rank_faces(record):
    """Two perturbed spheres 8 m apart, leaf 64 (far blocks of hundreds of
    points whose faces are stored low rank, Eq. (3.12)): the tensor-core
    apply of U' T_p against the SIMT apply and the oracle's rows."""
    base_xyz, base_tri = syn.icosphere(2)
    rng = np.random.default_rng(7)
    a = base_xyz * (1 + 0.05 * rng.normal(size=(len(base_xyz), 1)))
    b = base_xyz * (1 + 0.05 * rng.normal(size=(len(base_xyz), 1))) + np.array([8.0, 0.3, -0.2])
    xyz = np.concatenate([a, b])
    tri = np.concatenate([base_tri, base_tri + len(base_xyz)]).astype(np.int32)
    s = bem.freqs_bdf2(16, 1e-4, 16)
    ctx = g.Context(eps=1e-6, leaf=64, precision=g.BEM_MIXED)
    ctx.material(*syn.STEEL)
    ctx.freqs(s)
    t = ctx.mesh(xyz, tri).tree(g.BEM_ROWS_NODES, g.BEM_SL)
    op = t.compress()
    assert op.stats().n_faces_lowrank > 0
    X = torch.tensor(syn.complex_normal(3, (len(s), t.n_cols, 3)), dtype=torch.complex64, device="cuda")
    Y1 = torch.empty((len(s), t.n_rows, 3), dtype=torch.complex64, device="cuda")
    Y0 = torch.empty_like(Y1)
    op.apply(X, Y1)
    op.set_apply_kernel(0)
    op.apply(X, Y0)
    y1 = Y1.cpu().numpy().astype(np.complex128)
    d = _rel(y1, Y0.cpu().numpy().astype(np.complex128))
    rows = np.arange(0, t.n_rows, 7)
    R = bem.Operator(xyz, tri, syn.STEEL, rows="nodes", kernel="sl").block(rows, np.arange(t.n_cols), s)
    e = _rel(y1[:, rows], np.einsum("ijkab,kjb->kia", R, X.cpu().numpy().astype(np.complex128)))
    record("tc_vs_simt_lowrank", d)
    record("tc_vs_oracle_lowrank", e)
    assert d < 1e-6 and e < 1e-6, (d, e)


def test_apply_kernel_switch_rejects_fp64_and_bad_kind():
    ctx = g.Context(eps=1e-6, leaf=8, precision=g.BEM_FP64)
    ctx.material(*syn.STEEL)
    ctx.freqs(bem.freqs_bdf2(16, 1e-4, 4))
    xyz, tri = syn.cube_grid(1)
    op = ctx.mesh(xyz, tri).tree(0, 0).compress()
    assert op.stats().apply_kernel == 0
    with pytest.raises(g.BemError) as e:
        op.set_apply_kernel(1)
    assert e.value.status == g.BEM_ERR_ARG
    with pytest.raises(g.BemError):
        op.set_apply_kernel(2)
