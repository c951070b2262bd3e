"""Parity at many frequencies and large phases (the large configuration's
range): K = 128 of N = 256 and K = 256 of N = 512 BDF2 frequencies, with
phases Im(s) r / c2 up to ~500 rad between collocation point and element.

* Entries against the oracle, element by element on sampled (row, column)
  pairs at every frequency: on a unit cube (dt chosen so that the largest
  sampled phase reaches 500 rad) and on the slotted hollow cylinder of the
  large configuration itself (60,048 triangles, dt = 0.6 h / c1).  FP64
  within 1e-10 per 3x3 block; MIXED within the per-block bound of the FP32
  entry path (see MIXED_BLOCK_TOL).
* Compression (eps = 1e-5, the large configuration's tolerance) and batched
  apply at K = 256 on a coarse slotted cylinder, both precisions, against
  exact rows (FP64 entries, element-wise parity-checked above)."""
import numpy as np
import pytest

import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2607_15292_b300 as g
from oracle import bem  # noqa: E402

ROWS, KERN = {"nodes": 1, "centroids": 0}, {"sl": 0, "dl": 1}
RHO, LAM, MU = syn.STEEL
C1, C2 = np.sqrt((LAM + 2 * MU) / RHO), np.sqrt(MU / RHO)
# per-block relative error of the FP32 entry path: u = 2^-24 times the
# cancellation of the kernel formulas (series below |s| r / c2 = 2, closed
# form above: at most e^2 < 2^3), of the quadrature sum over an element
# (at most 2^2), and 2^3 for the 3 x 3 products and the float-float phase
# reduction: 2^-24 2^3 2^2 2^3 = 2^-16 on resolved meshes.  Within an element
# the phase exp(-i Im(s) dr / c2) of a quadrature point is taken in FP32 at
# the offset dr from the reference distance, with an error of u Im(s) h / c2:
# on meshes whose elements span more than 2^3 rad the bound grows in
# proportion, MIXED_BLOCK_TOL * max(1, max Im(s) h / (2^3 c2)).
MIXED_BLOCK_TOL = 2.0 ** -16


def _mixed_tol(s, xyz, tri):
    P = xyz[tri]
    h = np.linalg.norm(np.concatenate([P[:, 1] - P[:, 0], P[:, 2] - P[:, 1], P[:, 0] - P[:, 2]]), axis=1).max()
    return MIXED_BLOCK_TOL * max(1.0, np.abs(s.imag).max() * h / (8.0 * C2))


def _ctx(s, precision, eps=1e-6):
    ctx = g.Context(eps=eps, precision=precision)
    ctx.material(*syn.STEEL)
    ctx.freqs(s)
    return ctx


def _h_mean(xyz, tri):
    P = xyz[tri]
    return float(np.linalg.norm(np.concatenate([P[:, 1] - P[:, 0], P[:, 2] - P[:, 1], P[:, 0] - P[:, 2]]),
                                axis=1).mean())


def _pairs(xyz, tri, kern, rows, per_row, seed):
    """For each row: the columns nearest to it (singular and near rules) and
    seeded random columns (all distances up to the diameter)."""
    rng = np.random.default_rng(seed)
    geo_c = xyz[tri].mean(axis=1) if kern == "sl" else xyz
    out = []
    for i in rows:
        d = np.linalg.norm(geo_c - xyz[i], axis=1)
        near = np.argsort(d)[:4]
        far = np.argsort(d)[-2:]
        rnd = rng.choice(len(geo_c), per_row - 6, replace=False)
        out.append((i, np.unique(np.concatenate([near, far, rnd]))))
    return out


def _check_entries(xyz, tri, kern, s, rows, per_row, seed, tol_mixed, record):
    op = bem.Operator(xyz, tri, syn.STEEL, rows="nodes", kernel=kern)
    pairs = _pairs(xyz, tri, kern, rows, per_row, seed)
    K = len(s)
    want = np.concatenate([op.block([i], cols, s)[0] for i, cols in pairs])          # (P, K, 3, 3)
    req = np.array([(i, j, k) for i, cols in pairs for j in cols for k in range(K)], dtype=np.int32)
    geo_c = xyz[tri].mean(axis=1) if kern == "sl" else xyz
    r = np.array([np.linalg.norm(geo_c[j] - xyz[i]) for i, cols in pairs for j in cols])
    phase = (np.abs(s.imag)[None, :] * r[:, None] / C2).max()
    errs = {}
    for precision in (0, 1):
        ctx = _ctx(s, precision)
        mesh = ctx.mesh(xyz, tri)
        cdt = torch.complex128 if precision == 0 else torch.complex64
        out = torch.empty((len(req), 3, 3), dtype=cdt, device="cuda")
        mesh.entries(ROWS["nodes"], KERN[kern], torch.tensor(req, device="cuda"), out)
        got = out.cpu().numpy().astype(np.complex128).reshape(want.shape)
        nrm = np.linalg.norm(want.reshape(len(want), K, 9), axis=2)                     # (P, K)
        floor = (1e-12 if precision == 0 else 1e-6) * nrm.max(axis=0, keepdims=True)
        e = np.linalg.norm((got - want).reshape(len(want), K, 9), axis=2) / (nrm + floor)
        errs[precision] = float(e.max())
        record(f"entries_block_max_p{precision}", errs[precision])
    record("max_phase_rad", phase)
    assert errs[0] < 1e-10, (errs, phase)
    assert errs[1] < tol_mixed, (errs, phase)
    return phase


@pytest.mark.parametrize("N,K", [(256, 128), (512, 256)])
@pytest.mark.parametrize("kern", ["sl", "dl"])
def test_entries_large_phase_cube(N, K, kern, record):
    """Unit cube, 2 x 2 squares per face: dt such that the largest phase
    Im(s_k) r / c2 over the frequencies and the cube's diameter is 500 rad
    (the sampled pairs reach at least 400): elements far larger than the
    wavelength and the decay length, where the MIXED reference exponential
    must not produce 0 x inf."""
    xyz, tri = syn.cube_grid(2)
    s1 = bem.freqs_bdf2(N, 1.0, K)
    rmax = np.sqrt(3.0)
    dt = np.abs(s1.imag).max() * rmax / (C2 * 500.0)
    s = bem.freqs_bdf2(N, dt, K)
    rows = np.arange(len(xyz))[::3]
    phase = _check_entries(xyz, tri, kern, s, rows, 12, 7, _mixed_tol(s, xyz, tri), record)
    assert phase > 400.0


@pytest.mark.parametrize("kern", ["sl", "dl"])
def test_entries_slotted_cylinder_config5(kern, record):
    """The large configuration's mesh (60,048 triangles), K = 256 of N = 512,
    dt = 0.6 h / c1: 12 seeded rows x 24 columns x 256 frequencies."""
    xyz, tri = syn.slotted_cylinder()
    dt = 0.6 * _h_mean(xyz, tri) / C1
    s = bem.freqs_bdf2(512, dt, 256)
    rows = np.random.default_rng(3).choice(len(xyz), 12, replace=False)
    tol = _mixed_tol(s, xyz, tri)
    assert tol < 1.5 * MIXED_BLOCK_TOL      # elements spanning ~2^3 rad at the largest Im(s): about resolved
    phase = _check_entries(xyz, tri, kern, s, rows, 24, 11, tol, record)
    assert phase > 300.0


def test_compress_apply_k256_slotted_cylinder_eps_1e5(record):
    """Coarse 12-slot variant of the slotted cylinder (1,536 triangles),
    K = 256 of N = 512, dt = 0.6 h / c1, eps = 1e-5: the batched apply of
    the compressed single and double layers, FP64 and MIXED, against exact
    rows on 16 seeded rows, all columns and frequencies: within eps."""
    xyz, tri = syn.slotted_cylinder(n_half_land=1, n_wall=1, n_bottom=1, n_z=6, n_r=2, slots=12)
    assert len(tri) == 1536
    eps = 1e-5
    dt = 0.6 * _h_mean(xyz, tri) / C1
    s = bem.freqs_bdf2(512, dt, 256)
    K = len(s)
    rows = np.sort(np.random.default_rng(21).choice(len(xyz), 16, replace=False))
    ctxE = _ctx(s, 0)
    meshE = ctxE.mesh(xyz, tri)
    for kern in ("sl", "dl"):
        ncol = len(tri) if kern == "sl" else len(xyz)
        X = syn.complex_normal(30 + KERN[kern], (K, ncol, 3))
        r_, c_, k_ = np.meshgrid(rows, np.arange(ncol), np.arange(K), indexing="ij")
        req = torch.tensor(np.stack([r_.ravel(), c_.ravel(), k_.ravel()], 1).astype(np.int32), device="cuda")
        E = torch.empty((req.shape[0], 3, 3), dtype=torch.complex128, device="cuda")
        meshE.entries(ROWS["nodes"], KERN[kern], req, E)
        Yex = torch.einsum("ijkab,kjb->kia", E.view(len(rows), ncol, K, 3, 3),
                           torch.tensor(X, device="cuda")).cpu().numpy()
        del E, req
        for precision in (0, 1):
            ctx = _ctx(s, precision, eps)
            op = ctx.mesh(xyz, tri).tree(ROWS["nodes"], KERN[kern]).compress()
            cdt = torch.complex128 if precision == 0 else torch.complex64
            Y = torch.empty((K, len(xyz), 3), dtype=cdt, device="cuda")
            op.apply(torch.tensor(X, dtype=cdt, device="cuda"), Y)
            got = Y.cpu().numpy().astype(np.complex128)[:, rows]
            err = np.linalg.norm(got - Yex) / np.linalg.norm(Yex)
            st = op.stats()
            record(f"k256_{kern}_p{precision}_err", err)
            record(f"k256_{kern}_p{precision}_rank_mean", st.rank_mean)
            record(f"k256_{kern}_p{precision}_compression_rate", st.compression_rate)
            assert err < eps, (kern, precision, err, op.stats().rank_mean)
            del op
            torch.cuda.empty_cache()
