"""The unit-cube Dirichlet problem of the paper's convergence study
(Sec. 4.1: the Table 1 meshes, time steps and step counts, 3D-ACA
tolerances of Table 2, c1 = 1, c2 = sqrt(1/2), rho = 1, the study's source
point and direction, the analytic field of Appendix A in oracle/stokes.py):
u prescribed at the nodes, the traction t at the element midpoints from
V t = (C + K) u by RK-CQ with 2-stage Radau IIA (bem_rkcq_apply of C + K,
then bem_rkcq_solve of V), FP64, the convergence run on the half
frequency set (conjugate pairs).  Parity with the oracle's dense RK-CQ
pipeline on level 1; the error against the analytic traction on levels 1
to 4 and its order (first order expected for the piecewise constant
traction).  Level 4 (6,144 elements, half set K = 82) runs in MIXED: its
FP64 operators (~140 GB with the half set) do not fit beside the
compression's working storage; FP32 entry rounding (~1e-7) is far below
its discretisation error (~2e-2 relative)."""
import time

import numpy as np
import pytest

import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2607_15292_b300 as g
from oracle import rkcq, stokes  # noqa: E402

MAT = syn.PAPER_CUBE_MATERIAL
SRC = stokes.CUBE_SOURCE
LEVELS = {1: (0.3, 10, 1e-2), 2: (0.15, 20, 1e-3), 3: (0.075, 40, 1e-4), 4: (0.0375, 80, 1e-5)}  # dt, N, eps


def _geometry(lev):
    xyz, tri = syn.paper_cube(lev)
    c = xyz[tri].mean(1)
    nrm = np.cross(xyz[tri[:, 1]] - xyz[tri[:, 0]], xyz[tri[:, 2]] - xyz[tri[:, 0]])
    area = 0.5 * np.linalg.norm(nrm, axis=1)
    return xyz, tri, c, nrm / (2.0 * area)[:, None], area


def _analytic(lev):
    xyz, tri, c, nrm, area = _geometry(lev)
    dt, N, _ = LEVELS[lev]
    ts = rkcq.stage_times(N, dt)[:, :, None]
    u = stokes.displacement(xyz[None, None], ts, MAT, SRC["p"], SRC["d"], SRC["a"], SRC["tc"])
    t = stokes.traction(c[None, None], nrm[None, None], ts, MAT, SRC["p"], SRC["d"], SRC["a"], SRC["tc"])
    return u, t


def _library(lev, u, eps, precision=0, half=False):
    xyz, tri, _, _, _ = _geometry(lev)
    dt, N, _ = LEVELS[lev]
    ctx = g.Context(eps=eps, precision=precision, leaf=16, eta=2.0)
    ctx.material(*MAT)
    ctx.freqs(g.freqs_radau2(N, dt, half)[0])
    mesh = ctx.mesh(xyz, tri)
    t0 = time.perf_counter()
    V = mesh.tree(g.BEM_ROWS_CENTROIDS, g.BEM_SL).compress()
    A = mesh.tree(g.BEM_ROWS_CENTROIDS, g.BEM_DL).compress()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    ud = torch.tensor(u, dtype=torch.float64, device="cuda")
    b = torch.empty((N + 1, 2, len(tri), 3), dtype=torch.float64, device="cuda")
    g.rkcq_apply(A, ud, b, N, dt)
    t = torch.empty_like(b)
    it, rr = g.rkcq_solve(V, b, t, N, dt, tol=1e-10 if precision == 0 else 1e-7, max_iter=1000)
    t2 = time.perf_counter()
    st = [V.stats(), A.stats()]
    return t.cpu().numpy(), it, (t1 - t0, t2 - t1, [x.stored_bytes / 1e9 for x in st], [x.rank_mean for x in st])


def _lmax(th, t, area):
    """max over the steps of the L2 norm in space of the error at the step
    points t_(n+1) (the last stage)."""
    e = th[:, 1] - t[:, 1]
    return float(np.sqrt((area[None, :] * (e ** 2).sum(-1)).sum(-1)).max())


@pytest.mark.parametrize("half", [False, True])
def test_cube_dirichlet_level1_vs_oracle(record, half):
    xyz, tri, _, _, _ = _geometry(1)
    dt, N, _ = LEVELS[1]
    u, _ = _analytic(1)
    ref = rkcq.dirichlet_traction(xyz, tri, MAT, u, N, dt)
    th, it, _ = _library(1, u, 1e-10, half=half)
    err = np.abs(th - ref).max() / np.abs(ref).max()
    record("cube_l1_rel_err_vs_oracle", err)
    assert err < 1e-6, err


def test_cube_dirichlet_convergence(record):
    errs = []
    for lev in (1, 2, 3, 4):
        u, t = _analytic(lev)
        th, it, (tc, ts, gb, rk) = _library(lev, u, LEVELS[lev][2], precision=0 if lev < 4 else 1, half=True)
        area = _geometry(lev)[4]
        e = _lmax(th, t, area)
        errs.append(e)
        record(f"cube_l{lev}_lmax", e)
        record(f"cube_l{lev}_lmax_rel", e / _lmax(np.zeros_like(t), t, area))
        record(f"cube_l{lev}_iters_max", int(it.max()))
        record(f"cube_l{lev}_compress_s", tc)
        record(f"cube_l{lev}_rkcq_s", ts)
        for name, a, b in (("stored_gb", *gb), ("rank_mean", *rk)):
            record(f"cube_l{lev}_{name}_V", a)
            record(f"cube_l{lev}_{name}_A", b)
    eoc = [np.log2(errs[i] / errs[i + 1]) for i in range(3)]
    for i, e in enumerate(eoc):
        record(f"cube_eoc_{i + 1}{i + 2}", e)
    assert all(errs[i + 1] < errs[i] for i in range(3)), errs
    assert min(eoc) > 1.0, (errs, eoc)


def test_cube_pivot_frequencies(record):
    """The frequencies Algorithm 1 keeps (bem_op_pivot_freqs) on level 2 of
    the cube, half set, both operators: valid (k_1 = 0, one index per face,
    each at most once per block, in range, -1 beyond the rank and for
    dense and rank-0 blocks); the share of blocks using each frequency and
    the mean Re(s) of the kept frequencies against the set's are recorded
    (the paper observes that small Re(s) is preferred)."""
    xyz, tri, _, _, _ = _geometry(2)
    dt, N, eps = LEVELS[2]
    s = g.freqs_radau2(N, dt, True)[0]
    ctx = g.Context(eps=eps, precision=0, leaf=16, eta=2.0)
    ctx.material(*MAT)
    ctx.freqs(s)
    mesh = ctx.mesh(xyz, tri)
    K = len(s)
    for name, kern in (("V", g.BEM_SL), ("A", g.BEM_DL)):
        op = mesh.tree(g.BEM_ROWS_CENTROIDS, kern).compress()
        ks, info = op.pivot_freqs(), op.blocks()
        aca = (info[:, 0] == 0) & (info[:, 1] > 0)
        assert aca.any()
        for b in np.nonzero(aca)[0]:
            r = int(info[b, 1])
            row = ks[b]
            assert row[0] == 0 and row[0] == info[b, 2]
            assert ((row[:r] >= 0) & (row[:r] < K)).all() and len(set(row[:r].tolist())) == r
            assert (row[r:] == -1).all()
        assert (ks[~aca] == -1).all()
        counts = np.bincount(ks[ks >= 0], minlength=K)
        share = counts / aca.sum()
        top = np.argsort(-counts)[:4]
        for i, k in enumerate(top):
            record(f"pivot_{name}_top{i}_k", int(k))
            record(f"pivot_{name}_top{i}_share", float(share[k]))
            record(f"pivot_{name}_top{i}_re_s", float(s[k].real))
        record(f"pivot_{name}_mean_re_s_kept", float((counts * s.real).sum() / counts.sum()))
        record(f"pivot_{name}_mean_re_s_set", float(s.real.mean()))
        record(f"pivot_{name}_unused", int((counts == 0).sum()))
