"""Host-side checks of libgcqbem that need no GPU: the library loads and
exports every symbol of include/gcqbem.h, the host logic (frequencies,
cluster and block trees) matches the oracle, and invalid input is rejected
with a status (never an abort)."""
import os
import re

import numpy as np
import pytest

import synthetic as syn
import paper_2607_15292_b300 as g
from oracle import bem, pipeline

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gcqbem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bem_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(g._lib, n), n
    assert set(names) == set(g.EXPORTED)


def test_freqs_match_oracle():
    for N, dt, K in [(16, 1e-4, 16), (64, 2e-5, 64), (256, 4e-5, 128), (512, 9e-7, 256)]:
        s = g.freqs_bdf2(N, dt, K)
        np.testing.assert_allclose(s, bem.freqs_bdf2(N, dt, K), rtol=1e-14, atol=0)


@pytest.mark.parametrize("N,dt", [(1, 1e-3), (10, 4e-5), (31, 1e-4), (127, 2e-6)])
def test_radau2_freqs_and_symbols_match_oracle(N, dt):
    """The library's RK-CQ frequencies are the oracle's as a set (each of
    the two eigenvalues per l, whichever order), and its symbols
    reassemble the oracle's Delta(zeta_l): P_l diag(s_l dt) P_l^-1 =
    Delta(zeta_l), P_l^-1 P_l = I."""
    from oracle import cq, rkcq
    s, sym = g.freqs_radau2(N, dt)
    L = N + 1
    ref = rkcq.freqs_radau2(N, dt).reshape(L, 2)
    lam = cq.lam_c(N)
    for l in range(L):
        mine = s[2 * l: 2 * l + 2]
        d = min(np.abs(mine - ref[l]).max(), np.abs(mine[::-1] - ref[l]).max())
        assert d <= 1e-11 * np.abs(ref[l]).max(), (l, mine, ref[l])
        assert mine[0].imag <= mine[1].imag + 1e-12 * np.abs(mine).max()
        P, Pi = sym[l, 0], sym[l, 1]
        Dl = rkcq.delta(lam * np.exp(-2j * np.pi * l / L))
        np.testing.assert_allclose(P @ np.diag(mine * dt) @ Pi, Dl, rtol=0, atol=1e-11 * np.abs(Dl).max())
        np.testing.assert_allclose(Pi @ P, np.eye(2), rtol=0, atol=1e-12)
    with pytest.raises(g.BemError):
        g.freqs_radau2(0, dt)
    with pytest.raises(g.BemError):
        g.freqs_radau2(N, -dt)


def _perturbed_sphere(level, seed):
    xyz, tri = syn.icosphere(level)
    rng = np.random.default_rng(seed)
    return xyz * (1 + 0.05 * rng.normal(size=(len(xyz), 1))), tri


@pytest.mark.parametrize("leaf,eta", [(8, 2.0), (16, 1.0), (32, 2.0)])
@pytest.mark.parametrize("rows,kern", [(g.BEM_ROWS_NODES, g.BEM_SL), (g.BEM_ROWS_NODES, g.BEM_DL),
                                       (g.BEM_ROWS_CENTROIDS, g.BEM_SL), (g.BEM_ROWS_CENTROIDS, g.BEM_DL)])
def test_trees_bit_exact_vs_oracle(leaf, eta, rows, kern):
    """Generic (perturbed) geometry: permutations and block lists identical."""
    xyz, tri = _perturbed_sphere(3, leaf)
    ctx = g.Context(device=-1, leaf=leaf, eta=eta)
    t = ctx.mesh(xyz, tri).tree(rows, kern)
    rp, cp, bl = t.export()
    op = bem.Operator(xyz, tri, syn.STEEL, rows="nodes" if rows == g.BEM_ROWS_NODES else "centroids",
                      kernel="sl" if kern == g.BEM_SL else "dl")
    rt, ct, blocks = pipeline.trees(op, leaf, eta)
    assert (rp == rt.idx).all() and (cp == ct.idx).all()
    obl = np.array([[b.rows.offset, b.rows.size, b.cols.offset, b.cols.size, int(b.far)] for b in blocks])
    assert bl.shape == obl.shape and (bl == obl).all()


@pytest.mark.parametrize("mesh", ["cube", "sphere"])
def test_tree_valid_on_symmetric_meshes(mesh):
    """Degenerate covariances (cube, icosphere): the principal axis is not
    unique, so only validity is checked: a partition of I x J, leaf sizes,
    admissibility of far blocks."""
    xyz, tri = syn.cube_grid(6) if mesh == "cube" else syn.icosphere(3)
    ctx = g.Context(device=-1, leaf=16, eta=2.0)
    t = ctx.mesh(xyz, tri).tree(g.BEM_ROWS_NODES, g.BEM_SL)
    rp, cp, bl = t.export()
    assert sorted(rp.tolist()) == list(range(len(xyz)))
    assert sorted(cp.tolist()) == list(range(len(tri)))
    cover = np.zeros((t.n_rows, t.n_cols), np.int32)
    for r0, m, c0, n, far in bl:
        cover[r0:r0 + m, c0:c0 + n] += 1
        if not far:
            assert m <= 16 and n <= 16
    assert (cover == 1).all()
    assert t.n_far > 0


def test_invalid_input_is_rejected():
    with pytest.raises(g.BemError) as e:
        g.Context(device=-1, eps=0.0)
    assert e.value.status == g.BEM_ERR_ARG
    ctx = g.Context(device=-1)
    with pytest.raises(g.BemError) as e:
        ctx.material(7850.0, 1e11, -1.0)
    assert e.value.status == g.BEM_ERR_ARG
    xyz, tri = syn.cube_grid(1)
    bad = tri.copy()
    bad[3, 1] = len(xyz) + 5
    with pytest.raises(g.BemError) as e:
        ctx.mesh(xyz, bad)
    assert e.value.status == g.BEM_ERR_MESH
    flat = tri.copy()
    flat[0] = [0, 0, 1]
    with pytest.raises(g.BemError) as e:
        ctx.mesh(xyz, flat)
    assert e.value.status == g.BEM_ERR_MESH
    with pytest.raises(g.BemError) as e:
        ctx.freqs([-1.0 + 2j])
    assert e.value.status == g.BEM_ERR_ARG
    # device work on a host-only context is a state error, not a crash
    ctx.material(*syn.STEEL)
    ctx.freqs([1e3 + 0j])
    t = ctx.mesh(xyz, tri).tree(g.BEM_ROWS_NODES, g.BEM_SL)
    with pytest.raises(g.BemError) as e:
        t.compress(stream=0)
    assert e.value.status == g.BEM_ERR_STATE
    assert g.freqs_bdf2.__doc__
    with pytest.raises(g.BemError):
        g.freqs_bdf2(4, 1e-3, 9)        # K > N + 1


def test_derivative_kernel_trees_match_their_layer():
    """The wave-speed derivative operators share the columns and the block
    cluster tree of their layer (host-only context); unknown kernel ids are
    rejected."""
    ctx = g.Context(device=-1)
    xyz, tri = syn.icosphere(2)
    m = ctx.mesh(xyz, tri)
    for base, derived in ((g.BEM_SL, (g.BEM_SL_DCP, g.BEM_SL_DCS)), (g.BEM_DL, (g.BEM_DL_DCP, g.BEM_DL_DCS))):
        for rows in (g.BEM_ROWS_NODES, g.BEM_ROWS_CENTROIDS):
            tb = m.tree(rows, base)
            rb, cb, bb = tb.export()
            for k in derived:
                t = m.tree(rows, k)
                assert (t.n_rows, t.n_cols, t.n_blocks, t.n_far) == (tb.n_rows, tb.n_cols, tb.n_blocks, tb.n_far)
                r, c, b = t.export()
                assert np.array_equal(r, rb) and np.array_equal(c, cb) and np.array_equal(b, bb)
    for bad in (-1, 6, 99):
        with pytest.raises(g.BemError) as e:
            m.tree(g.BEM_ROWS_NODES, bad)
        assert e.value.status == g.BEM_ERR_ARG
