"""Host side of the multi-operator work list (bem_op_compress_batch): the
job order, argument checks on host-only contexts, and the multi-mesh
workload recipe (sizes and frequency counts)."""
import numpy as np
import pytest

import synthetic as syn
import paper_2607_15292_b300 as g


def test_batch_order_longest_first_ties_by_index():
    cost = [5, 9, 9, 1, 0, 7]
    assert list(g.batch_order(cost)) == [1, 2, 5, 0, 3, 4]
    assert list(g.batch_order([])) == []
    rng = np.random.default_rng(3)
    c = rng.integers(0, 50, size=200)
    o = g.batch_order(c)
    assert sorted(o.tolist()) == list(range(200))
    assert np.all(np.diff(c[o]) <= 0)
    for a, b in zip(o[:-1], o[1:]):            # stable among equal costs
        if c[a] == c[b]:
            assert a < b


def test_batch_rejects_host_only_contexts():
    ctx = g.Context(device=-1)
    ctx.material(*syn.STEEL)
    ctx.freqs([1e3 + 0j])
    xyz, tri = syn.cube_grid(1)
    m = ctx.mesh(xyz, tri)
    trees = [m.tree(g.BEM_ROWS_NODES, g.BEM_SL), m.tree(g.BEM_ROWS_NODES, g.BEM_DL)]
    with pytest.raises(g.BemError) as e:
        g.compress_batch(trees, 2)
    assert e.value.status == g.BEM_ERR_STATE


def test_batch_workload_recipe():
    b = syn.batch_meshes()
    assert len(b) == 32
    ntri = [len(t) for _, _, t, _ in b]
    assert min(ntri) >= 588 and max(ntri) <= 7500
    assert all(n % 12 == 0 for n in ntri)
    assert {K for *_, K in b} <= {16, 32, 64, 128}
    assert len({K for *_, K in b}) == 4
    kinds = {name.rstrip("0123456789") for name, *_ in b}
    assert kinds == {"cube", "cubesphere", "ellipsoid"}
    for name, xyz, tri, K in b[:6]:
        if name.startswith("cubesphere"):
            np.testing.assert_allclose(np.linalg.norm(xyz, axis=1), 1.0, rtol=1e-14)
        if name.startswith("ellipsoid"):
            q = (xyz[:, 0] / 2) ** 2 + xyz[:, 1] ** 2 + xyz[:, 2] ** 2
            np.testing.assert_allclose(q, 1.0, rtol=1e-14)
    again = syn.batch_meshes(4)
    for (n1, x1, t1, k1), (n2, x2, t2, k2) in zip(b[:4], again):
        assert n1 == n2 and k1 == k2 and np.array_equal(x1, x2) and np.array_equal(t1, t2)


def test_op_load_rejects_host_only_context_and_missing_file(tmp_path):
    ctx = g.Context(device=-1)
    ctx.material(*syn.STEEL)
    ctx.freqs([1e3 + 0j])
    xyz, tri = syn.cube_grid(1)
    t = ctx.mesh(xyz, tri).tree(g.BEM_ROWS_NODES, g.BEM_SL)
    with pytest.raises(g.BemError) as e:
        g.Operator.load(t, str(tmp_path / "absent.op"))
    assert e.value.status == g.BEM_ERR_STATE
