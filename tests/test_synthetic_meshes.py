"""Pins of the synthetic slotted hollow cylinder (the large configuration's
mesh): counts from the construction, a closed and consistently oriented
genus-one surface, outward normals on every face kind, and the enclosed
volume equal to the polygonal cross-section's area times the length."""
import numpy as np
import pytest

import synthetic as syn


def _shoelace(p):
    x, y = p[:, 0], p[:, 1]
    return 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))


@pytest.mark.parametrize("params", [dict(n_half_land=1, n_wall=1, n_bottom=1, n_z=3, n_r=2, slots=6),
                                    dict(n_half_land=2, n_wall=2, n_bottom=3, n_z=4, n_r=3, slots=36)])
def test_slotted_cylinder_is_closed_outward_and_counted(params):
    xyz, tri = syn.slotted_cylinder(**params)
    nh, nw, nb = params["n_half_land"], params["n_wall"], params["n_bottom"]
    S, U = 2 * nh + 2 * nw + nb, 2 * nh + nb
    assert len(tri) == 2 * params["slots"] * (params["n_z"] * (S + U) + 2 * (U * params["n_r"] + 2 * nh * nw))
    # every directed edge once, its reverse once: closed and consistently oriented
    d = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])
    keys = d[:, 0].astype(np.int64) * len(xyz) + d[:, 1]
    rev = d[:, 1].astype(np.int64) * len(xyz) + d[:, 0]
    assert len(np.unique(keys)) == len(keys)
    assert np.array_equal(np.sort(keys), np.sort(rev))
    E = len(keys) // 2
    assert len(xyz) - E + len(tri) == 0                      # genus one
    P = xyz[tri]
    cr = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    area = 0.5 * np.linalg.norm(cr, axis=1)
    assert area.min() > 0
    nrm = cr / (2 * area[:, None])
    # outward normals: outer wall radially out, bore lands radially in, caps -z / +z
    r = np.linalg.norm(xyz[:, :2], axis=1)
    c = P.mean(axis=1)
    rhat = np.concatenate([c[:, :2] / np.linalg.norm(c[:, :2], axis=1, keepdims=True), np.zeros((len(c), 1))], 1)
    g = syn.SLOTTED_CYLINDER
    on_out = np.all(np.isclose(r[tri], g["r_out"]), axis=1) & ~np.all(np.isclose(xyz[tri][:, :, 2], 0.0), axis=1) \
        & ~np.all(np.isclose(xyz[tri][:, :, 2], g["length"]), axis=1)
    on_land = np.all(np.isclose(r[tri], g["r_in"]), axis=1) & ~np.all(np.isclose(xyz[tri][:, :, 2], 0.0), axis=1) \
        & ~np.all(np.isclose(xyz[tri][:, :, 2], g["length"]), axis=1)
    assert on_out.sum() > 0 and on_land.sum() > 0
    assert (np.einsum("ij,ij->i", nrm[on_out], rhat[on_out]) > 0.99).all()
    assert (np.einsum("ij,ij->i", nrm[on_land], rhat[on_land]) < -0.99).all()
    bot = np.all(np.isclose(xyz[tri][:, :, 2], 0.0), axis=1)
    top = np.all(np.isclose(xyz[tri][:, :, 2], g["length"]), axis=1)
    assert np.allclose(nrm[bot, 2], -1.0) and np.allclose(nrm[top, 2], 1.0)
    # enclosed volume = (outer polygon - bore polygon) x length, exactly
    vol = np.einsum("ij,ij->i", P[:, 0], np.cross(P[:, 1], P[:, 2])).sum() / 6.0
    # the boundary of the z = 0 cap: two closed loops (outer circle, bore
    # profile), walked edge by edge; cross-section = outer - bore polygon
    cap = tri[bot]
    de = {(int(a), int(b)) for t in cap for a, b in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0]))}
    nxt = {a: b for a, b in de if (b, a) not in de}
    loops = []
    while nxt:
        a0, loop = next(iter(nxt)), []
        a = a0
        while True:
            loop.append(a)
            a = nxt.pop(a)
            if a == a0:
                break
        loops.append(xyz[loop])
    assert len(loops) == 2
    radii = [np.linalg.norm(lp[:, :2], axis=1) for lp in loops]
    outer, bore = (0, 1) if radii[0].max() > radii[1].max() else (1, 0)
    assert np.allclose(radii[outer], g["r_out"]) and len(loops[outer]) == params["slots"] * U
    assert len(loops[bore]) == params["slots"] * S
    want = (_shoelace(loops[outer]) - _shoelace(loops[bore])) * g["length"]
    assert vol == pytest.approx(want, rel=1e-12)
    # slot geometry: bore radii between r_in and r_in + depth, both reached
    assert radii[bore].min() == pytest.approx(g["r_in"]) and radii[bore].max() == pytest.approx(g["r_in"] + g["depth"])


def test_slotted_cylinder_default_is_the_large_configuration_size():
    xyz, tri = syn.slotted_cylinder()
    assert len(tri) == 60048


@pytest.mark.parametrize("dims", [(1.0, 1.0, 0.5, 0.5), (3.0, 2.0, 1.0, 0.5), (20.0, 20.0, 10.0, 0.4)])
def test_box_counts_volume_and_closed_orientation(dims):
    lx, ly, lz, h = dims
    xyz, tri = syn.box(lx, ly, lz, h)
    nx, ny, nz = (round(e / h) for e in (lx, ly, lz))
    assert len(tri) == 4 * (nx * ny + nx * nz + ny * nz)
    assert len(xyz) == len(tri) // 2 + 2                    # Euler: closed genus-0 triangulation
    P = xyz[tri]
    assert np.einsum("ij,ij->i", P[:, 0], np.cross(P[:, 1], P[:, 2])).sum() / 6.0 == pytest.approx(lx * ly * lz)
    # every directed edge appears once and its reverse once: closed, consistently oriented
    de = [(int(a), int(b)) for t in tri for a, b in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0]))]
    assert len(set(de)) == len(de) and all((b, a) in set(de) for a, b in de[:2000])
    assert np.allclose(xyz.min(0), 0.0) and np.allclose(xyz.max(0), (lx, ly, lz))


def test_box_adjoint_workload_inputs():
    w = syn.BOX_ADJOINT
    xyz, tri = syn.box(w["lx"], w["ly"], w["lz"], w["h"])
    assert (len(tri), len(xyz)) == (20000, 10002)
    rec = syn.box_receivers(xyz, w["receivers"])
    assert len(np.unique(rec)) == 64 and np.allclose(xyz[rec, 2], 0.0)
    g = syn.box_traction(xyz, tri, 20, w["dt"], w["width"], w["t0"], w["tw"])
    loaded = np.abs(g).sum(axis=(0, 2)) > 0
    c = xyz[tri].mean(axis=1)
    assert loaded.any() and np.allclose(c[loaded, 2], w["lz"])   # top face only
    assert np.all(g[:, :, :2] == 0.0) and np.all(g[:, :, 2] <= 0.0)
