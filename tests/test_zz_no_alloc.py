"""bem_entries_noalloc: the raw-entry call for callers that cannot allocate
device memory during a call (code inside another framework's memory pool, a
real-time loop that cannot take an allocation's latency, a fixed memory
budget).  Its range-check scratch is a static 1 KiB device array instead of
a per-call allocation.

Checked through the C ABI against the allocating bem_entries on two calls
in a row (the shared scratch must be reset between calls), plus its limits:
an out-of-range request is reported (also one in the second 65,536-request
chunk of a call) and the next call is clean, more than 16,777,216 requests
are refused before any device work, repeated calls leave the device's free
memory unchanged, and the double layer on node rows needs its rigid-body
diagonal prepared for the current material first.  This file is collected
last so that a run stopping at the first failure has run every other test;
it passes alone in a fresh process as well."""
import numpy as np
import pytest

import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2607_15292_b300 as g
from oracle import bem  # noqa: E402

ROWS = {"nodes": 1, "centroids": 0}
KERN = {"sl": 0, "dl": 1}
TOL = {0: 1e-10, 1: 2e-5}   # relative per 3x3 block, as in test_gpu_parity.py


def _ctx(precision):
    ctx = g.Context(eps=1e-6, precision=precision)
    ctx.material(*syn.STEEL)
    ctx.freqs(bem.freqs_bdf2(16, 1e-4, 16))
    return ctx


def _requests(m, n):
    ks = [0, 7, 15, -1]
    return torch.tensor([(i, j, k) for i in range(m) for j in range(n) for k in ks], dtype=torch.int32,
                        device="cuda")


def _block_err(a, b):
    a = a.reshape(len(a), -1)
    b = b.reshape(len(b), -1)
    floor = 1e-12 * np.abs(b).max()
    return (np.linalg.norm(a - b, axis=1) / (np.linalg.norm(b, axis=1) + floor)).max()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("rows,kern", [("centroids", "sl"), ("nodes", "sl"), ("nodes", "dl"), ("centroids", "dl")])
def test_noalloc_matches_entries_on_two_calls(precision, rows, kern):
    xyz, tri = syn.cube_grid(2)
    ctx = _ctx(precision)
    mesh = ctx.mesh(xyz, tri)
    m = len(xyz) if rows == "nodes" else len(tri)
    n = len(tri) if kern == "sl" else len(xyz)
    req = _requests(m, n)
    cdt = torch.complex128 if precision == 0 else torch.complex64
    ref = torch.empty((len(req), 3, 3), dtype=cdt, device="cuda")
    mesh.entries(ROWS[rows], KERN[kern], req, ref)             # allocating call (also prepares the mesh)
    want = ref.cpu().numpy().astype(np.complex128)
    for call in range(2):
        out = torch.full((len(req), 3, 3), float("nan"), dtype=cdt, device="cuda")
        mesh.entries_noalloc(ROWS[rows], KERN[kern], req, out)
        got = out.cpu().numpy().astype(np.complex128)
        assert np.isfinite(got).all(), call
        assert _block_err(got, want) < TOL[precision], call


def test_noalloc_limits_and_error_reporting():
    xyz, tri = syn.cube_grid(1)
    ctx = _ctx(0)
    mesh = ctx.mesh(xyz, tri)
    # double layer on node rows before the rigid-body diagonal exists: refused
    req = torch.tensor([[0, 0, 0]], dtype=torch.int32, device="cuda")
    out = torch.zeros((1, 3, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(g.BemError) as e:
        mesh.entries_noalloc(1, 1, req, out)
    assert e.value.status == g.BEM_ERR_STATE
    # too many requests: refused before any device access (the buffers are
    # far smaller than n, so the refusal must happen on the host)
    big = 256 * 65536 + 1
    st = g._lib.bem_entries_noalloc(mesh._p, 0, 0, g._dptr(req), big, g._dptr(out),
                                    g._stream_ptr(None))
    assert st == g.BEM_ERR_ARG
    assert b"16777216" in g._lib.bem_last_error(ctx.ptr)
    # an out-of-range request is reported, and the next call starts clean
    bad = torch.tensor([[0, 0, 0], [0, 10 ** 6, 0], [1, 2, 3]], dtype=torch.int32, device="cuda")
    out3 = torch.zeros((3, 3, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(g.BemError) as e:
        mesh.entries_noalloc(0, 0, bad, out3)
    assert e.value.status == g.BEM_ERR_ARG and "request 1" in str(e.value)
    o = out3.cpu().numpy()
    assert np.isfinite(o[0]).all() and np.isnan(o[1]).all() and np.isfinite(o[2]).all()
    good = torch.tensor([[0, 0, 0], [1, 2, 3]], dtype=torch.int32, device="cuda")
    out2 = torch.zeros((2, 3, 3), dtype=torch.complex128, device="cuda")
    mesh.entries_noalloc(0, 0, good, out2)
    ref = torch.zeros((2, 3, 3), dtype=torch.complex128, device="cuda")
    mesh.entries(0, 0, good, ref)
    assert torch.equal(out2, ref)


def test_noalloc_second_chunk_and_no_device_allocation():
    """70,000 requests span two range-check words; a bad request at index
    65,636 (in the second word) is reported by its index, and neither call
    changes the device's free memory (nothing is allocated)."""
    xyz, tri = syn.cube_grid(1)
    ctx = _ctx(0)
    mesh = ctx.mesh(xyz, tri)
    m, n, ks = len(tri), len(tri), [0, 7, 15, -1]
    combos = np.array([(i, j, k) for i in range(m) for j in range(n) for k in ks], dtype=np.int32)
    nreq = 70000
    req_h = combos[np.arange(nreq) % len(combos)]
    req = torch.tensor(req_h, device="cuda")
    ref = torch.empty((nreq, 3, 3), dtype=torch.complex128, device="cuda")
    out = torch.empty_like(ref)
    mesh.entries(0, 0, req, ref)
    mesh.entries_noalloc(0, 0, req, out)              # first call: resolves the array's address
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        out.fill_(float("nan"))
        mesh.entries_noalloc(0, 0, req, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert _block_err(out.cpu().numpy(), ref.cpu().numpy()) < TOL[0]
    bad_h = req_h.copy()
    bad_h[65636] = (0, 10 ** 6, 0)
    bad = torch.tensor(bad_h, device="cuda")
    with pytest.raises(g.BemError) as e:
        mesh.entries_noalloc(0, 0, bad, out)
    assert e.value.status == g.BEM_ERR_ARG and "request 65636" in str(e.value)
    o = out.cpu().numpy()
    assert np.isnan(o[65636]).all() and np.isfinite(np.delete(o, 65636, axis=0)).all()
    mesh.entries_noalloc(0, 0, req, out)              # clean again
    assert _block_err(out.cpu().numpy(), ref.cpu().numpy()) < TOL[0]
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_refuses_stale_rigid_body_diagonal():
    """After bem_material_set changes Poisson's ratio, the double layer on
    node rows needs its rigid-body diagonal rebuilt (by an allocating call)
    before bem_entries_noalloc serves it again."""
    xyz, tri = syn.cube_grid(1)
    ctx = _ctx(0)
    mesh = ctx.mesh(xyz, tri)
    req = torch.tensor([[0, 0, 0], [1, 3, 5]], dtype=torch.int32, device="cuda")
    out = torch.zeros((2, 3, 3), dtype=torch.complex128, device="cuda")
    mesh.entries(1, 1, req, out)
    mesh.entries_noalloc(1, 1, req, out)
    ctx.material(2700.0, 5.1e10, 2.6e10)            # aluminium-like: another nu
    with pytest.raises(g.BemError) as e:
        mesh.entries_noalloc(1, 1, req, out)
    assert e.value.status == g.BEM_ERR_STATE
    ref = torch.zeros_like(out)
    mesh.entries(1, 1, req, ref)                     # rebuilds the diagonal for the new material
    mesh.entries_noalloc(1, 1, req, out)
    assert torch.equal(out, ref)
