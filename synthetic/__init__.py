"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds only input generators: surface meshes of the workload
shapes, seeded random vectors and the material presets.  It contains none of
the boundary element method's arithmetic (no kernels, no quadrature, no
frequencies, no compression), so both the CPU oracle and the CUDA path may
take their inputs from here without sharing any computation.

Meshes are returned as ``(xyz, tri)``: ``xyz`` float64 (n_nodes, 3), ``tri``
int32 (n_tris, 3), every triangle oriented counter-clockwise when seen from
outside the solid (outward normal by the right-hand rule).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "STEEL", "PAPER_CUBE_MATERIAL", "lame_from_young",
    "cube_grid", "paper_cube", "refine", "icosphere", "ellipsoid", "cube_sphere", "slotted_cylinder",
    "SLOTTED_CYLINDER", "batch_meshes", "box", "BOX_ADJOINT", "box_receivers", "box_traction",
    "splitmix64", "uniform01", "normal", "complex_normal",
]


# --------------------------------------------------------------------------
# materials
# --------------------------------------------------------------------------

def lame_from_young(E: float, nu: float) -> tuple[float, float]:
    """Lame constants (lambda, mu) from Young's modulus and Poisson's ratio."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


_steel_lam, _steel_mu = lame_from_young(210e9, 0.3)
#: steel, rho = 7850 kg/m^3, E = 210 GPa, nu = 0.3 -> (rho, lambda, mu)
STEEL = (7850.0, _steel_lam, _steel_mu)
#: the paper's unit-cube material c1 = 1, c2 = sqrt(1/2), rho = 1 (Sec. 4.1):
#: mu = rho c2^2 = 1/2, lambda = rho c1^2 - 2 mu = 0 (nu = 0)
PAPER_CUBE_MATERIAL = (1.0, 0.0, 0.5)


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------

def _cube_face_frames():
    # (origin corner, u axis, v axis) with u x v = outward normal, unit cube
    # [-0.5, 0.5]^3
    h = 0.5
    return [
        (np.array([h, -h, -h]), np.array([0, 1, 0.]), np.array([0, 0, 1.])),   # +x
        (np.array([-h, -h, -h]), np.array([0, 0, 1.]), np.array([0, 1, 0.])),  # -x
        (np.array([-h, h, -h]), np.array([0, 0, 1.]), np.array([1, 0, 0.])),   # +y
        (np.array([-h, -h, -h]), np.array([1, 0, 0.]), np.array([0, 0, 1.])),  # -y
        (np.array([-h, -h, h]), np.array([1, 0, 0.]), np.array([0, 1, 0.])),   # +z
        (np.array([-h, -h, -h]), np.array([0, 1, 0.]), np.array([1, 0, 0.])),  # -z
    ]


class _NodeTable:
    """Merges coincident points (exact rational grid coordinates)."""

    def __init__(self, scale: int):
        self.scale = scale
        self.index: dict[tuple[int, int, int], int] = {}
        self.xyz: list[np.ndarray] = []

    def get(self, p: np.ndarray) -> int:
        key = tuple(int(round(c * self.scale)) for c in p)
        idx = self.index.get(key)
        if idx is None:
            idx = len(self.xyz)
            self.index[key] = idx
            self.xyz.append(np.asarray(p, dtype=np.float64))
        return idx


def cube_grid(n: int, size: float = 1.0) -> tuple[np.ndarray, np.ndarray]:
    """Surface of the cube [-size/2, size/2]^3, each face an n x n grid of
    squares, each square cut along its (i, j) -> (i+1, j+1) diagonal into two
    triangles: 12 n^2 triangles, 6 n^2 + 2 nodes."""
    nodes = _NodeTable(scale=4 * n)
    tris = []
    for origin, u, v in _cube_face_frames():
        def pt(i, j):
            return origin + (i / n) * u + (j / n) * v
        for i in range(n):
            for j in range(n):
                a = nodes.get(pt(i, j))
                b = nodes.get(pt(i + 1, j))
                c = nodes.get(pt(i + 1, j + 1))
                d = nodes.get(pt(i, j + 1))
                tris.append((a, b, c))
                tris.append((a, c, d))
    xyz = np.array(nodes.xyz) * size
    return xyz, np.array(tris, dtype=np.int32)


def paper_cube(level: int) -> tuple[np.ndarray, np.ndarray]:
    """The paper's unit-cube meshes (Sec. 4.1, Table 1): level 1 has 2 x 2
    squares per face, each cut into four triangles by both diagonals (96
    triangles, 50 nodes); every further level splits each triangle into four."""
    nodes = _NodeTable(scale=8)
    tris = []
    for origin, u, v in _cube_face_frames():
        def pt(x, y):
            return origin + x * u + y * v
        for i in range(2):
            for j in range(2):
                a = nodes.get(pt(i / 2, j / 2))
                b = nodes.get(pt((i + 1) / 2, j / 2))
                c = nodes.get(pt((i + 1) / 2, (j + 1) / 2))
                d = nodes.get(pt(i / 2, (j + 1) / 2))
                m = nodes.get(pt((i + 0.5) / 2, (j + 0.5) / 2))
                tris += [(a, b, m), (b, c, m), (c, d, m), (d, a, m)]
    xyz, tri = np.array(nodes.xyz), np.array(tris, dtype=np.int32)
    for _ in range(level - 1):
        xyz, tri = refine(xyz, tri)
    return xyz, tri


def refine(xyz: np.ndarray, tri: np.ndarray, project=None):
    """Uniform 1 -> 4 split of every triangle at its edge midpoints.
    ``project`` optionally maps new midpoints (e.g. onto a sphere)."""
    xyz = [p for p in np.asarray(xyz, dtype=np.float64)]
    mid: dict[tuple[int, int], int] = {}

    def midpoint(a, b):
        key = (min(a, b), max(a, b))
        idx = mid.get(key)
        if idx is None:
            p = 0.5 * (xyz[a] + xyz[b])
            if project is not None:
                p = project(p)
            idx = len(xyz)
            xyz.append(p)
            mid[key] = idx
        return idx

    out = []
    for a, b, c in np.asarray(tri):
        ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
        out += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]
    return np.array(xyz), np.array(out, dtype=np.int32)


def icosphere(level: int, radius: float = 1.0) -> tuple[np.ndarray, np.ndarray]:
    """Icosahedron refined ``level`` times with midpoints projected to the
    sphere: 20 * 4^level triangles, 10 * 4^level + 2 nodes."""
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array([
        [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
        [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
        [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int32)

    def project(p):
        return p / np.linalg.norm(p)

    for _ in range(level):
        v, f = refine(v, f, project)
    return v * radius, f


def ellipsoid(level: int, axes=(2.0, 1.0, 1.0)) -> tuple[np.ndarray, np.ndarray]:
    """Icosphere scaled to an ellipsoid with the given semi-axes."""
    xyz, tri = icosphere(level)
    return xyz * np.asarray(axes, dtype=np.float64), tri


def cube_sphere(n: int, radius: float = 1.0) -> tuple[np.ndarray, np.ndarray]:
    """cube_grid(n) with every node projected radially onto the sphere of the
    given radius: 12 n^2 triangles."""
    xyz, tri = cube_grid(n)
    return radius * xyz / np.linalg.norm(xyz, axis=1, keepdims=True), tri


def _orient_outward(xyz: np.ndarray, tri: np.ndarray) -> np.ndarray:
    """Makes the orientation of a closed triangulated surface consistent
    (breadth-first walk over shared edges: a neighbour must traverse the
    shared edge in the opposite direction), then outward (positive enclosed
    volume by the divergence theorem)."""
    tri = tri.copy()
    edge_tris = {}
    for t, (a, b, c) in enumerate(tri):
        for u, v in ((a, b), (b, c), (c, a)):
            edge_tris.setdefault((min(u, v), max(u, v)), []).append(t)
    seen = np.zeros(len(tri), dtype=bool)
    for start in range(len(tri)):
        if seen[start]:
            continue
        seen[start] = True
        stack = [start]
        while stack:
            t = stack.pop()
            a, b, c = tri[t]
            for u, v in ((a, b), (b, c), (c, a)):
                for o in edge_tris[(min(u, v), max(u, v))]:
                    if o == t or seen[o]:
                        continue
                    oa, ob, oc = tri[o]
                    same = (u, v) in ((oa, ob), (ob, oc), (oc, oa))
                    if same:          # traverses the shared edge the same way: flip
                        tri[o] = tri[o][[0, 2, 1]]
                    seen[o] = True
                    stack.append(o)
    P = xyz[tri]
    vol = np.einsum("ij,ij->i", P[:, 0], np.cross(P[:, 1], P[:, 2])).sum() / 6.0
    return tri if vol > 0 else tri[:, [0, 2, 1]]


#: slotted hollow cylinder of the large configuration: outer radius 0.3 m,
#: inner radius 0.2 m, length 0.5 m, 36 axial slots cut into the bore,
#: 0.02 m deep, 4 degrees wide, full length
SLOTTED_CYLINDER = dict(r_out=0.3, r_in=0.2, length=0.5, slots=36, depth=0.02, slot_deg=4.0)


def slotted_cylinder(n_half_land: int = 2, n_wall: int = 2, n_bottom: int = 3, n_z: int = 40, n_r: int = 7,
                     r_out: float = 0.3, r_in: float = 0.2, length: float = 0.5, slots: int = 36,
                     depth: float = 0.02, slot_deg: float = 4.0) -> tuple[np.ndarray, np.ndarray]:
    """Closed surface of a hollow cylinder (axis z, 0 <= z <= length) whose
    bore carries `slots` axial slots of the given depth and angular width.

    Every node lies on one polar grid (repeated at the axial levels): per
    slot pitch U = 2 n_half_land + n_bottom angles (half land, slot, half
    land, from the middle of one land to the middle of the next) and the
    radii r_in + depth k / n_wall (k = 0..n_wall, the slot walls) then
    r_in + depth + (r_out - r_in - depth) l / n_r (l = 1..n_r).  The bore
    profile of a pitch has S = 2 n_half_land + 2 n_wall + n_bottom segments
    (land at r_in, wall out, slot bottom at r_in + depth, wall back, land);
    the outer circle has U segments per pitch; the lateral surfaces have
    n_z axial segments; the end caps are the polar cells of the material
    (all angles beyond the slot bottoms, the land angles below them).  Every
    quadrilateral is split into two triangles along the diagonal whose
    smaller triangle is the larger: 2 slots [n_z (S + U) + 2 (U n_r +
    2 n_half_land n_wall)] triangles of a genus-one surface (V - E + F = 0).
    The defaults give 60,048 triangles, the size of the large configuration."""
    land = 2.0 * np.pi / slots - np.deg2rad(slot_deg)
    hl = 0.5 * land
    wslot = np.deg2rad(slot_deg)
    pitch = 2.0 * np.pi / slots
    U = 2 * n_half_land + n_bottom
    a_loc = np.concatenate([hl * np.arange(n_half_land) / n_half_land,
                            hl + wslot * np.arange(n_bottom) / n_bottom,
                            hl + wslot + hl * np.arange(n_half_land) / n_half_land])
    ang = (np.arange(slots)[:, None] * pitch + a_loc[None, :]).ravel()            # slots * U angles
    NA = len(ang)
    radii = np.concatenate([r_in + depth * np.arange(n_wall + 1) / n_wall,
                            r_in + depth + (r_out - r_in - depth) * np.arange(1, n_r + 1) / n_r])
    top = len(radii) - 1
    # bore profile of one pitch as (radius level, local angle index)
    prof = [(0, u) for u in range(n_half_land)]
    prof += [(k, n_half_land) for k in range(n_wall)]
    prof += [(n_wall, n_half_land + u) for u in range(n_bottom)]
    prof += [(n_wall - k, n_half_land + n_bottom) for k in range(n_wall)]
    prof += [(0, n_half_land + n_bottom + u) for u in range(n_half_land)]
    S = len(prof)
    bore = [(k, p * U + u) for p in range(slots) for k, u in prof]
    zs = np.linspace(0.0, length, n_z + 1)
    node = {}
    pts = []

    def nd(j, k, u):
        key = (j, k, u % NA)
        if key not in node:
            node[key] = len(pts)
            a = ang[u % NA]
            pts.append((radii[k] * np.cos(a), radii[k] * np.sin(a), zs[j]))
        return node[key]
    quads = []
    for j in range(n_z):
        for i in range(len(bore)):
            (k0, u0), (k1, u1) = bore[i], bore[(i + 1) % len(bore)]
            if u1 < u0:
                u1 += NA
            quads.append((nd(j, k0, u0), nd(j, k1, u1), nd(j + 1, k1, u1), nd(j + 1, k0, u0)))
        for u in range(NA):
            quads.append((nd(j, top, u), nd(j, top, u + 1), nd(j + 1, top, u + 1), nd(j + 1, top, u)))
    land_seg = [u for u in range(U) if u < n_half_land or u >= n_half_land + n_bottom]
    for j in (0, n_z):
        for k in range(top):
            segs = range(NA) if k >= n_wall else [p * U + u for p in range(slots) for u in land_seg]
            for u in segs:
                quads.append((nd(j, k, u), nd(j, k, u + 1), nd(j, k + 1, u + 1), nd(j, k + 1, u)))
    xyz = np.array(pts, dtype=np.float64)
    q = np.array(quads, dtype=np.int64)

    def area2(a, b, c):
        return np.linalg.norm(np.cross(xyz[b] - xyz[a], xyz[c] - xyz[a]), axis=1)
    d02 = np.minimum(area2(q[:, 0], q[:, 1], q[:, 2]), area2(q[:, 0], q[:, 2], q[:, 3]))
    d13 = np.minimum(area2(q[:, 0], q[:, 1], q[:, 3]), area2(q[:, 1], q[:, 2], q[:, 3]))
    use13 = d13 > d02
    t1 = np.where(use13[:, None], q[:, [0, 1, 3]], q[:, [0, 1, 2]])
    t2 = np.where(use13[:, None], q[:, [1, 2, 3]], q[:, [0, 2, 3]])
    tri = np.concatenate([t1, t2])
    return xyz, _orient_outward(xyz, tri).astype(np.int32)


def box(lx: float, ly: float, lz: float, h: float) -> tuple[np.ndarray, np.ndarray]:
    """Surface of the box [0, lx] x [0, ly] x [0, lz], each face a grid of
    squares of side h (the extents must be multiples of h), each square cut
    along one diagonal into two triangles, oriented outward.  With
    nx, ny, nz = lx/h, ly/h, lz/h: 4 (nx ny + nx nz + ny nz) triangles and
    half as many nodes plus two (closed genus-0 surface)."""
    n = [int(round(e / h)) for e in (lx, ly, lz)]
    if any(abs(k * h - e) > 1e-9 * max(1.0, e) or k < 1 for k, e in zip(n, (lx, ly, lz))):
        raise ValueError("box: extents must be positive multiples of h")
    ext = np.array([lx, ly, lz], dtype=np.float64)
    nodes = _NodeTable(scale=1)
    tris = []
    # (fixed axis, value 0 or 1, u axis, v axis): two faces per axis
    for ax in range(3):
        u_ax, v_ax = [a for a in range(3) if a != ax]
        for side in (0, 1):
            for i in range(n[u_ax]):
                for j in range(n[v_ax]):
                    def key(di, dj):
                        g = [0, 0, 0]
                        g[ax] = side * n[ax]
                        g[u_ax] = i + di
                        g[v_ax] = j + dj
                        return nodes.get(np.array(g, dtype=np.float64))
                    a, b, c, d = key(0, 0), key(1, 0), key(1, 1), key(0, 1)
                    tris.append((a, b, c))
                    tris.append((a, c, d))
    grid = np.array(nodes.xyz)
    xyz = grid * (ext / np.array(n, dtype=np.float64))
    return xyz, _orient_outward(xyz, np.array(tris, dtype=np.int32))


#: the adjoint workload: 20 x 20 x 10 m box, 0.4 m grid (20,000 triangles,
#: 10,002 nodes), Gaussian traction pulse on the top face, 64 receivers on
#: the bottom face, N = 254 BDF2 steps of 4e-5 s (128 frequencies)
BOX_ADJOINT = dict(lx=20.0, ly=20.0, lz=10.0, h=0.4, N=254, dt=4e-5, receivers=64, width=2.0, t0=2e-3, tw=5e-4)


def box_receivers(xyz: np.ndarray, n: int, seed: int = 7) -> np.ndarray:
    """n distinct node indices on the bottom face z = min z, in a seeded
    order (splitmix64 keys)."""
    z0 = xyz[:, 2].min()
    cand = np.nonzero(np.abs(xyz[:, 2] - z0) <= 1e-9 * max(1.0, float(np.abs(xyz).max())))[0]
    if n > len(cand):
        raise ValueError("box_receivers: fewer bottom-face nodes than receivers")
    order = np.argsort(splitmix64(seed, len(cand)), kind="stable")
    return np.sort(cand[order[:n]]).astype(np.int32)


def box_traction(xyz: np.ndarray, tri: np.ndarray, N: int, dt: float, width: float, t0: float, tw: float,
                 seed: int = 11, amp: float = 1e6, offsets=None) -> np.ndarray:
    """Traction samples g (N + 1, n_tris, 3) in Pa, real: on the top-face
    elements (centroid z = max z) a downward load
    amp exp(-|c - p|^2 / (2 w^2)) exp(-(t_n - t0)^2 / (2 tw^2)), p a seeded
    point of the top face; zero elsewhere.  With offsets (m values, in
    units of dt) the samples are taken at t = (n + offsets_i) dt instead:
    g (N + 1, m, n_tris, 3)."""
    c = xyz[tri].mean(axis=1)
    zt = xyz[:, 2].max()
    top = np.abs(c[:, 2] - zt) <= 1e-9 * max(1.0, float(np.abs(xyz).max()))
    lo, hi = xyz[:, :2].min(0), xyz[:, :2].max(0)
    u = uniform01(seed, 2)
    p = lo + (0.25 + 0.5 * u) * (hi - lo)
    space = np.exp(-((c[:, :2] - p) ** 2).sum(1) / (2.0 * width ** 2)) * top
    if offsets is None:
        t = dt * np.arange(N + 1)
    else:
        t = dt * (np.arange(N + 1)[:, None] + np.asarray(offsets, dtype=float)[None, :])
    time = np.exp(-((t - t0) ** 2) / (2.0 * tw ** 2))
    g = np.zeros(t.shape + (len(tri), 3))
    g[..., 2] = -amp * time[..., None] * space
    return g


def batch_meshes(count: int = 32, n_max: int = 25):
    """The multi-mesh workload: mesh i (i = 0..count-1) takes three
    splitmix64 words of seed 1000 + i: u0 mod 3 picks a cube grid, a
    cube-sphere or a 2:1:1 ellipsoid (scaled cube-sphere), 7 + u1 mod 19
    (capped at n_max) the grid size n (12 n^2 triangles, 588 to 7,500), and
    u2 mod 4 the frequency count K in {16, 32, 64, 128}.  Returns a list of
    (name, xyz, tri, K)."""
    out = []
    for i in range(count):
        u = splitmix64(1000 + i, 3)
        kind = int(u[0] % 3)
        n = min(7 + int(u[1] % 19), n_max)
        K = (16, 32, 64, 128)[int(u[2] % 4)]
        if kind == 0:
            xyz, tri = cube_grid(n)
            name = f"cube{n}"
        elif kind == 1:
            xyz, tri = cube_sphere(n)
            name = f"cubesphere{n}"
        else:
            xyz, tri = cube_sphere(n)
            xyz = xyz * np.array([2.0, 1.0, 1.0])
            name = f"ellipsoid{n}"
        out.append((name, xyz, tri, K))
    return out


# --------------------------------------------------------------------------
# seeded random numbers: splitmix64 counter stream -> uniforms -> Box-Muller
# --------------------------------------------------------------------------

_M64 = (1 << 64) - 1


def splitmix64(seed: int, n: int) -> np.ndarray:
    """First n outputs of the splitmix64 generator started at ``seed``
    (Steele, Lea, Flood 2014): state += 0x9E3779B97F4A7C15, then the
    xor-shift-multiply finaliser.  Returned as uint64."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & _M64) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int) -> np.ndarray:
    """n uniforms in (0, 1): top 53 bits of splitmix64, offset by half a ulp."""
    z = splitmix64(seed, n)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(seed: int, n: int) -> np.ndarray:
    """n standard normal float64 numbers by Box-Muller on uniform01 pairs."""
    m = (n + 1) // 2
    u = uniform01(seed, 2 * m)
    u1, u2 = u[0::2], u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * m)
    out[0::2] = rad * np.cos(2.0 * np.pi * u2)
    out[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return out[:n]


def complex_normal(seed: int, shape) -> np.ndarray:
    """complex128 array, real and imaginary parts iid N(0, 1)."""
    n = int(np.prod(shape))
    x = normal(seed, 2 * n)
    return (x[0::2] + 1j * x[1::2]).reshape(shape)
