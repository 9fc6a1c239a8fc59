"""Seeded synthetic workloads: meshes, array layouts, incidence angles, test vectors.

This module holds geometry and random numbers only, none of the method's
arithmetic (no basis functions, integrals, grids or operators).  Both the
CPU oracle and the CUDA library consume what it produces, so it is the one
module they share.

Units: lengths in wavelengths (lambda = 1, k0 = 2*pi).

Workloads (the paper measures on its own reflectarray/helix geometries, which
it does not publish; these seeded loop arrays stand in for them):

* square PEC loop, outer side 0.4, trace width 0.04, zero thickness, z = 0,
  meshed by a seeded Delaunay triangulation (~400 RWG edges);
* equivalent box 0.45 x 0.45 x 0.1 around each element, structured mesh with
  outward-oriented triangles (~300 RWG edges);
* arrays of such elements on a 0.5 pitch in the z = 0 plane;
* PEC spheres (icosphere) for the Mie-series checks.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.spatial import Delaunay

MASTER_SEED = 20171206


def rng(config_index: int, stream: int = 0) -> np.random.Generator:
    """Independent PCG64 substream for (config, stream)."""
    return np.random.Generator(np.random.PCG64([MASTER_SEED, int(config_index), int(stream)]))


@dataclass
class Mesh:
    """Triangle mesh: vertices (nv, 3) float64 and triangles (nt, 3) int32."""

    xyz: np.ndarray
    tri: np.ndarray
    name: str = ""

    def __post_init__(self):
        self.xyz = np.ascontiguousarray(self.xyz, dtype=np.float64)
        self.tri = np.ascontiguousarray(self.tri, dtype=np.int32)

    def translated(self, d) -> "Mesh":
        return Mesh(self.xyz + np.asarray(d, dtype=np.float64)[None, :], self.tri.copy(), self.name)

    def areas(self) -> np.ndarray:
        p = self.xyz[self.tri]
        return 0.5 * np.linalg.norm(np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), axis=1)


def _square_ring(side: float, n_per_side: int) -> np.ndarray:
    """Points on the boundary of a centred square, n_per_side segments per side, CCW."""
    h = side / 2.0
    corners = np.array([[-h, -h], [h, -h], [h, h], [-h, h]])
    pts = []
    for c in range(4):
        a, b = corners[c], corners[(c + 1) % 4]
        for i in range(n_per_side):
            t = i / n_per_side
            pts.append(a + t * (b - a))
    return np.array(pts)


def square_loop_mesh(outer: float = 0.4, width: float = 0.04, spacing: float = 0.0185,
                     gen: np.random.Generator | None = None, jitter: float = 0.25) -> Mesh:
    """Seeded Delaunay mesh of a square annulus (zero-thickness PEC loop) at z = 0.

    Nodes: the outer and inner boundary squares at `spacing`, plus a middle ring
    whose nodes are shifted along the ring by up to +-jitter*spacing (seeded).
    """
    if gen is None:
        gen = rng(0, 1)
    inner = outer - 2.0 * width
    n_out = max(4, int(round(outer / spacing)))
    n_in = max(4, int(round(inner / spacing)))
    mid = outer - width
    n_mid = max(4, int(round(mid / spacing)))
    p_out = _square_ring(outer, n_out)
    p_in = _square_ring(inner, n_in)
    p_mid = _square_ring(mid, n_mid)
    # jitter the middle ring along its sides (corners stay put)
    hmid = mid / 2.0
    step = mid / n_mid
    for i in range(len(p_mid)):
        if i % n_mid == 0:
            continue
        side = i // n_mid
        d = np.array([[1, 0], [0, 1], [-1, 0], [0, -1]][side], dtype=np.float64)
        p_mid[i] += d * gen.uniform(-jitter, jitter) * step
    pts = np.vstack([p_out, p_mid, p_in])
    dt = Delaunay(pts)
    tri = dt.simplices.copy()
    cen = pts[tri].mean(axis=1)
    hi = inner / 2.0
    keep = ~((np.abs(cen[:, 0]) < hi) & (np.abs(cen[:, 1]) < hi))
    tri = tri[keep]
    # CCW orientation (normal +z)
    p = pts[tri]
    cr = (p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) - (p[:, 1, 1] - p[:, 0, 1]) * (p[:, 2, 0] - p[:, 0, 0])
    flip = cr < 0
    tri[flip] = tri[flip][:, [0, 2, 1]]
    xyz = np.zeros((len(pts), 3))
    xyz[:, :2] = pts
    m = Mesh(xyz, tri, "square_loop")
    area = m.areas().sum()
    want = outer * outer - inner * inner
    if abs(area - want) > 1e-9 * want or m.areas().min() < 1e-6 * want / len(tri):
        raise RuntimeError("loop triangulation failed validation; change the seed or spacing")
    return m


def box_mesh(lx: float = 0.45, ly: float = 0.45, lz: float = 0.1,
             nx: int = 6, ny: int = 6, nz: int = 1) -> Mesh:
    """Structured, closed, outward-oriented triangulation of a centred box."""
    verts: dict[tuple[int, int, int], int] = {}
    xyz: list[list[float]] = []
    n = (nx, ny, nz)
    L = (lx, ly, lz)

    def vid(i, j, k):
        key = (i, j, k)
        if key not in verts:
            verts[key] = len(xyz)
            xyz.append([-L[0] / 2 + L[0] * i / nx, -L[1] / 2 + L[1] * j / ny, -L[2] / 2 + L[2] * k / nz])
        return verts[key]

    tris: list[list[int]] = []
    for axis in range(3):
        b, c = (axis + 1) % 3, (axis + 2) % 3  # e_b x e_c = e_axis
        for side in (0, 1):
            for ib in range(n[b]):
                for ic in range(n[c]):
                    def node(db, dc):
                        idx = [0, 0, 0]
                        idx[axis] = side * n[axis]
                        idx[b] = ib + db
                        idx[c] = ic + dc
                        return vid(*idx)
                    q00, q10, q11, q01 = node(0, 0), node(1, 0), node(1, 1), node(0, 1)
                    if side == 1:  # outward normal +e_axis: (b, c) order is CCW
                        tris.append([q00, q10, q11])
                        tris.append([q00, q11, q01])
                    else:          # outward normal -e_axis: reverse
                        tris.append([q00, q11, q10])
                        tris.append([q00, q01, q11])
    return Mesh(np.array(xyz), np.array(tris), "box")


def icosphere_mesh(radius: float = 0.2, level: int = 2) -> Mesh:
    """Icosahedron subdivided `level` times and projected on the sphere (outward CCW)."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = [[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0], [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
         [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]]
    f = [[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11], [1, 5, 9], [5, 11, 4], [11, 10, 2],
         [10, 7, 6], [7, 1, 8], [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9], [4, 9, 5],
         [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    faces = [list(x) for x in f]
    for _ in range(level):
        cache: dict[tuple[int, int], int] = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                p = verts[a] + verts[b]
                verts.append(p / np.linalg.norm(p))
                cache[key] = len(verts) - 1
            return cache[key]
        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [[a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca]]
        faces = nf
    xyz = np.array(verts) * radius
    tri = np.array(faces)
    p = xyz[tri]
    nrm = np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0])
    flip = (nrm * p.mean(axis=1)).sum(axis=1) < 0
    tri[flip] = tri[flip][:, [0, 2, 1]]
    return Mesh(xyz, tri, "sphere")


@dataclass
class ElementType:
    """One distinct array element: scatterer mesh and its equivalent surface."""

    scatterer: Mesh
    equiv: Mesh
    name: str = ""


@dataclass
class ArrayLayout:
    """Elements on a square lattice: element e has type types[e] and centre offsets[e]."""

    types: list
    type_of: np.ndarray
    offsets: np.ndarray
    nx: int = 0
    ny: int = 0
    pitch: float = 0.5
    extra: dict = field(default_factory=dict)

    @property
    def n_elem(self) -> int:
        return len(self.type_of)


def loop_element(outer: float = 0.4, config_index: int = 0, stream: int = 1,
                 box=(0.45, 0.45, 0.1), box_div=(6, 6, 1)) -> ElementType:
    m = square_loop_mesh(outer=outer, gen=rng(config_index, stream))
    b = box_mesh(*box, *box_div)
    return ElementType(m, b, f"loop{outer:g}")


def loop_array(nx: int, ny: int, pitch: float = 0.5, outers=(0.4,), config_index: int = 0) -> ArrayLayout:
    """nx x ny array of loop elements; with several outer sizes, types are drawn
    uniformly per cell from a seeded stream."""
    types = [loop_element(o, config_index, 1 + i) for i, o in enumerate(outers)]
    if len(types) == 1:
        type_of = np.zeros(nx * ny, dtype=np.int32)
    else:
        type_of = rng(config_index, 100).integers(0, len(types), size=nx * ny).astype(np.int32)
    offs = np.zeros((nx * ny, 3))
    e = 0
    for j in range(ny):
        for i in range(nx):
            offs[e] = (pitch * i, pitch * j, 0.0)
            e += 1
    return ArrayLayout(types, type_of, offs, nx, ny, pitch)


def fed_loop_mesh(outer: float = 0.4, width: float = 0.04, n_per_side: int = 22):
    """Structured mesh of the square loop for a driven element: three square rings
    (outer edge, middle, inner edge) with the same number of nodes per side,
    joined by quads split into two triangles, so that every radial line of nodes
    is a chain of mesh edges.  The feed gap is the chain at the middle of the side
    y = -outer/2 (n_per_side even: a node at x = 0); the feed direction is +x
    (along the trace there).  Returns (mesh, gap edges as vertex pairs, direction)."""
    if n_per_side % 2:
        raise ValueError("n_per_side must be even (a node at the middle of each side)")
    rings = [_square_ring(outer - 2.0 * width * f, n_per_side) for f in (0.0, 0.5, 1.0)]
    npr = 4 * n_per_side
    pts = np.vstack(rings)
    tri = []
    for k in range(2):
        for i in range(npr):
            a, b = k * npr + i, k * npr + (i + 1) % npr
            c, d = (k + 1) * npr + i, (k + 1) * npr + (i + 1) % npr
            if (i // (n_per_side // 2)) % 2 == 0:
                tri += [[a, b, d], [a, d, c]]
            else:
                tri += [[a, b, c], [b, d, c]]
    tri = np.array(tri, dtype=np.int32)
    p = pts[tri]
    cr = (p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) - (p[:, 1, 1] - p[:, 0, 1]) * (p[:, 2, 0] - p[:, 0, 0])
    flip = cr < 0
    tri[flip] = tri[flip][:, [0, 2, 1]]
    xyz = np.zeros((len(pts), 3))
    xyz[:, :2] = pts
    m = Mesh(xyz, tri, "fed_loop")
    i0 = n_per_side // 2   # node at x = 0 on the side y = -outer/2
    gap = [(i0, npr + i0), (npr + i0, 2 * npr + i0)]
    return m, gap, (1.0, 0.0, 0.0)


def rwg_index(mesh: Mesh, pairs) -> np.ndarray:
    """Index of the RWG function on each interior edge (vertex pair), in the
    library's numbering: interior edges in lexicographic (min, max) order."""
    cnt: dict = {}
    for t in mesh.tri:
        for i in range(3):
            a, b = int(t[(i + 1) % 3]), int(t[(i + 2) % 3])
            k = (min(a, b), max(a, b))
            cnt[k] = cnt.get(k, 0) + 1
    interior = sorted(k for k, c in cnt.items() if c == 2)
    pos = {k: i for i, k in enumerate(interior)}
    return np.array([pos[(min(a, b), max(a, b))] for a, b in pairs], dtype=np.int64)


def fed_loop_element(outer: float = 0.4, box=(0.45, 0.45, 0.1), box_div=(6, 6, 1)):
    """Driven loop element: (ElementType, gap RWG indices, feed direction)."""
    m, gap, d = fed_loop_mesh(outer)
    return ElementType(m, box_mesh(*box, *box_div), "fed_loop%g" % outer), rwg_index(m, gap), d


def fed_loop_array(nx: int, ny: int, pitch: float = 0.5) -> ArrayLayout:
    """nx x ny array of the driven loop; layout.extra holds the feed (gap, direction)."""
    et, gap, d = fed_loop_element()
    offs = np.array([(pitch * i, pitch * j, 0.0) for j in range(ny) for i in range(nx)], dtype=np.float64)
    return ArrayLayout([et], np.zeros(nx * ny, dtype=np.int32), offs, nx, ny, pitch,
                       extra={"gap": gap, "direction": d})


def ground_plane_array(layout: ArrayLayout, z_ground: float) -> ArrayLayout:
    """The layout plus the image of every element in the PEC plane z = z_ground
    (image theory).  The loop elements are planar at z = 0 of their own frame, so
    an image element has the same type at the mirrored offset (x, y, 2 z_g - z);
    images follow the originals (elements n .. 2n - 1)."""
    off = np.array(layout.offsets, dtype=np.float64, copy=True)
    img = off.copy()
    img[:, 2] = 2.0 * z_ground - img[:, 2]
    extra = dict(layout.extra)
    extra["z_ground"] = z_ground
    extra["n_original"] = layout.n_elem
    return ArrayLayout(layout.types, np.concatenate([layout.type_of, layout.type_of]), np.vstack([off, img]),
                       layout.nx, layout.ny, layout.pitch, extra=extra)


def meander_mesh(extent: float = 0.28, width: float = 0.01, gap: float = 0.005, dx: float = 0.005) -> Mesh:
    """Serpentine strip at z = 0 inside a square of side `extent` (centred): runs
    along x of trace width `width`, separated by `gap` (the smallest feature),
    joined at alternating ends by connectors of height `gap`.  Structured mesh:
    every run is a row of dx x width quads, every connector one dx x gap quad
    sharing its edges with the runs' end cells; each quad is split into two
    triangles (normal +z)."""
    pitch = width + gap
    n_runs = int(np.floor((extent + gap) / pitch + 1e-9))
    nx = int(round(extent / dx))
    x = -extent / 2 + dx * np.arange(nx + 1)
    y0 = -(n_runs * pitch - gap) / 2
    xyz, tri = [], []
    rows = []   # per run: (bottom node ids, top node ids)
    for k in range(n_runs):
        yb = y0 + k * pitch
        bot = [len(xyz) + i for i in range(nx + 1)]
        xyz += [[xi, yb, 0.0] for xi in x]
        top = [len(xyz) + i for i in range(nx + 1)]
        xyz += [[xi, yb + width, 0.0] for xi in x]
        rows.append((bot, top))
        for i in range(nx):
            a, b, c, d = bot[i], bot[i + 1], top[i + 1], top[i]
            tri += [[a, b, c], [a, c, d]]
    for k in range(n_runs - 1):
        i = nx - 1 if k % 2 == 0 else 0          # right end after even runs, left end after odd ones
        a, b = rows[k][1][i], rows[k][1][i + 1]   # top edge of run k
        c, d = rows[k + 1][0][i + 1], rows[k + 1][0][i]   # bottom edge of run k + 1
        tri += [[a, b, c], [a, c, d]]
    return Mesh(np.array(xyz), np.array(tri, dtype=np.int64), "meander")


# Reduced multiscale element for oracle parity (the oracle's dense fills of the
# full 2547-RWG element take minutes): the same loop, a coarser meander (7 runs
# of 0.02-wide trace, 0.01 gaps: 535 RWG in all), the 6 x 6 x 1 box.
MEANDER_REDUCED = dict(extent=0.2, width=0.02, gap=0.01, dx=0.02)
MEANDER_REDUCED_BOX = (6, 6, 1)


def merge_meshes(a: Mesh, b: Mesh, name: str = "") -> Mesh:
    return Mesh(np.vstack([a.xyz, b.xyz]), np.vstack([a.tri, b.tri + len(a.xyz)]), name)


def multiscale_element(config_index: int = 3, stream: int = 1, meander=None,
                       box=(0.45, 0.45, 0.1), box_div=(8, 8, 2)) -> ElementType:
    """Multiscale element: the 0.4-wavelength square loop with a meandered trace
    inside it (0.005-wavelength gaps and cells), in the 0.45 x 0.45 x 0.1 box meshed
    8 x 8 x 2 (576 RWG).  `meander` overrides the meander_mesh arguments."""
    ring = square_loop_mesh(outer=0.4, gen=rng(config_index, stream))
    mz = meander_mesh(**(meander or {}))
    return ElementType(merge_meshes(ring, mz, "loop_meander"), box_mesh(*box, *box_div), "loop_meander")


def multiscale_array(nx: int, ny: int, pitch: float = 0.5, config_index: int = 3, meander=None,
                     box_div=(8, 8, 2)) -> ArrayLayout:
    """nx x ny array of identical multiscale elements."""
    et = multiscale_element(config_index, 1, meander, box_div=box_div)
    offs = np.zeros((nx * ny, 3))
    e = 0
    for j in range(ny):
        for i in range(nx):
            offs[e] = (pitch * i, pitch * j, 0.0)
            e += 1
    return ArrayLayout([et], np.zeros(nx * ny, dtype=np.int32), offs, nx, ny, pitch)


def planewave_grid(n_theta: int = 8, n_phi: int = 8, theta_max_deg: float = 60.0, phi_max_deg: float = 90.0):
    """(theta, phi, pol) for an n_theta x n_phi incidence grid; pol alternates
    theta-hat (0) / phi-hat (1) with the parity of (i + j)."""
    th = np.deg2rad(np.linspace(0.0, theta_max_deg, n_theta))
    ph = np.deg2rad(np.linspace(0.0, phi_max_deg, n_phi))
    T, P, POL = [], [], []
    for i in range(n_theta):
        for j in range(n_phi):
            T.append(th[i]); P.append(ph[j]); POL.append((i + j) % 2)
    return np.array(T), np.array(P), np.array(POL, dtype=np.int32)


def random_cvec(n: int, config_index: int = 0, stream: int = 7, nrhs: int = 1) -> np.ndarray:
    """Seeded complex128 test vector(s), shape (n,) or (n, nrhs)."""
    g = rng(config_index, stream)
    shape = (n,) if nrhs == 1 else (n, nrhs)
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


# Default AIM grid phase for the loop arrays: grid nodes at phase + h*Z^3.
# Chosen so that no equivalent-box basis centroid falls on a rounding tie.
DEFAULT_GRID_PHASE = (0.0137, 0.0291, 0.0913)
