"""RWG and dual (Buffa-Christiansen) basis functions (oracle).

Sec. II-A: the current on S_m is expanded in RWG functions, eq. (J_expand);
n x H^ on the equivalent surface in RWG functions, eq. (Hhat_expand), with n
the normal pointing INTO the closed surface; n x E^ in dual RWG functions,
eq. (Ehat_expand), built on the barycentric refinement of the mesh.

Conventions (the paper leaves them open):

* RWG n lives on interior edge (a, b), a < b; edges are numbered in
  lexicographic order of (a, b).  T+ is the adjacent triangle with the smaller
  index, T- the other.  On T+: f = l/(2 A+) (r - p+); on T-: f = l/(2 A-) (p- - r),
  p+- the free vertices.  div f = +l/A+ on T+, -l/A- on T-.
* Barycentric refinement: primal triangle t = (p0, p1, p2) splits into six
  triangles of area A/6; refined triangle 6t+2i = (p_i, m_{i,i+1}, g) and
  6t+2i+1 = (p_i, g, m_{i+2,i}) (m = edge midpoint, g = centroid); both keep
  the primal orientation.
* Dual function of edge e (closed, outward-oriented surfaces only): a
  divergence-conforming RT0 field on the refined mesh, supported on the dual
  cells (the 2K refined triangles around a primal vertex with K triangles) of
  the two end points of e.  It carries a total flux l_e across the dual edge
  g+ -> m_e -> g- (half through each refined edge), from the cell of v_s to
  the cell of v_t, where v_s -> v_t is the direction in which e is traversed
  in T+.  Each refined triangle of the source cell emits l_e/(2 K_s), each of
  the sink cell absorbs l_e/(2 K_t), the flux being passed round each cell
  symmetrically (no circulation), which is the Buffa-Christiansen
  construction (Andriulli et al. 2008, cited with eq. (Ehat_expand)).
  On a refined triangle with vertices q_0..q_2 and outward fluxes Phi_i across
  the edge opposite q_i the field is sum_i Phi_i/(2A) (r - q_i).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class RWG:
    xyz: np.ndarray          # (nv, 3)
    tri: np.ndarray          # (nt, 3)
    area: np.ndarray         # (nt,)
    normal: np.ndarray       # (nt, 3) unit normal from the vertex order
    edges: np.ndarray        # (n, 2) vertex pairs of interior edges (RWG order)
    tplus: np.ndarray        # (n,)
    tminus: np.ndarray       # (n,)
    vplus: np.ndarray        # (n,) free vertex of T+
    vminus: np.ndarray       # (n,) free vertex of T-
    length: np.ndarray       # (n,)
    tri_rwg: np.ndarray      # (nt, 3) RWG index of the edge opposite local vertex i, -1 if none
    tri_sign: np.ndarray     # (nt, 3) +1 if t is T+ of that RWG, -1 if T-, 0 if none
    all_edges: np.ndarray    # (ne, 2) every edge (boundary edges included), sorted
    tri_alledge: np.ndarray  # (nt, 3) index into all_edges of the edge opposite local vertex i

    @property
    def n(self) -> int:
        return len(self.length)

    def centroid(self) -> np.ndarray:
        """Area-weighted centroid of each RWG support (T+ u T-)."""
        gp = self.xyz[self.tri[self.tplus]].mean(axis=1)
        gm = self.xyz[self.tri[self.tminus]].mean(axis=1)
        ap = self.area[self.tplus][:, None]
        am = self.area[self.tminus][:, None]
        return (ap * gp + am * gm) / (ap + am)


def build_rwg(xyz: np.ndarray, tri: np.ndarray) -> RWG:
    """RWG functions on every interior edge (eq. (J_expand), (Hhat_expand))."""
    xyz = np.asarray(xyz, dtype=np.float64)
    tri = np.asarray(tri, dtype=np.int64)
    nt = len(tri)
    p = xyz[tri]
    cr = np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0])
    nrm = np.linalg.norm(cr, axis=1)
    area = 0.5 * nrm
    normal = cr / nrm[:, None]
    keys = {}
    for t in range(nt):
        for i in range(3):
            a, b = tri[t, (i + 1) % 3], tri[t, (i + 2) % 3]
            k = (min(a, b), max(a, b))
            keys.setdefault(k, []).append((t, i))
    all_keys = sorted(keys)
    all_index = {k: j for j, k in enumerate(all_keys)}
    tri_alledge = np.zeros((nt, 3), dtype=np.int64)
    for k, lst in keys.items():
        if len(lst) > 2:
            raise ValueError("non-manifold edge %r" % (k,))
        for t, i in lst:
            tri_alledge[t, i] = all_index[k]
    interior = [k for k in all_keys if len(keys[k]) == 2]
    n = len(interior)
    edges = np.array(interior, dtype=np.int64).reshape(-1, 2)
    tplus = np.zeros(n, dtype=np.int64)
    tminus = np.zeros(n, dtype=np.int64)
    vplus = np.zeros(n, dtype=np.int64)
    vminus = np.zeros(n, dtype=np.int64)
    tri_rwg = -np.ones((nt, 3), dtype=np.int64)
    tri_sign = np.zeros((nt, 3), dtype=np.int64)
    for e, k in enumerate(interior):
        (t1, i1), (t2, i2) = sorted(keys[k])
        tplus[e], tminus[e] = t1, t2
        vplus[e], vminus[e] = tri[t1, i1], tri[t2, i2]
        tri_rwg[t1, i1] = e
        tri_sign[t1, i1] = 1
        tri_rwg[t2, i2] = e
        tri_sign[t2, i2] = -1
    length = np.linalg.norm(xyz[edges[:, 1]] - xyz[edges[:, 0]], axis=1) if n else np.zeros(0)
    return RWG(xyz, tri, area, normal, edges, tplus, tminus, vplus, vminus, length,
               tri_rwg, tri_sign, np.array(all_keys, dtype=np.int64).reshape(-1, 2), tri_alledge)


def rwg_eval(rwg: RWG, t: int, i: int, r: np.ndarray) -> np.ndarray:
    """Value at points r (.., 3) of the RWG on edge opposite local vertex i of triangle t."""
    e = rwg.tri_rwg[t, i]
    s = rwg.tri_sign[t, i]
    return s * rwg.length[e] / (2.0 * rwg.area[t]) * (r - rwg.xyz[rwg.tri[t, i]])


@dataclass
class Refined:
    xyz: np.ndarray     # refined vertices: primal vertices, then edge midpoints, then centroids
    tri: np.ndarray     # (6 nt, 3)
    area: np.ndarray    # (6 nt,)
    parent: np.ndarray  # (6 nt,) primal triangle


def barycentric_refinement(rwg: RWG) -> Refined:
    xyz, tri = rwg.xyz, rwg.tri
    nv, nt, ne = len(xyz), len(tri), len(rwg.all_edges)
    mids = 0.5 * (xyz[rwg.all_edges[:, 0]] + xyz[rwg.all_edges[:, 1]])
    cents = xyz[tri].mean(axis=1)
    rx = np.vstack([xyz, mids, cents])
    rt = np.zeros((6 * nt, 3), dtype=np.int64)
    for t in range(nt):
        g = nv + ne + t
        for i in range(3):
            j, k = (i + 1) % 3, (i + 2) % 3
            m_ij = nv + rwg.tri_alledge[t, k]   # edge (i, j) is opposite local vertex k
            m_ki = nv + rwg.tri_alledge[t, j]   # edge (k, i) is opposite local vertex j
            rt[6 * t + 2 * i] = (tri[t, i], m_ij, g)
            rt[6 * t + 2 * i + 1] = (tri[t, i], g, m_ki)
    p = rx[rt]
    area = 0.5 * np.linalg.norm(np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), axis=1)
    return Refined(rx, rt, area, np.repeat(np.arange(nt), 6))


@dataclass
class BCDual:
    """Dual functions as a list of (function, refined triangle, outward fluxes)."""

    refined: Refined
    fn: np.ndarray      # (E,) dual function index
    rtri: np.ndarray    # (E,) refined triangle
    flux: np.ndarray    # (E, 3) outward flux across the edge opposite refined vertex i
    n: int


def _cycle_at_vertex(rwg: RWG, v: int, vert_tris) -> list[int]:
    """Refined triangles around primal vertex v in CCW order (about the outward normal)."""
    tri = rwg.tri
    tl = vert_tris[v]
    nxt = {}
    for t in tl:
        i = int(np.where(tri[t] == v)[0][0])
        nxt[int(tri[t, (i + 1) % 3])] = (t, i)
    t0 = tl[0]
    order = []
    t = t0
    for _ in range(len(tl)):
        i = int(np.where(tri[t] == v)[0][0])
        order += [6 * t + 2 * i, 6 * t + 2 * i + 1]
        prev_v = int(tri[t, (i + 2) % 3])
        t = nxt[prev_v][0]
    if t != t0 or len(order) != 2 * len(tl):
        raise ValueError("vertex %d is not an interior manifold vertex" % v)
    return order


def build_bc(rwg: RWG) -> BCDual:
    """Dual (Buffa-Christiansen) functions for every RWG of a closed surface (eq. (Ehat_expand))."""
    ref = barycentric_refinement(rwg)
    tri = rwg.tri
    vert_tris = [[] for _ in range(len(rwg.xyz))]
    for t in range(len(tri)):
        for i in range(3):
            vert_tris[tri[t, i]].append(t)
    cycles = {}
    fn, rt, fl = [], [], []

    def opp_local(rtri_a, rtri_b):
        sa = set(ref.tri[rtri_a])
        shared = sa & set(ref.tri[rtri_b])
        for i in range(3):
            if ref.tri[rtri_a, i] not in shared:
                return i
        raise RuntimeError

    for e in range(rwg.n):
        tp, tm = rwg.tplus[e], rwg.tminus[e]
        a, b = rwg.edges[e]
        ip = [i for i in range(3) if {tri[tp, i], tri[tp, (i + 1) % 3]} == {a, b}][0]
        vs, vt = int(tri[tp, ip]), int(tri[tp, (ip + 1) % 3])
        le = rwg.length[e]
        for v in (vs, vt):
            if v not in cycles:
                cycles[v] = _cycle_at_vertex(rwg, v, vert_tris)
        # sink cell around vt: start at T+'s (vt, g+, m_e), walk clockwise to T-'s (vt, m_e, g-)
        it = (ip + 1) % 3
        cyc = cycles[vt]
        K = len(cyc) // 2
        start = cyc.index(6 * tp + 2 * it + 1)
        seq = [cyc[(start - j) % len(cyc)] for j in range(2 * K)]
        im = int(np.where(tri[tm] == vt)[0][0])
        if seq[-1] != 6 * tm + 2 * im:
            raise RuntimeError("dual cell walk mismatch (sink)")
        flux = {r: np.zeros(3) for r in seq}
        flux[seq[0]][0] -= le / 2.0
        flux[seq[-1]][0] -= le / 2.0
        for j in range(2 * K - 1):
            F = le * (K - 1 - j) / (2.0 * K)
            flux[seq[j]][opp_local(seq[j], seq[j + 1])] += F
            flux[seq[j + 1]][opp_local(seq[j + 1], seq[j])] -= F
        for r in seq:
            fn.append(e); rt.append(r); fl.append(flux[r])
        # source cell around vs: start at T+'s (vs, m_e, g+), walk counter-clockwise to T-'s (vs, g-, m_e)
        cyc = cycles[vs]
        K = len(cyc) // 2
        start = cyc.index(6 * tp + 2 * ip)
        seq = [cyc[(start + j) % len(cyc)] for j in range(2 * K)]
        im = int(np.where(tri[tm] == vs)[0][0])
        if seq[-1] != 6 * tm + 2 * im + 1:
            raise RuntimeError("dual cell walk mismatch (source)")
        flux = {r: np.zeros(3) for r in seq}
        flux[seq[0]][0] += le / 2.0
        flux[seq[-1]][0] += le / 2.0
        for j in range(2 * K - 1):
            F = le * (K - 1 - j) / (2.0 * K)
            flux[seq[j]][opp_local(seq[j], seq[j + 1])] -= F
            flux[seq[j + 1]][opp_local(seq[j + 1], seq[j])] += F
        for r in seq:
            fn.append(e); rt.append(r); fl.append(flux[r])
    return BCDual(ref, np.array(fn), np.array(rt), np.array(fl), rwg.n)


def bc_eval_coeffs(bc: BCDual):
    """Per support entry: alpha, beta such that the dual field is alpha*r - beta on that refined triangle."""
    ref = bc.refined
    A = ref.area[bc.rtri]
    q = ref.xyz[ref.tri[bc.rtri]]                       # (E, 3, 3)
    alpha = bc.flux.sum(axis=1) / (2.0 * A)
    beta = np.einsum("ei,eij->ej", bc.flux, q) / (2.0 * A)[:, None]
    return alpha, beta
