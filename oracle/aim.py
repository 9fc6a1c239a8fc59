"""Adaptive integral method for G^(E^,J^) on an array (oracle), Sec. V.

G^(E^,J^) ~ G_NF + sum_psi I_psi H_psi P_psi, psi in {A_x, A_y, A_z, phi}:
  (i)   projection: Y1_psi = P_psi Y, grid currents and charges on a stencil of
        (N_O + 1)^3 nodes per basis (interpolation polynomials of order N_O);
  (ii)  convolution: Y2_psi = H_psi Y1_psi, H[u, u'] = G(r_u - r_u') applied by
        zero-padded FFT (G is position invariant);
  (iii) interpolation: Y3_psi = I_psi Y2_psi, summed over psi;
  near field: G_NF = exact entries minus the grid contribution, for pairs whose
        stencils are within N_NF cells.

Readings of points the paper leaves open:
* grid nodes r_u = phase + h u (u integer 3-vector);
* anchor of basis n: nearest node (round half up) to the area-weighted
  centroid of its support for odd N_O + 1; floor for even N_O + 1; a centroid
  within 1e-9 of a rounding tie is rejected;
* stencil = anchor + {-N_O/2 .. N_O/2}^3 (odd N_O + 1) or
  {-(N_O-1)/2 .. (N_O+1)/2}^3 (even);
* W_u = tensor-product Lagrange polynomial of the stencil, P weights
  Pi_{n,psi}[u] = int f_{n,psi} W_u dS (psi = x, y, z) and
  Pi_{n,phi}[u] = int div f_n W_u dS, integrated exactly (degree 3 N_O + 1);
  this is the moment-matching projection, and I = P^T (Galerkin testing);
* the four H_psi are the same free-space kernel; the constants
  c_A = -j w mu0 and c_phi = +j w mu0/k^2 (from Lmat) multiply the psi terms;
* H[0] = G(0) := 0;
* near pairs: Chebyshev distance between anchors <= N_NF grid cells;
  G_NF[m, n] = G^(E^,J^)[m, n] - (grid contribution)[m, n];
* linear convolution via padding each axis to 2 N.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.fft as sfft
import scipy.sparse as sp

from .basis import RWG
from .macromodel import coupling_block, translated_rwg
from .operators import ETA0
from .potentials import green
from .quadrature import collapsed_gauss, points


@dataclass
class AIMParams:
    h: float = 0.1
    order: int = 2
    n_nf: int = 3
    phase: tuple = (0.0, 0.0, 0.0)


def stencil_offsets_1d(order: int) -> np.ndarray:
    n = order + 1
    lo = -(order // 2) if n % 2 == 1 else -((n // 2) - 1)
    return np.arange(lo, lo + n)


def stencil_offsets(order: int) -> np.ndarray:
    """(S, 3) integer offsets, x fastest: s = (iz * n + iy) * n + ix."""
    o = stencil_offsets_1d(order)
    n = len(o)
    out = np.zeros((n ** 3, 3), dtype=np.int64)
    for iz in range(n):
        for iy in range(n):
            for ix in range(n):
                out[(iz * n + iy) * n + ix] = (o[ix], o[iy], o[iz])
    return out


def anchors(centroids: np.ndarray, p: AIMParams) -> np.ndarray:
    s = (centroids - np.asarray(p.phase)[None, :]) / p.h
    if (p.order + 1) % 2 == 1:
        fr = s - np.floor(s)
        if np.any(np.abs(fr - 0.5) < 1e-9):
            raise ValueError("basis centroid on a rounding tie of the AIM grid; shift the grid phase")
        return np.floor(s + 0.5).astype(np.int64)
    fr = s - np.floor(s)
    if np.any(np.minimum(fr, 1.0 - fr) < 1e-9):
        raise ValueError("basis centroid on a grid plane; shift the grid phase")
    return np.floor(s).astype(np.int64)


def lagrange(sv: np.ndarray, nodes: np.ndarray) -> np.ndarray:
    """1D Lagrange basis of `nodes` at points sv -> (len(sv), len(nodes))."""
    out = np.ones((len(sv), len(nodes)))
    for a in range(len(nodes)):
        for b in range(len(nodes)):
            if a != b:
                out[:, a] *= (sv - nodes[b]) / (nodes[a] - nodes[b])
    return out


def projection_weights(rwg: RWG, anc: np.ndarray, p: AIMParams) -> np.ndarray:
    """Pi (N, S, 4): moment-matching projection of each RWG onto its stencil (step (i))."""
    bq, wq = collapsed_gauss(3 * p.order + 1)
    o1 = stencil_offsets_1d(p.order).astype(np.float64)
    n1 = len(o1)
    S = n1 ** 3
    Pi = np.zeros((rwg.n, S, 4))
    ph = np.asarray(p.phase)
    for side, tt, vv, sg in ((0, rwg.tplus, rwg.vplus, 1.0), (1, rwg.tminus, rwg.vminus, -1.0)):
        T = rwg.xyz[rwg.tri[tt]]                                  # (N,3,3)
        q = points(T, bq)                                          # (N,Q,3)
        A = rwg.area[tt]
        f = sg * (rwg.length / (2.0 * A))[:, None, None] * (q - rwg.xyz[vv][:, None, :])   # (N,Q,3)
        div = sg * rwg.length / A                                  # (N,)
        loc = (q - ph[None, None, :]) / p.h - anc[:, None, :]      # stencil-local coordinates
        Lx = lagrange(loc[..., 0].ravel(), o1).reshape(rwg.n, -1, n1)
        Ly = lagrange(loc[..., 1].ravel(), o1).reshape(rwg.n, -1, n1)
        Lz = lagrange(loc[..., 2].ravel(), o1).reshape(rwg.n, -1, n1)
        W = np.einsum("nqc,nqb,nqa->nqcba", Lz, Ly, Lx).reshape(rwg.n, -1, S)  # s = (iz*n+iy)*n+ix
        wA = wq[None, :] * A[:, None]                              # (N,Q)
        Pi[:, :, 0:3] += np.einsum("nq,nqs,nqx->nsx", wA, W, f)
        Pi[:, :, 3] += np.einsum("nq,nqs->ns", wA, W) * div[:, None]
    return Pi


def grid_green(delta: np.ndarray, h: float, k: float) -> np.ndarray:
    """H for integer offsets delta (..., 3): G(h |delta|), 0 at delta = 0."""
    R = h * np.linalg.norm(delta.astype(np.float64), axis=-1)
    out = np.zeros(R.shape, dtype=np.complex128)
    nz = R > 0
    out[nz] = green(R[nz], k)
    return out


def fft_kernel(N, h: float, k: float) -> np.ndarray:
    """Circulant embedding of H on a (2Nx, 2Ny, 2Nz) grid, transformed."""
    P = [2 * n for n in N]
    idx = [np.where(np.arange(P[a]) < N[a], np.arange(P[a]), np.arange(P[a]) - P[a]) for a in range(3)]
    D = np.stack(np.meshgrid(*idx, indexing="ij"), axis=-1)
    Kp = grid_green(D, h, k)
    for a in range(3):   # offset +-N is never used by a linear convolution of length N
        sl = [slice(None)] * 3
        sl[a] = N[a]
        Kp[tuple(sl)] = 0.0
    return sfft.fftn(Kp, workers=-1)


def convolve(Q: np.ndarray, Khat: np.ndarray) -> np.ndarray:
    """Phi[u] = sum_u' H[u - u'] Q[u'] for grids Q (..., Nx, Ny, Nz) (step (ii))."""
    N = Q.shape[-3:]
    P = Khat.shape
    Qp = np.zeros(Q.shape[:-3] + P, dtype=np.complex128)
    Qp[..., :N[0], :N[1], :N[2]] = Q
    # library FFTs (scipy.fft, on all host cores); the same transforms as numpy's
    out = sfft.ifftn(sfft.fftn(Qp, axes=(-3, -2, -1), workers=-1) * Khat, axes=(-3, -2, -1), workers=-1)
    return out[..., :N[0], :N[1], :N[2]]


def brute_convolve(Q: np.ndarray, h: float, k: float) -> np.ndarray:
    """Direct sum of step (ii) (pins only; small grids)."""
    N = Q.shape[-3:]
    u = np.stack(np.meshgrid(*[np.arange(n) for n in N], indexing="ij"), axis=-1).reshape(-1, 3)
    H = grid_green(u[:, None, :] - u[None, :, :], h, k)
    return (Q.reshape(Q.shape[:-3] + (-1,)) @ H.T).reshape(Q.shape)


class BlockCache:
    """G^(E^,J^) blocks between element pairs, computed once per (type, type,
    relative offset): the blocks of identical elements are reused (Sec. III) and
    the free-space Green's function depends only on r - r' (Sec. V)."""

    def __init__(self, models, k: float):
        self.models = models
        self.k = k
        self.cache: dict = {}

    def get(self, ta: int, tb: int, rel: np.ndarray) -> np.ndarray:
        key = (ta, tb) + tuple(np.round(np.asarray(rel, dtype=np.float64), 9))
        if key not in self.cache:
            ra = self.models[ta].rwg_e
            rb = translated_rwg(self.models[tb].rwg_e, rel)
            self.cache[key] = coupling_block(ra, rb, self.k)
        return self.cache[key]


@dataclass
class AIMArray:
    """The AIM-accelerated exterior operator y = D x - G (T A^-1 B x) (eq. (MV_product1))."""

    models: list
    type_of: np.ndarray
    offsets: np.ndarray
    params: AIMParams
    k: float
    blocks: BlockCache = None
    rows_only: bool = False
    # filled by setup
    off: np.ndarray = None
    elem_of: np.ndarray = None
    anc: np.ndarray = None
    lo: np.ndarray = None
    N: tuple = None
    Pi: np.ndarray = None
    nodes: np.ndarray = None
    Khat: np.ndarray = None
    GNF: sp.csr_matrix = None
    c_A: complex = 0
    c_phi: complex = 0

    def __post_init__(self):
        k = self.k
        self.c_A = -1j * k * ETA0
        self.c_phi = 1j * ETA0 / k
        if self.blocks is None:
            self.blocks = BlockCache(self.models, k)
        sizes = np.array([self.models[t].rwg_e.n for t in self.type_of])
        self.off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        self.elem_of = np.repeat(np.arange(len(self.type_of)), sizes)
        anc, Pi = [], []
        for e, t in enumerate(self.type_of):
            r = translated_rwg(self.models[t].rwg_e, self.offsets[e])
            a = anchors(r.centroid(), self.params)
            anc.append(a)
            Pi.append(projection_weights(r, a, self.params))
        anc = np.vstack(anc)
        so = stencil_offsets(self.params.order)
        self.lo = anc.min(axis=0) + so.min(axis=0)
        hi = anc.max(axis=0) + so.max(axis=0)
        self.N = tuple(int(x) for x in (hi - self.lo + 1))
        self.anc = anc - self.lo
        self.Pi = np.concatenate(Pi, axis=0)
        g = self.anc[:, None, :] + so[None, :, :]                 # (Nb, S, 3)
        Nx, Ny, Nz = self.N
        self.nodes = (g[..., 0] * Ny + g[..., 1]) * Nz + g[..., 2]   # flat index in (Nx,Ny,Nz) C order
        self.Khat = fft_kernel(self.N, self.params.h, k)
        if not self.rows_only:
            self.GNF = self.near_field_rows(np.arange(self.off[-1]))

    @property
    def n(self) -> int:
        return int(self.off[-1])

    # ---- near field -------------------------------------------------------
    def near_pairs(self, rows: np.ndarray):
        """For each row m: columns n with Chebyshev(anchor_m - anchor_n) <= N_NF."""
        nnf = self.params.n_nf
        buckets: dict = {}
        for n, a in enumerate(map(tuple, self.anc)):
            buckets.setdefault(a, []).append(n)
        out = []
        for m in rows:
            a = self.anc[m]
            cols = []
            for dx in range(-nnf, nnf + 1):
                for dy in range(-nnf, nnf + 1):
                    for dz in range(-nnf, nnf + 1):
                        cols += buckets.get((a[0] + dx, a[1] + dy, a[2] + dz), [])
            out.append(np.sort(np.array(cols, dtype=np.int64)))
        return out

    def exact_entries(self, m: int, cols: np.ndarray) -> np.ndarray:
        ea = self.elem_of[m]
        out = np.zeros(len(cols), dtype=np.complex128)
        eb = self.elem_of[cols]
        for b in np.unique(eb):
            sel = eb == b
            blk = self.blocks.get(int(self.type_of[ea]), int(self.type_of[b]), self.offsets[b] - self.offsets[ea])
            out[sel] = blk[m - self.off[ea], cols[sel] - self.off[b]]
        return out

    def grid_entries(self, m: int, cols: np.ndarray) -> np.ndarray:
        """(I H P)[m, n] for the given columns."""
        so = stencil_offsets(self.params.order)
        da = self.anc[m][None, :] - self.anc[cols]                 # (c,3)
        dd = da[:, None, None, :] + so[None, :, None, :] - so[None, None, :, :]   # (c,S,S,3)
        H = grid_green(dd, self.params.h, self.k)
        Pm = self.Pi[m]                                            # (S,4)
        Pn = self.Pi[cols]                                         # (c,S,4)
        v = np.einsum("sx,cst,ctx->cx", Pm, H, Pn)
        return self.c_A * v[:, :3].sum(axis=1) + self.c_phi * v[:, 3]

    def near_field_rows(self, rows: np.ndarray) -> sp.csr_matrix:
        """Rows of G_NF = exact - grid contribution over the near pairs."""
        rows = np.asarray(rows, dtype=np.int64)
        pairs = self.near_pairs(rows)
        cnt = np.array([len(c) for c in pairs], dtype=np.int64)
        mi = np.repeat(rows, cnt)
        ni = np.concatenate(pairs) if len(pairs) else np.zeros(0, dtype=np.int64)
        val = np.zeros(len(mi), dtype=np.complex128)
        # exact entries, one element-pair block at a time
        ea, eb = self.elem_of[mi], self.elem_of[ni]
        key = ea * len(self.type_of) + eb
        for kk in np.unique(key):
            sel = key == kk
            a, b = divmod(int(kk), len(self.type_of))
            blk = self.blocks.get(int(self.type_of[a]), int(self.type_of[b]), self.offsets[b] - self.offsets[a])
            val[sel] = blk[mi[sel] - self.off[a], ni[sel] - self.off[b]]
        # grid contribution, grouped by anchor offset
        so = stencil_offsets(self.params.order)
        da = self.anc[mi] - self.anc[ni]
        w = 2 * self.params.n_nf + 1
        dkey = ((da[:, 0] + self.params.n_nf) * w + da[:, 1] + self.params.n_nf) * w + da[:, 2] + self.params.n_nf
        for kk in np.unique(dkey):
            sel = np.where(dkey == kk)[0]
            d = da[sel[0]]
            H = grid_green(d[None, None, :] + so[:, None, :] - so[None, :, :], self.params.h, self.k)
            v = np.einsum("gsx,st,gtx->gx", self.Pi[mi[sel]], H, self.Pi[ni[sel]])
            val[sel] -= self.c_A * v[:, :3].sum(axis=1) + self.c_phi * v[:, 3]
        indptr = np.concatenate([[0], np.cumsum(cnt)])
        return sp.csr_matrix((val, ni, indptr), shape=(len(rows), self.n))

    # ---- far field (steps i-iii) -----------------------------------------
    def project(self, u: np.ndarray) -> np.ndarray:
        """Step (i): Q_psi = P_psi u, grids (4, Nx, Ny, Nz) (single vector u)."""
        Q = np.zeros((4, int(np.prod(self.N))), dtype=np.complex128)
        for c in range(4):
            np.add.at(Q[c], self.nodes.ravel(), (self.Pi[:, :, c] * u[:, None]).ravel())
        return Q.reshape((4,) + self.N)

    def interpolate(self, Phi: np.ndarray, rows=None) -> np.ndarray:
        """Step (iii) with I = P^T, summed over psi with c_A, c_phi."""
        F = Phi.reshape(4, -1)
        idx = slice(None) if rows is None else rows
        nodes = self.nodes[idx]
        Pi = self.Pi[idx]
        v = np.einsum("nsc,cns->nc", Pi, F[:, nodes])
        return self.c_A * v[:, :3].sum(axis=1) + self.c_phi * v[:, 3]

    def far(self, u: np.ndarray, rows=None) -> np.ndarray:
        return self.interpolate(convolve(self.project(u), self.Khat), rows)

    def gapply(self, u: np.ndarray) -> np.ndarray:
        """G^(E^,J^) u by AIM: far field (steps i-iii) plus the precorrected near field."""
        return self.far(u) + self.GNF @ u

    # ---- full operator ----------------------------------------------------
    def macro(self, x: np.ndarray) -> np.ndarray:
        """u = T A^-1 B x, block diagonal (Sec. III)."""
        u = np.zeros_like(x)
        for e, t in enumerate(self.type_of):
            u[self.off[e]:self.off[e + 1]] = self.models[t].M @ x[self.off[e]:self.off[e + 1]]
        return u

    def dapply(self, x: np.ndarray, rows=None) -> np.ndarray:
        v = np.zeros_like(x)
        for e, t in enumerate(self.type_of):
            v[self.off[e]:self.off[e + 1]] = self.models[t].D @ x[self.off[e]:self.off[e + 1]]
        return v if rows is None else v[rows]

    def matvec(self, x: np.ndarray) -> np.ndarray:
        """y = D x - (G_FF + G_NF) T A^-1 B x for one vector x (eq. (MV_product1))."""
        u = self.macro(x)
        return self.dapply(x) - (self.far(u) + self.GNF @ u)

    def matvec_rows(self, x: np.ndarray, rows: np.ndarray) -> np.ndarray:
        """Selected rows of matvec(x), computing only those rows' near field."""
        u = self.macro(x)
        G = self.near_field_rows(rows)
        return self.dapply(x, rows) - (self.far(u, rows) + G @ u)
