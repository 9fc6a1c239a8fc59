"""Galerkin operator fills (oracle): L, K, D, excitation, far field.

Definitions (Sec. II-C, II-D, IV):
  <f, g> = int f . g dS.
  [L X](r) = (1 + grad grad . / k^2) int G X,   [K X](r) = curl int G X.
With RWG normal continuity the L form integrates by parts:
  Lmat[m, n] = int int f_m . f_n G - k^-2 int int (div f_m)(div' f_n) G.
For tangential test functions n x n x F tests as -F, so every
  jw mu0 <f_m, n x n x L f_n> = -jw mu0 Lmat[m, n],
  <f_m, -n x n x K g_n>      = <f_m, K g_n>  = Kmat[m, n].
K is evaluated as the limit from outside the closed equivalent surface (the
Stratton-Chu identity is zero outside V): on the surface itself this is the
principal value plus 1/2 <f_m, n x g_n>, n the inward normal, i.e.
Kmat_outside = Kmat_PV + D/2 with D[m, n] = <f_m, n x g_n> (Sec. IV).

Quadrature: 7-point (degree 5) rule on every test triangle; the source 1/R
part in closed form (singularity extraction), the smooth remainder G1 with
the 7-point rule on primal source triangles (L) or the 3-point rule on
refined source triangles (K).  D is exact with the 3-point rule.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .basis import RWG, BCDual, bc_eval_coeffs
from .potentials import static_integrals, g1, g1_grad_factor
from .quadrature import tri3, tri7, points

ETA0 = 376.730313668       # free-space impedance (ohm)
TWO_PI = 2.0 * np.pi


def _local_coeffs(rwg: RWG):
    """For each (triangle, local vertex): RWG index (0 if none) and sign*length (0 if none)."""
    idx = np.where(rwg.tri_rwg >= 0, rwg.tri_rwg, 0)
    coef = np.where(rwg.tri_rwg >= 0, rwg.tri_sign * rwg.length[idx], 0.0)
    return idx, coef


def efie_matrix(test: RWG, src: RWG, k: float, chunk: int = 24) -> np.ndarray:
    """Lmat[m, n] (see module doc) between two RWG sets."""
    b7, w7 = tri7()
    Tt = test.xyz[test.tri]
    Ts = src.xyz[src.tri]
    rt = points(Tt, b7)                                    # (nT, 7, 3)
    rs = points(Ts, b7)                                    # (nS, 7, 3)
    At, As = test.area, src.area
    it, ct = _local_coeffs(test)
    is_, cs = _local_coeffs(src)
    # source local functions phi'_j(r') = (r' - p'_j)/(2A')
    ps = Ts                                                # p'_j = vertex j of source triangle
    Ws = w7[None, :] * As[:, None]                         # (nS, 7)
    phis = (rs[:, :, None, :] - ps[:, None, :, :]) / (2.0 * As)[:, None, None, None]  # (nS,7,3j,3x)
    out = np.zeros((test.n, src.n), dtype=np.complex128)
    inv4pi = 1.0 / (4.0 * np.pi)
    for c0 in range(0, len(Tt), chunk):
        c1 = min(c0 + chunk, len(Tt))
        c = c1 - c0
        P = rt[c0:c1].reshape(-1, 3)
        st = static_integrals(P, Ts, need=("S0", "Sv"))
        S0 = st["S0"].reshape(c, 7, -1)                    # (c,7,nS)
        Sv = st["Sv"].reshape(c, 7, -1, 3)
        rho = st["rho"].reshape(c, 7, -1, 3)
        Wt = w7[None, :] * At[c0:c1, None]                 # (c,7)
        phit = (rt[c0:c1, :, None, :] - Tt[c0:c1, None, :, :]) / (2.0 * At[c0:c1])[:, None, None, None]  # (c,7,3i,3x)
        # static: inner vector integral for local j: (Sv + (rho - p'_j) S0)/(2A')
        Vj = (Sv[:, :, :, None, :] + (rho[:, :, :, None, :] - ps[None, None, :, :, :]) * S0[..., None, None]) \
            / (2.0 * As)[None, None, :, None, None]        # (c,7,nS,3j,3x)
        I0 = np.einsum("tq,tqix,tqsjx->tisj", Wt, phit, Vj)
        I0 -= (np.einsum("tq,tqs->ts", Wt, S0) / (k * k) / At[c0:c1, None] / As[None, :])[:, None, :, None]
        I0 *= inv4pi
        # smooth: product quadrature of G1
        R = np.linalg.norm(rt[c0:c1, :, None, None, :] - rs[None, None, :, :, :], axis=-1)  # (c,7,nS,7)
        G = g1(R, k)
        WG = G * Wt[:, :, None, None] * Ws[None, None, :, :]
        I1 = np.einsum("tqsr,tqix,srjx->tisj", WG, phit, phis, optimize=True)
        I1 -= (WG.sum(axis=(1, 3)) / (k * k) / At[c0:c1, None] / As[None, :])[:, None, :, None]
        I = (I0 + I1) * ct[c0:c1, :, None, None] * cs[None, None, :, :]
        np.add.at(out, (it[c0:c1, :, None, None], is_[None, None, :, :]), I)
    return out


def k_matrix(test: RWG, bc: BCDual, k: float, chunk: int = 12) -> np.ndarray:
    """Kmat_PV[m, n] = <f_m, K g_n> (principal value on the source plane)."""
    b7, w7 = tri7()
    b3, w3 = tri3()
    ref = bc.refined
    Tr = ref.xyz[ref.tri]                                  # (nR,3,3)
    rr = points(Tr, b3)                                    # (nR,3,3)
    Wr = w3[None, :] * ref.area[:, None]                   # (nR,3)
    alpha, beta = bc_eval_coeffs(bc)
    S = sp.csr_matrix((np.ones(len(bc.fn)), (np.arange(len(bc.fn)), bc.fn)), shape=(len(bc.fn), bc.n))
    Tt = test.xyz[test.tri]
    rt = points(Tt, b7)
    it, ct = _local_coeffs(test)
    out = np.zeros((test.n, bc.n), dtype=np.complex128)
    inv4pi = 1.0 / (4.0 * np.pi)
    for c0 in range(0, len(Tt), chunk):
        c1 = min(c0 + chunk, len(Tt))
        c = c1 - c0
        P = rt[c0:c1].reshape(-1, 3)                       # (p,3)
        st = static_integrals(P, Tr, need=("grad",))
        V = st["grad"] * inv4pi + 0j                       # (p,nR,3)
        D = P[:, None, None, :] - rr[None, :, :, :]        # (p,nR,3,3)
        R = np.linalg.norm(D, axis=-1)
        cf = g1_grad_factor(R, k) * Wr[None]               # (p,nR,3)
        V += np.einsum("prq,prqx->prx", cf, D)
        Ve = V[:, bc.rtri, :]                              # (p,E,3)
        bt = alpha[None, :, None] * P[:, None, :] - beta[None, :, :]   # (p,E,3)
        W = np.cross(Ve, bt)                               # (p,E,3)
        Wn = (S.T @ W.transpose(1, 0, 2).reshape(len(bc.fn), -1)).reshape(bc.n, c * 7, 3)  # (N,p,3)
        Wn = Wn.reshape(bc.n, c, 7, 3)
        At = test.area[c0:c1]
        phit = (rt[c0:c1, :, None, :] - Tt[c0:c1, None, :, :]) / (2.0 * At)[:, None, None, None]  # (c,7,3i,3x)
        Wt = w7[None, :] * At[:, None]
        contrib = np.einsum("tq,tqix,ntqx->tin", Wt, phit, Wn) * ct[c0:c1, :, None]
        np.add.at(out, (it[c0:c1, :, None], np.arange(bc.n)[None, None, :]), contrib)
    return out


def mixed_gram(test: RWG, bc: BCDual) -> np.ndarray:
    """D[m, n] = <f_m, n_in x g_n> on a closed outward-oriented surface (Sec. IV)."""
    b3, w3 = tri3()
    ref = bc.refined
    alpha, beta = bc_eval_coeffs(bc)
    out = np.zeros((test.n, bc.n))
    nin = -test.normal
    for e in range(len(bc.fn)):
        rt_ = bc.rtri[e]
        T = ref.parent[rt_]
        q = b3 @ ref.xyz[ref.tri[rt_]]                      # (3,3)
        g = alpha[e] * q - beta[e]
        ng = np.cross(nin[T][None, :], g)
        for i in range(3):
            m = test.tri_rwg[T, i]
            if m < 0:
                continue
            f = test.tri_sign[T, i] * test.length[m] / (2.0 * test.area[T]) * (q - test.xyz[test.tri[T, i]])
            out[m, bc.fn[e]] += ref.area[rt_] * np.sum(w3 * np.einsum("qx,qx->q", f, ng))
    return out


def rwg_gram(rwg: RWG) -> np.ndarray:
    """<f_m, f_n> (exact with the 3-point rule)."""
    b3, w3 = tri3()
    out = np.zeros((rwg.n, rwg.n))
    for t in range(len(rwg.tri)):
        q = b3 @ rwg.xyz[rwg.tri[t]]
        for i in range(3):
            m = rwg.tri_rwg[t, i]
            if m < 0:
                continue
            fm = rwg.tri_sign[t, i] * rwg.length[m] / (2 * rwg.area[t]) * (q - rwg.xyz[rwg.tri[t, i]])
            for j in range(3):
                n = rwg.tri_rwg[t, j]
                if n < 0:
                    continue
                fn = rwg.tri_sign[t, j] * rwg.length[n] / (2 * rwg.area[t]) * (q - rwg.xyz[rwg.tri[t, j]])
                out[m, n] += rwg.area[t] * np.sum(w3 * np.einsum("qx,qx->q", fm, fn))
    return out


def bc_gram(bc: BCDual) -> np.ndarray:
    """<g_m, g_n> for dual functions (exact with the 3-point rule on refined triangles)."""
    b3, w3 = tri3()
    ref = bc.refined
    alpha, beta = bc_eval_coeffs(bc)
    out = np.zeros((bc.n, bc.n))
    by_tri: dict[int, list[int]] = {}
    for e in range(len(bc.fn)):
        by_tri.setdefault(int(bc.rtri[e]), []).append(e)
    for r, lst in by_tri.items():
        q = b3 @ ref.xyz[ref.tri[r]]
        vals = [alpha[e] * q - beta[e] for e in lst]
        for a, ea in enumerate(lst):
            for b_, eb in enumerate(lst):
                out[bc.fn[ea], bc.fn[eb]] += ref.area[r] * np.sum(w3 * np.einsum("qx,qx->q", vals[a], vals[b_]))
    return out


def bc_field_moments(bc: BCDual, field) -> np.ndarray:
    """<g_n, F> for a vector field F(points (P,3)) -> (P,3) complex."""
    b3, w3 = tri3()
    ref = bc.refined
    alpha, beta = bc_eval_coeffs(bc)
    q = points(ref.xyz[ref.tri], b3)                       # (nR,3,3)
    F = field(q.reshape(-1, 3)).reshape(q.shape)
    out = np.zeros(bc.n, dtype=np.complex128)
    for e in range(len(bc.fn)):
        r = bc.rtri[e]
        g = alpha[e] * q[r] - beta[e]
        out[bc.fn[e]] += ref.area[r] * np.sum(w3 * np.einsum("qx,qx->q", g, F[r]))
    return out


def field_moments(rwg: RWG, field) -> np.ndarray:
    """<f_n, F> with the 7-point rule; field maps points (P,3) -> (P,3) complex."""
    b7, w7 = tri7()
    T = rwg.xyz[rwg.tri]
    q = points(T, b7)                                      # (nT,7,3)
    F = field(q.reshape(-1, 3)).reshape(q.shape)
    it, ct = _local_coeffs(rwg)
    out = np.zeros(rwg.n, dtype=np.complex128)
    for i in range(3):
        phi = (q - T[:, i, None, :]) / (2.0 * rwg.area)[:, None, None]
        val = np.einsum("q,tqx,tqx->t", w7, phi, F) * rwg.area * ct[:, i]
        np.add.at(out, it[:, i], val)
    return out


def planewave(theta: float, phi: float, pol: int, k: float, E0: float = 1.0):
    """Incident plane wave arriving from direction (theta, phi): k^ = -r^(theta, phi),
    polarisation theta^ (pol 0) or phi^ (pol 1), exp(+jwt) convention."""
    st, ct_, sp_, cp = np.sin(theta), np.cos(theta), np.sin(phi), np.cos(phi)
    khat = -np.array([st * cp, st * sp_, ct_])
    p = np.array([ct_ * cp, ct_ * sp_, -st]) if pol == 0 else np.array([-sp_, cp, 0.0])

    def field(r):
        return E0 * p[None, :] * np.exp(-1j * k * (r @ khat))[:, None]
    return field


def excitation(rwg: RWG, theta, phi, pol, k: float) -> np.ndarray:
    """V^[n] = <f_n, n x n x E_inc> = -<f_n, E_inc> (Sec. IV, eq. (V1); tested with the
    equivalent-surface RWG functions).  Returns (N, nrhs)."""
    th = np.atleast_1d(theta); ph = np.atleast_1d(phi); po = np.atleast_1d(pol)
    return np.stack([-field_moments(rwg, planewave(th[i], ph[i], int(po[i]), k)) for i in range(len(th))], axis=1)


def far_field(rwg: RWG, coeff: np.ndarray, theta: np.ndarray, phi: np.ndarray, k: float) -> np.ndarray:
    """Far-field pattern F(r^) with E ~ F exp(-jkr)/r radiated by sum_n coeff_n f_n:
    F = -j w mu0/(4 pi) (I - r^ r^) . sum_n coeff_n int f_n exp(jk r^.r') dS'.
    Returns (ndir, 3) complex (Cartesian)."""
    b7, w7 = tri7()
    T = rwg.xyz[rwg.tri]
    q = points(T, b7)
    it, ct = _local_coeffs(rwg)
    # current density at quadrature points
    Jq = np.zeros(q.shape, dtype=np.complex128)
    for i in range(3):
        phi_i = (q - T[:, i, None, :]) / (2.0 * rwg.area)[:, None, None]
        Jq += phi_i * (ct[:, i] * coeff[it[:, i]])[:, None, None]
    Wq = (w7[None, :] * rwg.area[:, None]).reshape(-1)
    Jq = Jq.reshape(-1, 3)
    qf = q.reshape(-1, 3)
    th = np.atleast_1d(theta); ph = np.atleast_1d(phi)
    rh = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=1)
    ph_ = np.exp(1j * k * (rh @ qf.T)) * Wq[None, :]          # (ndir, nq)
    N = ph_ @ Jq                                               # (ndir, 3)
    Nt = N - rh * np.sum(rh * N, axis=1)[:, None]
    return -1j * k * ETA0 / (4.0 * np.pi) * Nt


def rcs(F: np.ndarray, E0: float = 1.0) -> np.ndarray:
    """Bistatic RCS sigma = 4 pi |F|^2/|E0|^2 (lambda^2 units when k = 2 pi)."""
    return 4.0 * np.pi * np.sum(np.abs(F) ** 2, axis=1) / (E0 * E0)
