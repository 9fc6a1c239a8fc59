"""Driven elements (delta-gap feeds) and a PEC ground plane by image theory (oracle).

Test infrastructure: only tests/, the benchmark's CPU leg and smoke() use this.

Delta-gap feed (Sec. VI: each helix is driven by a delta-gap source at its
centre).  The paper derives the macromodel for an incident field and states
that it carries over to driven elements without giving the equations; the
reading implemented here follows its own steps:
  * a gap of voltage V across a chain of edges is an impressed field
    V delta(xi) xi^ across the gap, xi^ the chosen feed direction; in the MoM
    form (Z = j k eta0 L, right-hand side <f, E>) edge g of the gap gets
    f_g = s_g V l_g, s_g = sign of (xi^ . n_g) with n_g the in-plane normal of
    edge g pointing from its T+ to its T- triangle;
  * the scatterer's equation, eq. (EFIEdiscretized1), gains that impressed
    field, G^(E,J) J + G^(E,H^) H^ + G^(E,E^) E^ = -f (paper's sign, in which
    the incident field enters as -<f, E_inc>); eq. (EFIEdiscretized2) on the
    equivalent surface is unchanged (no source there);
  * eliminating H^ as in eq. (Hdiscretized1): A J + B E^ = -f, so
    J = -A^-1 B E^ + J_f with J_f = -A^-1 f (the element's current with its
    equivalent surface shorted, E^ = 0), and J^ = T J = -M E^ + T J_f;
  * the exterior equation, eq. (EFIEDiscretized_Outer), D E^ = -G J^ + V^,
    becomes (D - G M) E^ = V^ - G J^_f with J^_f = T J_f: the same operator
    as eq. (finalsystem) with the excitation V^_eff = V^ - G J^_f.

Ground plane (Sec. VI: "image theory" for the reflectarrays' ground plane).
A PEC plane z = z_g is replaced by the image of every element below it (the
planar elements here map onto themselves under z -> -z in their own frame, so
an image element has the same type at the mirrored offset) and by the image of
the incident field, E_img(r) = S E_inc(R r), R(x, y, z) = (x, y, 2 z_g - z),
S = diag(-1, -1, 1): the total field's tangential part then vanishes on the
plane.
"""
from __future__ import annotations

import numpy as np

from .basis import RWG
from .operators import ETA0, efie_matrix, field_moments, planewave


# ---------------------------------------------------------------- delta gap
def gap_signs(rwg: RWG, port: np.ndarray, direction) -> np.ndarray:
    """s_g = sign(xi^ . n_g), n_g the in-plane normal of edge g from T+ to T-."""
    d = np.asarray(direction, dtype=np.float64)
    a = rwg.xyz[rwg.edges[port, 0]]
    b = rwg.xyz[rwg.edges[port, 1]]
    e = (b - a) / np.linalg.norm(b - a, axis=1)[:, None]
    cp = rwg.xyz[rwg.tri[rwg.tplus[port]]].mean(axis=1)
    cm = rwg.xyz[rwg.tri[rwg.tminus[port]]].mean(axis=1)
    c = cm - cp
    n = c - (c * e).sum(axis=1)[:, None] * e
    s = np.sign(n @ d)
    if np.any(s == 0):
        raise ValueError("feed direction parallel to a gap edge")
    return s


def feed_vector(rwg: RWG, port: np.ndarray, direction, volts: complex = 1.0) -> np.ndarray:
    """MoM right-hand side of a delta gap: f_g = s_g V l_g on the gap edges."""
    f = np.zeros(rwg.n, dtype=np.complex128)
    f[port] = gap_signs(rwg, port, direction) * rwg.length[port] * volts
    return f


def port_current(rwg: RWG, J: np.ndarray, port: np.ndarray, direction) -> np.ndarray:
    """Current through the gap along xi^: I = sum_g s_g J_g l_g (works on (n,) or (n, r))."""
    w = gap_signs(rwg, port, direction) * rwg.length[port]
    return np.tensordot(w, J[port], axes=(0, 0))


def element_feed(em, f: np.ndarray):
    """(J_f, J^_f) of one driven element: J_f = -A^-1 f, J^_f = T J_f."""
    Jf = -np.linalg.solve(em.A, f)
    return Jf, em.T @ Jf


def driven_currents(em, Ehat: np.ndarray, Jf: np.ndarray):
    """J = -A^-1 B E^ + J_f and J^ = T J for a driven element."""
    J = -np.linalg.solve(em.A, em.B @ Ehat) + Jf
    return J, em.T @ J


def direct_driven_mom(rwg: RWG, f: np.ndarray, k: float) -> np.ndarray:
    """Direct MoM of the scatterers alone: j k eta0 L J = f."""
    Z = 1j * k * ETA0 * efie_matrix(rwg, rwg, k)
    return np.linalg.solve(Z, f)


# ---------------------------------------------------------------- ground plane
def image_field(field, z_ground: float):
    """E_img(r) = S E(R r): the field of the sources' images below z = z_g."""
    S = np.array([-1.0, -1.0, 1.0])

    def fimg(r):
        rr = np.array(r, dtype=np.float64, copy=True)
        rr[:, 2] = 2.0 * z_ground - rr[:, 2]
        return field(rr) * S[None, :]
    return fimg


def ground_planewave(theta: float, phi: float, pol: int, k: float, z_ground: float):
    """Incident plane wave plus its image in the plane z = z_g."""
    f0 = planewave(theta, phi, pol, k)
    f1 = image_field(f0, z_ground)
    return lambda r: f0(r) + f1(r)


def ground_excitation(rwg: RWG, theta, phi, pol, k: float, z_ground: float) -> np.ndarray:
    """V^[n] = -<f_n, E_inc + E_img> (Sec. IV, eq. (V1) with the image field); (N, nrhs)."""
    th = np.atleast_1d(theta); ph = np.atleast_1d(phi); po = np.atleast_1d(pol)
    return np.stack([-field_moments(rwg, ground_planewave(th[i], ph[i], int(po[i]), k, z_ground))
                     for i in range(len(th))], axis=1)


def image_offsets(offsets: np.ndarray, z_ground: float) -> np.ndarray:
    """Offsets of the image elements: (x, y, 2 z_g - z)."""
    o = np.array(offsets, dtype=np.float64, copy=True)
    o[:, 2] = 2.0 * z_ground - o[:, 2]
    return o
