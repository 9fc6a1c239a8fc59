"""Closed-form static potential integrals over a flat triangle (oracle).

The Green's function of Sec. II-C, G = exp(-j k R)/(4 pi R), is split as
G = 1/(4 pi R) + G1 with G1 = (exp(-j k R) - 1)/(4 pi R) smooth.  The 1/R part
is integrated over the source triangle in closed form (singularity
extraction; Wilton et al. 1984, Graglia 1993 -- published formulas restated
here); G1 and its gradient are integrated by quadrature.

For an observation point r, a triangle with unit normal n (from its vertex
order) and edges i traversed counter-clockwise about n:
  rho = projection of r on the plane, d = (r - v0).n,
  s_i = unit edge direction, m_i = s_i x n (outward in-plane edge normal),
  l+-_i = (P+-_i - rho).s_i, t0_i = (P-_i - rho).m_i, R0_i^2 = t0_i^2 + d^2,
  R+-_i = |r - P+-_i|, f2_i = ln((R+ + l+)/(R- + l-)),
  beta_i = atan2(t0 l+, R0^2 + |d| R+) - atan2(t0 l-, R0^2 + |d| R-).
Then
  S0    = int 1/R dS'                = sum_i t0_i f2_i - |d| sum_i beta_i,
  Sv    = int (rho' - rho)/R dS'     = 1/2 sum_i m_i (R0^2 f2 + l+ R+ - l- R-),
  grad  = grad_r int 1/R dS'         = -n sgn(d) sum_i beta_i - sum_i m_i f2_i,
where sgn(0) = 0: on the plane the gradient is the principal value (the
half-residue of the K operator is added separately).  Heights |d| and edge
distances |t0| below 1e-10 * sqrt(area) are set to exactly 0 (rounding noise
of coplanar points); a point on an edge segment itself (R0 = 0 between the
end points) or on an end point takes f2 = 0, the principal value across that edge.
"""
from __future__ import annotations

import numpy as np

SNAP = 1e-10  # relative threshold below which a height or edge distance is taken as 0


def _f2(lp, lm, Rp, Rm, R0sq):
    """ln((R+ + l+)/(R- + l-)) evaluated without cancellation.

    Branches on the signs of l+- (l+ > l- always): both >= 0, both <= 0, or
    straddling (then R- + l- = R0^2/(R- - l-))."""
    out = np.zeros_like(lp)
    a = lm >= 0.0
    b = (~a) & (lp <= 0.0)
    c = ~(a | b)
    a = a & (Rm + lm > 0.0)          # an end point itself: principal value, 0
    b = b & (Rp - lp > 0.0)
    out[a] = np.log((Rp[a] + lp[a]) / (Rm[a] + lm[a]))
    out[b] = np.log((Rm[b] - lm[b]) / (Rp[b] - lp[b]))
    c0 = c & (R0sq == 0.0)          # on the edge segment itself: principal value, 0
    c1 = c & (R0sq > 0.0)
    out[c1] = np.log((Rp[c1] + lp[c1]) * (Rm[c1] - lm[c1]) / R0sq[c1])
    out[c0] = 0.0
    return out


def static_integrals(r: np.ndarray, tri_xyz: np.ndarray, need=("S0", "Sv", "grad")):
    """Closed-form integrals for all (point, triangle) pairs.

    r: (P, 3); tri_xyz: (T, 3, 3).  Returns dict with arrays of shape (P, T)
    for 'S0', (P, T, 3) for 'Sv', 'grad' and 'rho'.
    """
    r = np.asarray(r, dtype=np.float64)
    v = np.asarray(tri_xyz, dtype=np.float64)
    cr = np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0])
    n = cr / np.linalg.norm(cr, axis=1)[:, None]                     # (T,3)
    d = np.einsum("ptk,tk->pt", r[:, None, :] - v[None, :, 0, :], n)  # (P,T)
    rho = r[:, None, :] - d[..., None] * n[None]                     # (P,T,3)
    # coplanar points: a height below SNAP * (triangle size) is rounding noise and is
    # set to exactly 0 so that sgn(d) = 0 (principal value, no spurious half residue)
    scale = np.sqrt(0.5 * np.linalg.norm(cr, axis=1))[None, :]
    d = np.where(np.abs(d) < SNAP * scale, 0.0, d)
    ad = np.abs(d)
    S0 = np.zeros(d.shape)
    Sv = np.zeros(d.shape + (3,))
    gt = np.zeros(d.shape + (3,))
    bsum = np.zeros(d.shape)
    for i in range(3):
        Pm = v[:, i]
        Pp = v[:, (i + 1) % 3]
        s = Pp - Pm
        s = s / np.linalg.norm(s, axis=1)[:, None]
        m = np.cross(s, n)
        lp = np.einsum("ptk,tk->pt", Pp[None] - rho, s)
        lm = np.einsum("ptk,tk->pt", Pm[None] - rho, s)
        t0 = np.einsum("ptk,tk->pt", Pm[None] - rho, m)
        t0 = np.where(np.abs(t0) < SNAP * scale, 0.0, t0)
        R0sq = t0 * t0 + d * d
        Rp = np.linalg.norm(r[:, None, :] - Pp[None], axis=2)
        Rm = np.linalg.norm(r[:, None, :] - Pm[None], axis=2)
        f2 = _f2(lp, lm, Rp, Rm, R0sq)
        pos = R0sq > 0.0
        beta = np.where(pos, np.arctan2(t0 * lp, R0sq + ad * Rp) - np.arctan2(t0 * lm, R0sq + ad * Rm), 0.0)
        S0 += t0 * f2 - ad * beta
        bsum += beta
        if "Sv" in need:
            Sv += 0.5 * (R0sq * f2 + lp * Rp - lm * Rm)[..., None] * m[None]
        if "grad" in need:
            gt -= f2[..., None] * m[None]
    out = {"S0": S0, "rho": rho}
    if "Sv" in need:
        out["Sv"] = Sv
    if "grad" in need:
        out["grad"] = gt - (np.sign(d) * bsum)[..., None] * n[None]
    return out


def g1(R: np.ndarray, k: float) -> np.ndarray:
    """(exp(-jkR) - 1)/(4 pi R), with its limit -jk/(4 pi) at R = 0."""
    R = np.asarray(R, dtype=np.float64)
    out = np.empty(R.shape, dtype=np.complex128)
    z = R == 0.0
    nz = ~z
    x = k * R[nz]
    out[nz] = (-2.0 * np.sin(0.5 * x) ** 2 - 1j * np.sin(x)) / (4.0 * np.pi * R[nz])
    out[z] = -1j * k / (4.0 * np.pi)
    return out


def g1_grad_factor(R: np.ndarray, k: float) -> np.ndarray:
    """c(R) with grad_r G1(|r - r'|) = c(R) (r - r'); c = -((1+jkR) e^{-jkR} - 1)/(4 pi R^3), 0 at R = 0."""
    R = np.asarray(R, dtype=np.float64)
    out = np.zeros(R.shape, dtype=np.complex128)
    nz = R != 0.0
    x = k * R[nz]
    re = -2.0 * np.sin(0.5 * x) ** 2 + x * np.sin(x)
    im = x * np.cos(x) - np.sin(x)
    out[nz] = -(re + 1j * im) / (4.0 * np.pi * R[nz] ** 3)
    return out


def green(R: np.ndarray, k: float) -> np.ndarray:
    """Free-space Green's function exp(-jkR)/(4 pi R) (Sec. II-C)."""
    return np.exp(-1j * k * R) / (4.0 * np.pi * R)
