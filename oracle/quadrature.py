"""Triangle quadrature rules (oracle).

Rules are returned as (barycentric coords (n, 3), weights (n,)) with weights
summing to 1, so that  int_T f dS = area(T) * sum_q w_q f(r_q).

* ``tri3``  -- degree 2, 3 interior points (2/3, 1/6, 1/6).
* ``tri7``  -- degree 5, Radon's 7-point formula (closed form in sqrt(15)).
* ``collapsed_gauss(d)`` -- degree d: Gauss-Legendre product on the unit
  square mapped onto the triangle by the collapsed (Duffy) map
  x = u, y = v (1 - u), Jacobian (1 - u).  Used where the AIM projection needs
  exactness to degree 3*N_O + 1 (Sec. V, step (i)).
"""
from __future__ import annotations

import math

import numpy as np


def tri3():
    b = np.array([[2 / 3, 1 / 6, 1 / 6], [1 / 6, 2 / 3, 1 / 6], [1 / 6, 1 / 6, 2 / 3]])
    return b, np.full(3, 1.0 / 3.0)


def tri7():
    s = math.sqrt(15.0)
    a1 = (6.0 - s) / 21.0
    a2 = (6.0 + s) / 21.0
    w1 = (155.0 - s) / 1200.0
    w2 = (155.0 + s) / 1200.0
    b = [[1 / 3, 1 / 3, 1 / 3]]
    w = [9.0 / 40.0]
    for a, ww in ((a1, w1), (a2, w2)):
        c = 1.0 - 2.0 * a
        b += [[a, a, c], [a, c, a], [c, a, a]]
        w += [ww, ww, ww]
    return np.array(b), np.array(w)


def collapsed_gauss(degree: int):
    """Degree-`degree` rule from Gauss-Legendre on [0,1]^2 through x=u, y=v(1-u)."""
    nu = (degree + 3) // 2          # u-integrand has degree degree+1
    nv = (degree + 2) // 2          # v-integrand has degree degree
    xu, wu = np.polynomial.legendre.leggauss(nu)
    xv, wv = np.polynomial.legendre.leggauss(nv)
    u = 0.5 * (xu + 1.0)
    v = 0.5 * (xv + 1.0)
    wu = 0.5 * wu
    wv = 0.5 * wv
    B, W = [], []
    for i in range(nu):
        for j in range(nv):
            x = u[i]
            y = v[j] * (1.0 - u[i])
            B.append([1.0 - x - y, x, y])
            W.append(2.0 * wu[i] * wv[j] * (1.0 - u[i]))  # reference area 1/2 -> weights sum to 1
    return np.array(B), np.array(W)


def points(tri_xyz: np.ndarray, bary: np.ndarray) -> np.ndarray:
    """Quadrature points for triangles (T, 3, 3) -> (T, Q, 3)."""
    return np.einsum("qa,tai->tqi", bary, tri_xyz)
