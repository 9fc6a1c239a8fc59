"""Direct EFIE method of moments for PEC surfaces (oracle).

The standard MoM the paper compares against (Sec. I, Sec. VI): tangential
total E vanishes on the PEC, E_s = -jw mu0 L J, so
  jw mu0 Lmat J = <f, E_inc>,  Z = j k eta0 Lmat.
Used by the pins (Mie series, macromodel vs full MoM of the same array).
"""
from __future__ import annotations

import numpy as np

from .basis import RWG, build_rwg
from .operators import ETA0, efie_matrix, field_moments, planewave


def mom_solve(rwg: RWG, k: float, theta, phi, pol) -> np.ndarray:
    Z = 1j * k * ETA0 * efie_matrix(rwg, rwg, k)
    th = np.atleast_1d(theta); ph = np.atleast_1d(phi); po = np.atleast_1d(pol)
    V = np.stack([field_moments(rwg, planewave(th[i], ph[i], int(po[i]), k)) for i in range(len(th))], axis=1)
    return np.linalg.solve(Z, V)


def merge_meshes(meshes):
    """Concatenate (xyz, tri) meshes into one (disjoint surfaces)."""
    xyz, tri, off = [], [], 0
    for m in meshes:
        xyz.append(m.xyz); tri.append(m.tri + off); off += len(m.xyz)
    return np.vstack(xyz), np.vstack(tri)
