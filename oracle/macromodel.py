"""Per-element macromodel and the exterior system (oracle).

Sec. II-D/E/F: the six Stratton-Chu matrices of one element,
  G^(E,J)  = -jw mu0 Lmat(S, S)        G^(E^,J)  = -jw mu0 Lmat(S^, S)
  G^(E,H^) = -jw mu0 Lmat(S, S^)       G^(E^,H^) = -jw mu0 Lmat(S^, S^)
  G^(E,E^) = Kmat(S, S^')              G^(E^,E^) = Kmat_PV(S^, S^') + D/2
(the last evaluated as the limit from outside the equivalent surface);
eq. (Hdiscretized1): H^ = -G^(E^,H^)^-1 [G^(E^,E^) E^ + G^(E^,J) J];
eq. (JM): A = G^(E,J) - G^(E,H^) G^(E^,H^)^-1 G^(E^,J),
          B = G^(E,E^) - G^(E,H^) G^(E^,H^)^-1 G^(E^,E^);
eq. (JABE): J = -A^-1 B E^;  eq. (Tm1): T = G^(E^,H^)^-1 G^(E^,J).
Sec. III: the blocks are computed once per distinct element.
Sec. IV: D[m, n] = <f^_m, n x f^'_n>, G^(E^,J^)_{mm'} = -jw mu0 Lmat(S^_m, S^_m'),
final system (D - G^(E^,J^) T A^-1 B) E^ = V^, eq. (finalsystem).
All linear solves use LU factorisations, never explicit inverses.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla

from .basis import RWG, BCDual, build_rwg, build_bc
from .operators import ETA0, efie_matrix, k_matrix, mixed_gram


@dataclass
class ElementModel:
    rwg_s: RWG
    rwg_e: RWG
    bc: BCDual
    k: float
    G_EJ: np.ndarray
    G_EH: np.ndarray
    G_hEJ: np.ndarray
    G_hEH: np.ndarray
    G_EE: np.ndarray
    G_hEE: np.ndarray
    D: np.ndarray
    T: np.ndarray
    A: np.ndarray
    B: np.ndarray
    M: np.ndarray            # T A^-1 B, applied blockwise in eq. (MV_product1)

    def currents(self, Ehat: np.ndarray):
        """J = -A^-1 B E^ (eq. (JABE)) and J^ = T J (eq. (Tm1))."""
        J = -np.linalg.solve(self.A, self.B @ Ehat)
        return J, self.T @ J


def build_element(scat_xyz, scat_tri, eq_xyz, eq_tri, k: float) -> ElementModel:
    rs = build_rwg(scat_xyz, scat_tri)
    re = build_rwg(eq_xyz, eq_tri)
    bc = build_bc(re)
    c = -1j * k * ETA0
    G_EJ = c * efie_matrix(rs, rs, k)
    G_EH = c * efie_matrix(rs, re, k)
    G_hEJ = c * efie_matrix(re, rs, k)
    G_hEH = c * efie_matrix(re, re, k)
    G_EE = k_matrix(rs, bc, k)
    D = mixed_gram(re, bc)
    G_hEE = k_matrix(re, bc, k) + 0.5 * D
    lu = sla.lu_factor(G_hEH)
    T = sla.lu_solve(lu, G_hEJ)
    A = G_EJ - G_EH @ sla.lu_solve(lu, G_hEJ)
    B = G_EE - G_EH @ sla.lu_solve(lu, G_hEE)
    M = T @ np.linalg.solve(A, B)
    return ElementModel(rs, re, bc, k, G_EJ, G_EH, G_hEJ, G_hEH, G_EE, G_hEE, D, T, A, B, M)


def coupling_block(rwg_a: RWG, rwg_b: RWG, k: float) -> np.ndarray:
    """G^(E^,J^) block between two equivalent surfaces (eq. (Gouter1))."""
    return -1j * k * ETA0 * efie_matrix(rwg_a, rwg_b, k)


def translated_rwg(rwg: RWG, offset) -> RWG:
    from dataclasses import replace
    return replace(rwg, xyz=rwg.xyz + np.asarray(offset, dtype=np.float64)[None, :])


def dense_exterior_operator(models, type_of, offsets, k: float) -> np.ndarray:
    """Z = D - G^(E^,J^) T A^-1 B for a small array, G dense (eq. (finalsystem))."""
    sizes = [models[t].rwg_e.n for t in type_of]
    off = np.concatenate([[0], np.cumsum(sizes)])
    N = off[-1]
    Z = np.zeros((N, N), dtype=np.complex128)
    rw = [translated_rwg(models[t].rwg_e, offsets[e]) for e, t in enumerate(type_of)]
    for a in range(len(type_of)):
        for b in range(len(type_of)):
            G = coupling_block(rw[a], rw[b], k)
            Z[off[a]:off[a + 1], off[b]:off[b + 1]] = -G @ models[type_of[b]].M
        Z[off[a]:off[a + 1], off[a]:off[a + 1]] += models[type_of[a]].D
    return Z
