"""Pins of the oracle's driven elements (delta-gap feed) and ground plane (image
theory), the readings of Sec. VI written out in oracle/drive.py.

* Delta gap: the macromodel with the feed in the scatterer's equation must give
  the scatterer currents of the direct MoM of the same scatterer with the same
  gap (the paper's claim: exact up to discretisation; the loop's equivalent box
  is meshed 6x6x1, as in the plane-wave pins P3/P5), and the admittance matrix
  of two fed elements is symmetric (reciprocity): to round-off for the
  Galerkin direct MoM, to discretisation error for the macromodel system,
  which is not symmetric.
* Ground plane: the incident field plus its image has zero tangential part on
  the plane; the direct MoM of element + image is exactly antisymmetric
  (J_image = -J, horizontal currents); the macromodel of the doubled array
  agrees with that direct MoM to discretisation error.
A sign slip in the gap field, the image's polarisation or its phase fails one
of these by O(1)."""
import numpy as np
import pytest

from paper_1712_02443_gb300 import workloads as wl
from oracle import drive as dr
from oracle.basis import build_rwg
from oracle.macromodel import build_element, coupling_block, dense_exterior_operator, translated_rwg
from oracle.mom import merge_meshes
from oracle.operators import ETA0, efie_matrix, field_moments, planewave

K0 = 2.0 * np.pi


@pytest.fixture(scope="module")
def fed():
    et, gap, d = wl.fed_loop_element()
    em = build_element(et.scatterer.xyz, et.scatterer.tri, et.equiv.xyz, et.equiv.tri, K0)
    return et, em, gap, d


def test_fed_loop_mesh_has_a_straight_gap(fed):
    et, em, gap, d = fed
    a = em.rwg_s.xyz[em.rwg_s.edges[gap]]
    assert np.allclose(a[..., 0], 0.0) and np.all(a[..., 1] < -0.15)        # the cut x = 0 across the trace
    assert np.isclose(em.rwg_s.length[gap].sum(), 0.04)                      # spans the 0.04 trace width
    assert np.all(dr.gap_signs(em.rwg_s, gap, d) == dr.gap_signs(em.rwg_s, gap, d)[0])


def test_delta_gap_macromodel_matches_direct_mom(fed):
    et, em, gap, d = fed
    f = dr.feed_vector(em.rwg_s, gap, d, 1.0)
    Jd = dr.direct_driven_mom(em.rwg_s, f, K0)
    Jf, Jhf = dr.element_feed(em, f)
    G = coupling_block(em.rwg_e, em.rwg_e, K0)
    E = np.linalg.solve(em.D - G @ em.M, -G @ Jhf)
    J, _ = dr.driven_currents(em, E, Jf)
    assert np.linalg.norm(J - Jd) / np.linalg.norm(Jd) < 1e-2
    Yd = dr.port_current(em.rwg_s, Jd, gap, d)
    Ym = dr.port_current(em.rwg_s, J, gap, d)
    assert abs(Ym - Yd) / abs(Yd) < 1e-2
    # the feed matters: with the gap field reversed the currents reverse
    Jr, _ = dr.driven_currents(em, -E, -Jf)
    assert np.linalg.norm(Jr + Jd) / np.linalg.norm(Jd) < 1e-2


def test_delta_gap_reciprocity(fed):
    et, em, gap, d = fed
    offs = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0]])
    f = dr.feed_vector(em.rwg_s, gap, d, 1.0)
    Jf, Jhf = dr.element_feed(em, f)
    n, ns = em.rwg_e.n, em.rwg_s.n
    Z = dense_exterior_operator([em], [0, 0], offs, K0)
    rw = [translated_rwg(em.rwg_e, o) for o in offs]
    G = np.block([[coupling_block(rw[a], rw[b], K0) for b in range(2)] for a in range(2)])
    Ym = np.zeros((2, 2), dtype=np.complex128)
    for j in range(2):
        Jh = np.zeros(2 * n, dtype=np.complex128)
        Jh[j * n:(j + 1) * n] = Jhf
        E = np.linalg.solve(Z, -G @ Jh)
        for i in range(2):
            Ji, _ = dr.driven_currents(em, E[i * n:(i + 1) * n], Jf if i == j else 0 * Jf)
            Ym[i, j] = dr.port_current(em.rwg_s, Ji, gap, d)
    xyz, tri = merge_meshes([et.scatterer.translated(o) for o in offs])
    r2 = build_rwg(xyz, tri)
    Yd = np.zeros((2, 2), dtype=np.complex128)
    for j in range(2):
        ff = np.zeros(2 * ns, dtype=np.complex128)
        ff[j * ns:(j + 1) * ns] = f
        JJ = dr.direct_driven_mom(r2, ff, K0)
        for i in range(2):
            Yd[i, j] = dr.port_current(em.rwg_s, JJ[i * ns:(i + 1) * ns], gap, d)
    assert abs(Yd[0, 1] - Yd[1, 0]) <= 1e-10 * abs(Yd[0, 1])
    assert abs(Ym[0, 1] - Ym[1, 0]) <= 1e-2 * abs(Ym[0, 1])
    assert np.abs(Ym - Yd).max() <= 1e-2 * np.abs(Yd).max()
    assert abs(Yd[0, 1]) > 0.1 * abs(Yd[0, 0])   # the coupling is not negligible


def test_ground_field_has_no_tangential_part_on_the_plane():
    zg = -0.1
    g = wl.rng(9, 1)
    r = np.column_stack([g.uniform(-1, 1, 50), g.uniform(-1, 1, 50), np.full(50, zg)])
    for pol in (0, 1):
        E = dr.ground_planewave(0.6, 0.4, pol, K0, zg)(r)
        E0 = planewave(0.6, 0.4, pol, K0)(r)
        assert np.abs(E[:, :2]).max() <= 1e-12
        assert np.allclose(E[:, 2], 2 * E0[:, 2])


@pytest.mark.parametrize("pol", [0, 1])
def test_ground_plane_direct_and_macromodel(loop_model, pol):
    et = wl.loop_element()
    zg = -0.1
    lay = wl.ground_plane_array(wl.ArrayLayout([et], np.zeros(1, dtype=np.int32), np.zeros((1, 3))), zg)
    assert np.allclose(lay.offsets[1], [0, 0, -0.2])
    th, ph = 0.5, 0.35
    xyz, tri = merge_meshes([et.scatterer.translated(o) for o in lay.offsets])
    r2 = build_rwg(xyz, tri)
    Jm = np.linalg.solve(1j * K0 * ETA0 * efie_matrix(r2, r2, K0),
                         field_moments(r2, dr.ground_planewave(th, ph, pol, K0, zg)))
    ns = loop_model.rwg_s.n
    assert np.linalg.norm(Jm[ns:] + Jm[:ns]) <= 1e-10 * np.linalg.norm(Jm[:ns])
    Z = dense_exterior_operator([loop_model], lay.type_of, lay.offsets, K0)
    V = np.concatenate([dr.ground_excitation(translated_rwg(loop_model.rwg_e, o), th, ph, pol, K0, zg)[:, 0]
                        for o in lay.offsets])
    E = np.linalg.solve(Z, V)
    n = loop_model.rwg_e.n
    J = np.concatenate([loop_model.currents(E[e * n:(e + 1) * n])[0] for e in range(2)])
    assert np.linalg.norm(J - Jm) / np.linalg.norm(Jm) < 2e-2
    # the ground plane changes the currents by O(1) (the check has teeth)
    J0 = np.linalg.solve(1j * K0 * ETA0 * efie_matrix(loop_model.rwg_s, loop_model.rwg_s, K0),
                         field_moments(loop_model.rwg_s, planewave(th, ph, pol, K0)))
    assert np.linalg.norm(Jm[:ns] - J0) / np.linalg.norm(Jm[:ns]) > 0.2
