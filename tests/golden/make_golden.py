"""Writes the oracle's expected values used by the GPU parity tests and smoke().

Calls only the CPU oracle (oracle/) and the seeded input generators; nothing
here comes from the CUDA path.  Re-run after any change to the oracle's
arithmetic:  python tests/golden/make_golden.py

Files (numpy .npz, complex128):
  c1_2x2.npz      2x2 loop array: x, y = Z_AIM x (full), V (theta=0 x-pol),
                  E = solution of the AIM system to 1e-12, E_dense (dense
                  exterior operator) for reference, the currents J, J^ of E,
                  and the far field F and RCS of J^ on 38 directions.
  ragged_3x5.npz  3x5 loop array, 3 right-hand sides: y (N x 3, full) for
                  x = workloads.random_cvec(N, 0, 8, nrhs=3) (checksum stored).
  c2_16x16.npz    16x16 loop array: sampled rows and y[rows] for
                  x = workloads.random_cvec(N, 1, 7) (checksum stored).
  c3_types_6x6.npz  6x6 array of the four loop types (outer 0.30/0.34/0.38/0.42,
                  seeded per cell), 64 right-hand sides: sampled rows of
                  y = Z_AIM X for X = workloads.random_cvec(N, 2, 7, nrhs=64),
                  and of the plane-wave excitation for the 8 x 8 incidence grid.
  c4_meander_2x2.npz  2x2 array of the reduced multiscale element (loop with a
                  meandered inner trace, workloads.MEANDER_REDUCED, 6x6x1 box):
                  Y = Z_AIM X (full) for X = workloads.random_cvec(N, 3, 7, nrhs=8),
                  V (theta = 0, x-pol) and E = its solution to 1e-12.

  c3_solve_6x6.npz  the 6x6 four-type array: excitations and solutions (GMRES
                  to 1e-11) of incidences 0 and 37 of the 8 x 8 grid.
  c4_meander_2x2_post.npz  currents J, J^ of the stored multiscale solution E
                  and the far field F and RCS of J^ on 38 directions.
  c4_full_element_2x1.npz  2x1 array of the full multiscale element (2,547
                  scatterer RWG, 8x8x2 box): Y = Z_AIM X for
                  X = workloads.random_cvec(N, 3, 11, nrhs=2) (checksum stored).

  fed_2x2.npz     2x2 array of the driven loop (delta gap at the middle of one
                  side, oracle/drive.py): volts of two excitations, V^_eff,
                  E (GMRES to 1e-12), J, J^ and the port currents.
  ground_2x2.npz  2x2 loops over a PEC plane z = -0.1 with their images (8
                  elements): V^ of two incidences (incident + image wave), E,
                  and the RCS of all J^ on 20 upper-half-space directions.

python tests/golden/make_golden.py [c4 | extra | drive]   (only that part)
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from paper_1712_02443_gb300 import workloads as wl  # noqa: E402
from oracle.aim import AIMArray, AIMParams, BlockCache  # noqa: E402
from oracle.gmres import gmres  # noqa: E402
from oracle.macromodel import build_element, dense_exterior_operator, translated_rwg  # noqa: E402
from oracle.basis import build_rwg  # noqa: E402
from oracle.mom import merge_meshes  # noqa: E402
from oracle.operators import excitation, far_field, rcs  # noqa: E402

K0 = 2.0 * np.pi
H, ORDER, NNF = 0.1, 2, 3


def _check(x):
    """Checksum of a seeded input (the tests regenerate x from its seed)."""
    return np.array([x.sum(), (np.abs(x) ** 2).sum()])


def main():
    t0 = time.time()
    et = wl.loop_element()
    em = build_element(et.scatterer.xyz, et.scatterer.tri, et.equiv.xyz, et.equiv.tri, K0)
    params = AIMParams(H, ORDER, NNF, wl.DEFAULT_GRID_PHASE)
    blocks = BlockCache([em], K0)
    print("element", time.time() - t0)

    # c1: 2x2
    lay = wl.loop_array(2, 2)
    A = AIMArray([em], lay.type_of, lay.offsets, params, K0, blocks=blocks)
    x = wl.random_cvec(A.n, 0, 7)
    y = A.matvec(x)
    V = np.concatenate([excitation(translated_rwg(em.rwg_e, o), 0.0, 0.0, 0, K0)[:, 0] for o in lay.offsets])
    E, it, hist = gmres(A.matvec, V, tol=1e-12, restart=100, max_iter=2000)
    Z = dense_exterior_operator([em], lay.type_of, lay.offsets, K0)
    Ed = np.linalg.solve(Z, V)
    # currents of the solution (eq. (JABE), eq. (Tm1)) and the far field of J^
    nh = em.rwg_e.n
    JJ = [em.currents(E[e * nh:(e + 1) * nh]) for e in range(len(lay.offsets))]
    J = np.concatenate([c[0] for c in JJ])
    Jh = np.concatenate([c[1] for c in JJ])
    xyz, tri = merge_meshes([lay.types[0].equiv.translated(o) for o in lay.offsets])
    rw = build_rwg(xyz, tri)
    th = np.deg2rad(np.concatenate([np.arange(0, 181, 10.0), np.arange(0, 181, 10.0)]))
    ph = np.deg2rad(np.concatenate([np.zeros(19), np.full(19, 90.0)]))
    F = far_field(rw, Jh, th, ph, K0)
    np.savez_compressed(os.path.join(HERE, "c1_2x2.npz"), x=x, y=y, V=V, E=E, E_dense=Ed,
                        offsets=lay.offsets, gmres_iters=it, J=J, Jhat=Jh, theta=th, phi=ph, F=F, sigma=rcs(F))
    print("c1", time.time() - t0, "iters", it)

    # ragged 3x5, 3 RHS
    lay = wl.loop_array(3, 5)
    A = AIMArray([em], lay.type_of, lay.offsets, params, K0, blocks=blocks)
    X = wl.random_cvec(A.n, 0, 8, nrhs=3)
    Y = np.stack([A.matvec(X[:, j]) for j in range(3)], axis=1)
    np.savez_compressed(os.path.join(HERE, "ragged_3x5.npz"), x_check=_check(X), y=Y, offsets=lay.offsets)
    print("ragged", time.time() - t0)

    # c2: 16x16, sampled rows
    lay = wl.loop_array(16, 16)
    A = AIMArray([em], lay.type_of, lay.offsets, params, K0, blocks=blocks, rows_only=True)
    x = wl.random_cvec(A.n, 1, 7)
    g = wl.rng(1, 9)
    rows = np.unique(np.concatenate([np.arange(8), A.n - 8 + np.arange(8), g.choice(A.n, 48, replace=False)]))
    yr = A.matvec_rows(x, rows)
    np.savez_compressed(os.path.join(HERE, "c2_16x16.npz"), x_check=_check(x), rows=rows, y_rows=yr)
    print("c2", time.time() - t0)

    # c3 family: four element types, 64 right-hand sides (a 6x6 instance)
    outers = (0.30, 0.34, 0.38, 0.42)
    lay = wl.loop_array(6, 6, outers=outers, config_index=2)
    ems = [build_element(et.scatterer.xyz, et.scatterer.tri, et.equiv.xyz, et.equiv.tri, K0) for et in lay.types]
    print("c3 elements", time.time() - t0)
    A = AIMArray(ems, lay.type_of, lay.offsets, params, K0, rows_only=True)
    X = wl.random_cvec(A.n, 2, 7, nrhs=64)
    g = wl.rng(2, 9)
    rows = np.unique(np.concatenate([np.arange(4), A.n - 4 + np.arange(4), g.choice(A.n, 40, replace=False)]))
    G = A.near_field_rows(rows)
    Y = np.zeros((len(rows), 64), dtype=np.complex128)
    for j in range(64):
        u = A.macro(X[:, j])
        Y[:, j] = A.dapply(X[:, j], rows) - (A.far(u, rows) + G @ u)
    th, ph, pol = wl.planewave_grid()
    Vr = np.zeros((len(rows), 64), dtype=np.complex128)
    for e in np.unique(A.elem_of[rows]):
        sel = np.where(A.elem_of[rows] == e)[0]
        Ve = excitation(translated_rwg(ems[lay.type_of[e]].rwg_e, lay.offsets[e]), th, ph, pol, K0)
        Vr[sel] = Ve[rows[sel] - A.off[e]]
    np.savez_compressed(os.path.join(HERE, "c3_types_6x6.npz"), x_check=_check(X), rows=rows, y_rows=Y, V_rows=Vr,
                        type_of=lay.type_of)
    print("c3", time.time() - t0)


def multiscale():
    t0 = time.time()
    et = wl.multiscale_element(meander=wl.MEANDER_REDUCED, box_div=wl.MEANDER_REDUCED_BOX)
    em = build_element(et.scatterer.xyz, et.scatterer.tri, et.equiv.xyz, et.equiv.tri, K0)
    print("multiscale element", time.time() - t0)
    lay = wl.multiscale_array(2, 2, meander=wl.MEANDER_REDUCED, box_div=wl.MEANDER_REDUCED_BOX)
    A = AIMArray([em], lay.type_of, lay.offsets, AIMParams(H, ORDER, NNF, wl.DEFAULT_GRID_PHASE), K0)
    X = wl.random_cvec(A.n, 3, 7, nrhs=8)
    Y = np.stack([A.matvec(np.ascontiguousarray(X[:, j])) for j in range(8)], axis=1)
    V = np.concatenate([excitation(translated_rwg(em.rwg_e, o), 0.0, 0.0, 0, K0)[:, 0] for o in lay.offsets])
    E, it, hist = gmres(A.matvec, V, tol=1e-12, restart=200, max_iter=2000)
    print("gmres", it, hist[-1])
    np.savez_compressed(os.path.join(HERE, "c4_meander_2x2.npz"), x_check=_check(X), y=Y, V=V, E=E)
    print("c4", time.time() - t0)


def extra():
    """Solutions and post-processing for the end-to-end tests (oracle only)."""
    t0 = time.time()
    params = AIMParams(H, ORDER, NNF, wl.DEFAULT_GRID_PHASE)
    # c3 family 6x6: the solutions of two incidences of the 8 x 8 grid
    outers = (0.30, 0.34, 0.38, 0.42)
    lay = wl.loop_array(6, 6, outers=outers, config_index=2)
    ems = [build_element(et.scatterer.xyz, et.scatterer.tri, et.equiv.xyz, et.equiv.tri, K0) for et in lay.types]
    A = AIMArray(ems, lay.type_of, lay.offsets, params, K0)
    th, ph, pol = wl.planewave_grid()
    cols = np.array([0, 37])
    V = np.zeros((A.n, len(cols)), dtype=np.complex128)
    for e in range(len(lay.offsets)):
        Ve = excitation(translated_rwg(ems[lay.type_of[e]].rwg_e, lay.offsets[e]), th[cols], ph[cols], pol[cols], K0)
        V[A.off[e]:A.off[e + 1]] = Ve
    E = np.zeros_like(V)
    for j in range(len(cols)):
        E[:, j], it, hist = gmres(A.matvec, V[:, j], tol=1e-11, restart=200, max_iter=4000)
        print("c3 column", cols[j], "iterations", it, hist[-1])
    np.savez_compressed(os.path.join(HERE, "c3_solve_6x6.npz"), cols=cols, V=V, E=E, type_of=lay.type_of)
    print("c3 solve", time.time() - t0)

    # reduced multiscale 2x2: currents and far field of the stored solution
    et = wl.multiscale_element(meander=wl.MEANDER_REDUCED, box_div=wl.MEANDER_REDUCED_BOX)
    em = build_element(et.scatterer.xyz, et.scatterer.tri, et.equiv.xyz, et.equiv.tri, K0)
    lay = wl.multiscale_array(2, 2, meander=wl.MEANDER_REDUCED, box_div=wl.MEANDER_REDUCED_BOX)
    g = np.load(os.path.join(HERE, "c4_meander_2x2.npz"))
    E = g["E"]
    nh = em.rwg_e.n
    JJ = [em.currents(E[e * nh:(e + 1) * nh]) for e in range(len(lay.offsets))]
    J = np.concatenate([c[0] for c in JJ])
    Jh = np.concatenate([c[1] for c in JJ])
    xyz, tri = merge_meshes([lay.types[0].equiv.translated(o) for o in lay.offsets])
    rw = build_rwg(xyz, tri)
    thd = np.deg2rad(np.concatenate([np.arange(0, 181, 10.0), np.arange(0, 181, 10.0)]))
    phd = np.deg2rad(np.concatenate([np.zeros(19), np.full(19, 90.0)]))
    F = far_field(rw, Jh, thd, phd, K0)
    np.savez_compressed(os.path.join(HERE, "c4_meander_2x2_post.npz"), J=J, Jhat=Jh, theta=thd, phi=phd, F=F,
                        sigma=rcs(F))
    print("c4 post", time.time() - t0)

    # the full multiscale element (2,547 scatterer RWG, 8x8x2 box) on a 2x1 array:
    # the product of two right-hand sides, every entry
    et = wl.multiscale_element()
    em = build_element(et.scatterer.xyz, et.scatterer.tri, et.equiv.xyz, et.equiv.tri, K0)
    print("full multiscale element", time.time() - t0)
    lay = wl.multiscale_array(2, 1)
    A = AIMArray([em], lay.type_of, lay.offsets, params, K0)
    X = wl.random_cvec(A.n, 3, 11, nrhs=2)
    Y = np.stack([A.matvec(np.ascontiguousarray(X[:, j])) for j in range(2)], axis=1)
    np.savez_compressed(os.path.join(HERE, "c4_full_element_2x1.npz"), x_check=_check(X), y=Y,
                        n_scat=em.rwg_s.n if hasattr(em, "rwg_s") else -1)
    print("c4 full element", time.time() - t0)


def drive():
    """Driven elements and the ground plane (oracle/drive.py), on 2x2 arrays."""
    from oracle import drive as dr
    t0 = time.time()
    params = AIMParams(H, ORDER, NNF, wl.DEFAULT_GRID_PHASE)
    # fed loops: two excitations (all elements at 1 V; element 0 at 1 V and element 2 at 0.5j V)
    lay = wl.fed_loop_array(2, 2)
    et = lay.types[0]
    em = build_element(et.scatterer.xyz, et.scatterer.tri, et.equiv.xyz, et.equiv.tri, K0)
    gap, d = lay.extra["gap"], lay.extra["direction"]
    f = dr.feed_vector(em.rwg_s, gap, d, 1.0)
    Jf, Jhf = dr.element_feed(em, f)
    A = AIMArray([em], lay.type_of, lay.offsets, params, K0)
    volts = np.zeros((4, 2), dtype=np.complex128)
    volts[:, 0] = 1.0
    volts[0, 1], volts[2, 1] = 1.0, 0.5j
    nh, ns = em.rwg_e.n, em.rwg_s.n
    V = np.zeros((A.n, 2), dtype=np.complex128)
    E = np.zeros_like(V)
    J = np.zeros((4 * ns, 2), dtype=np.complex128)
    Jh = np.zeros_like(V)
    Ip = np.zeros((4, 2), dtype=np.complex128)
    for j in range(2):
        u = np.concatenate([Jhf * volts[e, j] for e in range(4)])
        V[:, j] = -A.gapply(u)
        E[:, j], it, hist = gmres(A.matvec, V[:, j], tol=1e-12, restart=100, max_iter=2000)
        for e in range(4):
            Je, Jhe = dr.driven_currents(em, E[e * nh:(e + 1) * nh, j], Jf * volts[e, j])
            J[e * ns:(e + 1) * ns, j] = Je
            Jh[e * nh:(e + 1) * nh, j] = Jhe
            Ip[e, j] = dr.port_current(em.rwg_s, Je, gap, d)
        print("fed column", j, "iterations", it, hist[-1])
    np.savez_compressed(os.path.join(HERE, "fed_2x2.npz"), volts=volts, V=V, E=E, J=J, Jhat=Jh, port_current=Ip,
                        gap=gap, direction=np.asarray(d))
    print("fed", time.time() - t0)
    # 2x2 loops over a PEC plane z = -0.1 (8 elements with the images), two incidences
    zg = -0.1
    base = wl.loop_array(2, 2)
    lay = wl.ground_plane_array(base, zg)
    et = base.types[0]
    em = build_element(et.scatterer.xyz, et.scatterer.tri, et.equiv.xyz, et.equiv.tri, K0)
    A = AIMArray([em], lay.type_of, lay.offsets, params, K0)
    th = np.array([0.5, 0.3]); ph = np.array([0.35, 1.0]); pol = np.array([0, 1])
    V = np.concatenate([dr.ground_excitation(translated_rwg(em.rwg_e, o), th, ph, pol, K0, zg) for o in lay.offsets])
    E = np.zeros_like(V)
    for j in range(2):
        E[:, j], it, hist = gmres(A.matvec, V[:, j], tol=1e-12, restart=100, max_iter=2000)
        print("ground column", j, "iterations", it, hist[-1])
    nh = em.rwg_e.n
    Jh = np.concatenate([np.stack([em.currents(E[e * nh:(e + 1) * nh, j])[1] for j in range(2)], axis=1)
                         for e in range(lay.n_elem)])
    xyz, tri = merge_meshes([et.equiv.translated(o) for o in lay.offsets])
    rw = build_rwg(xyz, tri)
    thd = np.deg2rad(np.concatenate([np.arange(0, 91, 10.0), np.arange(0, 91, 10.0)]))
    phd = np.deg2rad(np.concatenate([np.zeros(10), np.full(10, 90.0)]))
    sig = np.stack([rcs(far_field(rw, Jh[:, j], thd, phd, K0)) for j in range(2)], axis=1)
    np.savez_compressed(os.path.join(HERE, "ground_2x2.npz"), z_ground=zg, theta=th, phi=ph, pol=pol, V=V, E=E,
                        theta_ff=thd, phi_ff=phd, sigma=sig, offsets=lay.offsets)
    print("ground", time.time() - t0)


if __name__ == "__main__":
    if sys.argv[1:] == ["c4"]:
        multiscale()
    elif sys.argv[1:] == ["extra"]:
        extra()
    elif sys.argv[1:] == ["drive"]:
        drive()
    else:
        main()
        multiscale()
        extra()
        drive()
