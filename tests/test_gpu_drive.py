"""Driven elements (delta-gap feeds) and the PEC ground plane (image theory) on
the GPU against the oracle (tests/golden, written by oracle/drive.py through
make_golden.py).

Bars: excitations in complex128 to rounding (relative L2 <= 1e-10; the
library forms the ground-plane excitation as two plane waves in closed form,
the oracle by evaluating the incident field plus its image at the quadrature
points); complex64 excitation 1e-5; mixed-precision solves to 1e-6 within
1e-4 of the oracle's 1e-12 solutions, as are the currents and the port
currents; RCS within 0.05 dB where it is within 40 dB of its maximum."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1712_02443_gb300 as mm  # noqa: E402
from paper_1712_02443_gb300 import workloads as wl  # noqa: E402
from paper_1712_02443_gb300.arrays import build_types  # noqa: E402

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
K0 = 2.0 * np.pi


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def ctx():
    from paper_1712_02443_gb300.build import build
    build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = mm.mm_ctx_create(0)
    yield c
    mm.mm_ctx_destroy(c)


@pytest.fixture(scope="module")
def fed(ctx):
    lay = wl.fed_loop_array(2, 2)
    meshes, types = build_types(ctx, lay)
    mm.mm_type_set_feed(types[0], lay.extra["gap"], lay.extra["direction"])
    arr = mm.mm_array_create(ctx, [types[0]] * 4, lay.offsets, 0.1, 2, 3, wl.DEFAULT_GRID_PHASE)
    yield arr, lay
    mm.mm_array_destroy(arr)
    for t in types:
        mm.mm_type_destroy(t)
    for m in meshes:
        mm.mm_mesh_destroy(m)


def test_deltagap_excitation(fed):
    arr, lay = fed
    g = np.load(os.path.join(GOLD, "fed_2x2.npz"))
    n = mm.mm_array_info_get(arr)["n_unknowns"]
    V = torch.empty(n * 2, dtype=torch.complex128, device="cuda")
    mm.mm_rhs_deltagap(arr, g["volts"], V, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert _rel(V.cpu().numpy().reshape(n, 2), g["V"]) <= 1e-10


@pytest.mark.parametrize("prec", [mm.MM_C64, mm.MM_C64_F16])
def test_driven_solve_currents_ports(fed, prec):
    arr, lay = fed
    g = np.load(os.path.join(GOLD, "fed_2x2.npz"))
    info = mm.mm_array_info_get(arr)
    n, ns = info["n_unknowns"], info["n_scat_unknowns"]
    st = torch.cuda.current_stream()
    V = torch.empty(n * 2, dtype=torch.complex128, device="cuda")
    mm.mm_rhs_deltagap(arr, g["volts"], V, st)
    E = torch.empty_like(V)
    s = mm.mm_solve(arr, 2, V, E, tol=1e-6, restart=50, max_iter=2000, precision=prec, refine=1,
                    inner_tol=1e-5 if prec == mm.MM_C64 else 1e-3, precond=1, stream=st)
    assert s["converged"] and s["rel_residual"] <= 1e-6
    J = torch.empty(ns * 2, dtype=torch.complex128, device="cuda")
    Jh = torch.empty_like(E)
    mm.mm_currents_fed(arr, 2, E, g["volts"], J, Jh, st)
    torch.cuda.synchronize()
    assert _rel(E.cpu().numpy().reshape(n, 2), g["E"]) <= 1e-4
    Jg = J.cpu().numpy().reshape(ns, 2)
    assert _rel(Jg, g["J"]) <= 1e-4
    assert _rel(Jh.cpu().numpy().reshape(n, 2), g["Jhat"]) <= 1e-4
    # port currents through each element's gap: sum_g s_g J_g l_g
    from oracle.basis import build_rwg
    from oracle.drive import port_current
    et = lay.types[0]
    r = build_rwg(et.scatterer.xyz, et.scatterer.tri)
    per = ns // 4
    Ip = np.array([port_current(r, Jg[e * per:(e + 1) * per], g["gap"], g["direction"]) for e in range(4)])
    assert _rel(Ip, g["port_current"]) <= 1e-4


def test_deltagap_needs_a_feed(ctx):
    lay = wl.loop_array(2, 1)
    meshes, types = build_types(ctx, lay)
    arr = mm.mm_array_create(ctx, [types[0]] * 2, lay.offsets, 0.1, 2, 3, wl.DEFAULT_GRID_PHASE)
    try:
        V = torch.empty(mm.mm_array_info_get(arr)["n_unknowns"], dtype=torch.complex128, device="cuda")
        with pytest.raises(mm.MacroAIMError) as e:
            mm.mm_rhs_deltagap(arr, np.ones((2, 1)), V)
        assert e.value.status == mm.MM_EINVAL
    finally:
        mm.mm_array_destroy(arr)
        for t in types:
            mm.mm_type_destroy(t)
        for m in meshes:
            mm.mm_mesh_destroy(m)


@pytest.fixture(scope="module")
def ground(ctx):
    g = np.load(os.path.join(GOLD, "ground_2x2.npz"))
    base = wl.loop_array(2, 2)
    lay = wl.ground_plane_array(base, float(g["z_ground"]))
    assert np.allclose(lay.offsets, g["offsets"])
    meshes, types = build_types(ctx, base)
    arr = mm.mm_array_create(ctx, [types[0]] * lay.n_elem, lay.offsets, 0.1, 2, 3, wl.DEFAULT_GRID_PHASE)
    yield arr, g
    mm.mm_array_destroy(arr)
    for t in types:
        mm.mm_type_destroy(t)
    for m in meshes:
        mm.mm_mesh_destroy(m)


@pytest.mark.parametrize("prec", [mm.MM_C128, mm.MM_C64])
def test_ground_plane_excitation(ground, prec):
    arr, g = ground
    n = mm.mm_array_info_get(arr)["n_unknowns"]
    dt = torch.complex128 if prec == mm.MM_C128 else torch.complex64
    V = torch.empty(n * 2, dtype=dt, device="cuda")
    mm.mm_rhs_planewave_ground(arr, g["theta"], g["phi"], g["pol"], float(g["z_ground"]), V, prec,
                               torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert _rel(V.cpu().numpy().astype(np.complex128).reshape(n, 2), g["V"]) <= (1e-10 if prec == mm.MM_C128 else 1e-5)


def test_ground_plane_solve_and_rcs(ground):
    arr, g = ground
    n = mm.mm_array_info_get(arr)["n_unknowns"]
    st = torch.cuda.current_stream()
    V = torch.empty(n * 2, dtype=torch.complex128, device="cuda")
    mm.mm_rhs_planewave_ground(arr, g["theta"], g["phi"], g["pol"], float(g["z_ground"]), V, mm.MM_C128, st)
    E = torch.empty_like(V)
    s = mm.mm_solve(arr, 2, V, E, tol=1e-6, restart=50, max_iter=2000, precision=mm.MM_C64, refine=1,
                    inner_tol=1e-5, precond=1, stream=st)
    assert s["converged"]
    assert _rel(E.cpu().numpy().reshape(n, 2), g["E"]) <= 1e-4
    Jh = torch.empty_like(E)
    mm.mm_currents(arr, 2, E, None, Jh, st)
    torch.cuda.synchronize()
    sig = mm.mm_rcs(arr, 2, Jh, g["theta_ff"], g["phi_ff"])
    for j in range(2):
        ref = g["sigma"][:, j]
        top = ref >= ref.max() * 1e-4
        assert np.abs(10 * np.log10(sig[top, j] / ref[top])).max() <= 0.05
