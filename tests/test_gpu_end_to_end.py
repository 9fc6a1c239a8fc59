"""End to end on the GPU against the oracle: the mixed-precision solve (complex64,
BF16 or FP16 operator inside GMRES, FP64 Arnoldi and refinement) to the 2x2
configuration's tolerance 1e-6, then the currents J = -A^-1 B E^ and
J^ = T J (eq. (JABE), eq. (Tm1)) and the bistatic RCS of J^ (Sec. VI).

Bars (the stated solution tolerances): E^, J and J^ within 1e-4 relative L2 of
the oracle's 1e-12 solution and its currents; RCS within 0.05 dB wherever sigma
is within 40 dB of its maximum, and within 1e-4 of the maximum elsewhere.  The
expected values come from tests/golden/make_golden.py (oracle only)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1712_02443_gb300 as mm  # noqa: E402
from paper_1712_02443_gb300 import workloads as wl  # noqa: E402
from paper_1712_02443_gb300.arrays import loop_array, multiscale_array  # noqa: E402

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
C3_OUTERS = (0.30, 0.34, 0.38, 0.42)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _rcs_ok(sig, ref):
    top = ref >= ref.max() * 1e-4
    db = np.abs(10 * np.log10(sig[top] / ref[top])).max()
    lin = np.abs(sig[~top] - ref[~top]).max() / ref.max() if (~top).any() else 0.0
    assert db <= 0.05 and lin <= 1e-4, (db, lin)
    return db


@pytest.fixture(scope="module")
def ctx():
    from paper_1712_02443_gb300.build import build
    build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = mm.mm_ctx_create(0)
    yield c
    mm.mm_ctx_destroy(c)


def _solve_post(la, V, prec, theta, phi, precond=0, inner_tol=1e-3):
    Vd = torch.from_numpy(np.ascontiguousarray(V)).cuda()
    E = torch.empty_like(Vd)
    st = mm.mm_solve(la.array, 1, Vd, E, tol=1e-6, restart=50, max_iter=3000, precision=prec, refine=1,
                     inner_tol=inner_tol, precond=precond)
    assert st["converged"] and st["rel_residual"] <= 1e-6
    J = torch.empty(la.info["n_scat_unknowns"], dtype=torch.complex128, device="cuda")
    Jh = torch.empty_like(E)
    mm.mm_currents(la.array, 1, E, J, Jh, torch.cuda.current_stream())
    torch.cuda.synchronize()
    sig = mm.mm_rcs(la.array, 1, Jh, theta, phi)[:, 0]
    return E.cpu().numpy(), J.cpu().numpy(), Jh.cpu().numpy(), sig


@pytest.mark.parametrize("prec,precond", [(mm.MM_C64, 0), (mm.MM_C64_F16, 1), (mm.MM_C64_BF16, 1)])
def test_c1_solve_currents_rcs(ctx, prec, precond):
    g = np.load(os.path.join(GOLD, "c1_2x2.npz"))
    la = loop_array(ctx, 2, 2)
    try:
        E, J, Jh, sig = _solve_post(la, g["V"], prec, g["theta"], g["phi"], precond,
                                    inner_tol=1e-5 if prec == mm.MM_C64 else 1e-3)
    finally:
        la.close()
    assert _rel(E, g["E"]) <= 1e-4
    assert _rel(J, g["J"]) <= 1e-4
    assert _rel(Jh, g["Jhat"]) <= 1e-4
    _rcs_ok(sig, g["sigma"])


@pytest.mark.parametrize("prec", [mm.MM_C64_F16, mm.MM_C64_BF16, mm.MM_C64])
def test_multiscale_solve_currents_rcs(ctx, prec):
    """The reduced multiscale element (loop + meander, 535 scatterer RWG) on a 2x2 array."""
    g = np.load(os.path.join(GOLD, "c4_meander_2x2.npz"))
    gp = np.load(os.path.join(GOLD, "c4_meander_2x2_post.npz"))
    la = multiscale_array(ctx, 2, 2, meander=wl.MEANDER_REDUCED, box_div=wl.MEANDER_REDUCED_BOX)
    try:
        E, J, Jh, sig = _solve_post(la, g["V"], prec, gp["theta"], gp["phi"], precond=1,
                                    inner_tol=1e-5 if prec == mm.MM_C64 else 1e-3)
    finally:
        la.close()
    assert _rel(E, g["E"]) <= 1e-4
    assert _rel(J, gp["J"]) <= 1e-4
    assert _rel(Jh, gp["Jhat"]) <= 1e-4
    _rcs_ok(sig, gp["sigma"])


def test_c3_batch_alone_and_oracle(ctx):
    """64 incidences solved together to 1e-6 (independent Krylov spaces, one
    product per iteration): columns 0 and 37 agree with the same columns solved
    alone and with the oracle's solutions, all within 1e-4."""
    g = np.load(os.path.join(GOLD, "c3_solve_6x6.npz"))
    la = loop_array(ctx, 6, 6, outers=C3_OUTERS, config_index=2)
    try:
        assert np.array_equal(la.layout.type_of, g["type_of"])
        th, ph, pol = wl.planewave_grid()
        st = torch.cuda.current_stream()
        V = torch.empty(la.n * 64, dtype=torch.complex128, device="cuda")
        mm.mm_rhs_planewave(la.array, th, ph, pol, V, mm.MM_C128, st)
        E = torch.empty_like(V)
        s = mm.mm_solve(la.array, 64, V, E, tol=1e-6, restart=50, max_iter=4000, precision=mm.MM_C64, refine=1,
                        inner_tol=1e-5, precond=1, stream=st)
        assert s["converged"] and s["rel_residual"] <= 1e-6
        Eb = E.cpu().numpy().reshape(la.n, 64)
        Vb = V.cpu().numpy().reshape(la.n, 64)
        for k, j in enumerate(g["cols"]):
            assert _rel(Vb[:, j], g["V"][:, k]) <= 1e-12
            V1 = torch.from_numpy(np.ascontiguousarray(g["V"][:, k])).cuda()
            E1 = torch.empty_like(V1)
            s1 = mm.mm_solve(la.array, 1, V1, E1, tol=1e-6, restart=50, max_iter=4000, precision=mm.MM_C64,
                             refine=1, inner_tol=1e-5, precond=1, stream=st)
            assert s1["converged"]
            e1 = E1.cpu().numpy()
            assert _rel(Eb[:, j], e1) <= 1e-4
            assert _rel(e1, g["E"][:, k]) <= 1e-4
            assert _rel(Eb[:, j], g["E"][:, k]) <= 1e-4
    finally:
        la.close()


@pytest.mark.parametrize("prec", [mm.MM_C128, mm.MM_C64])
def test_full_multiscale_element_product(ctx, prec):
    """The full multiscale element (2,547 scatterer RWG, 576-RWG box) on a 2x1
    array, two right-hand sides, every entry of the product vs the oracle."""
    g = np.load(os.path.join(GOLD, "c4_full_element_2x1.npz"))
    la = multiscale_array(ctx, 2, 1)
    try:
        X = wl.random_cvec(la.n, 3, 11, nrhs=2)
        assert np.allclose([X.sum(), (np.abs(X) ** 2).sum()], g["x_check"])
        dt = torch.complex128 if prec == mm.MM_C128 else torch.complex64
        xd = torch.from_numpy(np.ascontiguousarray(X)).to(dt).cuda()
        yd = torch.empty_like(xd)
        mm.mm_apply(la.array, 2, xd, yd, prec, torch.cuda.current_stream())
        torch.cuda.synchronize()
        Y = yd.cpu().numpy().astype(np.complex128)
    finally:
        la.close()
    assert _rel(Y, g["y"]) <= (1e-11 if prec == mm.MM_C128 else 1e-5)
