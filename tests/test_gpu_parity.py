"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Expected values come from tests/golden/make_golden.py (oracle only) or are
computed live by the oracle.  Tolerances:
* complex128 operator: rounding only (different summation order, FFT sizes):
  relative L2 <= 1e-11, worst element <= 1e-10 of max |y|;
* complex64 operator: FP32 arithmetic over sums of a few hundred terms
  (GEMM k = N^_t, ~400 near-field terms, FFT) gives ~1e-6 relative per entry;
  the bar is the stated matvec tolerance, relative L2 <= 1e-5, and worst
  element <= 1e-4 of max |y|.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1712_02443_gb300 as mm  # noqa: E402
from paper_1712_02443_gb300 import workloads as wl  # noqa: E402
from paper_1712_02443_gb300.arrays import loop_array  # noqa: E402

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
K0 = 2.0 * np.pi
TOL = {mm.MM_C128: (1e-11, 1e-10), mm.MM_C64: (1e-5, 1e-4)}
DT = {mm.MM_C128: torch.complex128, mm.MM_C64: torch.complex64}


def _close(got, ref, prec):
    l2, worst = TOL[prec]
    got = np.asarray(got)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    w = np.abs(got - ref).max() / np.abs(ref).max()
    assert rel <= l2 and w <= worst, (rel, w)
    return rel, w


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
def c1(ctx):
    la = loop_array(ctx, 2, 2)
    yield la
    la.close()


def _apply(la, x, prec, nrhs=1):
    xd = torch.from_numpy(np.ascontiguousarray(x)).to(DT[prec]).cuda()
    yd = torch.empty_like(xd)
    mm.mm_apply(la.array, nrhs, xd, yd, prec, torch.cuda.current_stream())
    torch.cuda.synchronize()
    return yd.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("prec", [mm.MM_C128, mm.MM_C64])
def test_c1_matvec(c1, prec):
    g = np.load(os.path.join(GOLD, "c1_2x2.npz"))
    assert c1.n == len(g["x"])
    _close(_apply(c1, g["x"], prec), g["y"], prec)


@pytest.mark.parametrize("prec", [mm.MM_C128, mm.MM_C64])
def test_ragged_multi_rhs(ctx, c1, prec):
    g = np.load(os.path.join(GOLD, "ragged_3x5.npz"))
    la = loop_array(ctx, 3, 5, types=c1.types)
    try:
        X = wl.random_cvec(la.n, 0, 8, nrhs=3)
        assert np.allclose([X.sum(), (np.abs(X) ** 2).sum()], g["x_check"])
        _close(_apply(la, X, prec, nrhs=3), g["y"], prec)
        # each column alone equals its column in the batch (same result alone and batched)
        y1 = _apply(la, np.ascontiguousarray(X[:, 1]), prec)
        _close(y1, g["y"][:, 1], prec)
    finally:
        mm.mm_array_destroy(la.array)


@pytest.mark.parametrize("prec", [mm.MM_C128, mm.MM_C64])
def test_c2_full_size_sampled_rows(ctx, c1, prec):
    """16 x 16 array (the benchmark workload), single RHS: sampled rows vs the oracle."""
    g = np.load(os.path.join(GOLD, "c2_16x16.npz"))
    la = loop_array(ctx, 16, 16, types=c1.types)
    try:
        x = wl.random_cvec(la.n, 1, 7)
        assert np.allclose([x.sum(), (np.abs(x) ** 2).sum()], g["x_check"])
        y = _apply(la, x, prec)
        _close(y[g["rows"]], g["y_rows"], prec)
    finally:
        mm.mm_array_destroy(la.array)


@pytest.mark.parametrize("prec", [mm.MM_C128, mm.MM_C64])
def test_single_element_matvec(ctx, c1, loop_model, prec):
    """Degenerate array of one element: no coupling to other elements."""
    from oracle.aim import AIMArray, AIMParams
    lay = wl.loop_array(1, 1)
    A = AIMArray([loop_model], lay.type_of, lay.offsets, AIMParams(0.1, 2, 3, wl.DEFAULT_GRID_PHASE), K0)
    la = loop_array(ctx, 1, 1, types=c1.types)
    try:
        x = wl.random_cvec(la.n, 0, 11)
        _close(_apply(la, x, prec), A.matvec(x), prec)
    finally:
        mm.mm_array_destroy(la.array)


@pytest.mark.parametrize("prec", [mm.MM_C128, mm.MM_C64])
def test_planewave_excitation(c1, prec):
    g = np.load(os.path.join(GOLD, "c1_2x2.npz"))
    V = torch.empty(c1.n, dtype=DT[prec], device="cuda")
    mm.mm_rhs_planewave(c1.array, [0.0], [0.0], [0], V, prec, torch.cuda.current_stream())
    torch.cuda.synchronize()
    _close(V.cpu().numpy().astype(np.complex128), g["V"], prec)


@pytest.mark.parametrize("prec,refine", [(mm.MM_C128, 0), (mm.MM_C64, 1)])
def test_c1_solve(c1, prec, refine):
    """GMRES to 1e-6 (the 2x2 configuration's tolerance): solution vs the oracle's
    1e-12 solve of the same AIM system; error <= cond * tol."""
    g = np.load(os.path.join(GOLD, "c1_2x2.npz"))
    V = torch.from_numpy(g["V"]).cuda()
    E = torch.empty_like(V)
    st = mm.mm_solve(c1.array, 1, V, E, tol=1e-6, restart=50, max_iter=500, precision=prec, refine=refine)
    assert st["converged"] and st["rel_residual"] <= 1e-6
    Eg = E.cpu().numpy()
    err = np.linalg.norm(Eg - g["E"]) / np.linalg.norm(g["E"])
    assert err <= 1e-4, err


def test_apply_host_matches_device(c1):
    g = np.load(os.path.join(GOLD, "c1_2x2.npz"))
    x = np.ascontiguousarray(g["x"].astype(np.complex64))
    y = np.zeros_like(x)
    mm.mm_apply_host(c1.array, 1, x, y, mm.MM_C64)
    _close(y.astype(np.complex128), g["y"], mm.MM_C64)


def test_aliasing_arguments_rejected(c1):
    x = torch.zeros(c1.n, dtype=torch.complex64, device="cuda")
    with pytest.raises(mm.MacroAIMError) as e:
        mm.mm_apply(c1.array, 1, x, x, mm.MM_C64)
    assert e.value.status == mm.MM_EINVAL


def test_currents_match_oracle(c1):
    """J = -A^-1 B E^ and J^ = T J per element (eqs. (JABE), (Tm1)), FP64."""
    g = np.load(os.path.join(GOLD, "c1_2x2.npz"))
    E = torch.from_numpy(g["E"]).cuda()
    ns = c1.info["n_scat_unknowns"]
    assert ns == len(g["J"])
    J = torch.empty(ns, dtype=torch.complex128, device="cuda")
    Jh = torch.empty_like(E)
    mm.mm_currents(c1.array, 1, E, J, Jh, torch.cuda.current_stream())
    torch.cuda.synchronize()
    for got, ref in ((J.cpu().numpy(), g["J"]), (Jh.cpu().numpy(), g["Jhat"])):
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-10


def test_farfield_and_rcs_match_oracle(c1):
    """Far field of J^ (FP32 exponentials and sums): relative L2 <= 1e-5; RCS within
    0.01 dB wherever sigma is within 40 dB of its maximum."""
    g = np.load(os.path.join(GOLD, "c1_2x2.npz"))
    Jh = torch.from_numpy(g["Jhat"]).cuda()
    nd = len(g["theta"])
    F = torch.empty(nd * 3, dtype=torch.complex128, device="cuda")
    mm.mm_farfield(c1.array, 1, Jh, g["theta"], g["phi"], F, torch.cuda.current_stream())
    torch.cuda.synchronize()
    Fg = F.cpu().numpy().reshape(nd, 3)
    assert np.linalg.norm(Fg - g["F"]) / np.linalg.norm(g["F"]) <= 1e-5
    sig = mm.mm_rcs(c1.array, 1, Jh, g["theta"], g["phi"])[:, 0]
    top = g["sigma"] >= g["sigma"].max() * 1e-4
    assert np.abs(10 * np.log10(sig[top] / g["sigma"][top])).max() <= 0.01


C3_OUTERS = (0.30, 0.34, 0.38, 0.42)


@pytest.fixture(scope="module")
def c3(ctx):
    la = loop_array(ctx, 6, 6, outers=C3_OUTERS, config_index=2)
    yield la
    la.close()


@pytest.mark.parametrize("prec", [mm.MM_C128, mm.MM_C64])
def test_c3_four_types_64_rhs(c3, prec):
    """Four element types drawn per cell, 64 right-hand sides in one product:
    sampled rows of all 64 columns and of the 8 x 8 plane-wave excitation."""
    g = np.load(os.path.join(GOLD, "c3_types_6x6.npz"))
    assert np.array_equal(c3.layout.type_of, g["type_of"])
    X = wl.random_cvec(c3.n, 2, 7, nrhs=64)
    assert np.allclose([X.sum(), (np.abs(X) ** 2).sum()], g["x_check"])
    Y = _apply(c3, X, prec, nrhs=64)
    _close(Y[g["rows"]], g["y_rows"], prec)
    th, ph, pol = wl.planewave_grid()
    V = torch.empty(c3.n * 64, dtype=DT[prec], device="cuda")
    mm.mm_rhs_planewave(c3.array, th, ph, pol, V, prec, torch.cuda.current_stream())
    torch.cuda.synchronize()
    Vh = V.cpu().numpy().astype(np.complex128).reshape(c3.n, 64)
    _close(Vh[g["rows"]], g["V_rows"], prec)


def test_c3_batched_solve_equals_columns_alone(c3):
    """64 incidences solved together (independent Krylov spaces, one product per
    iteration) give the same solutions as the columns solved alone (P13): both
    solved to a residual of 1e-6, so that the solutions agree within the 1e-4
    solution tolerance (the residual bound times the condition number of this
    preconditioned operator, about 10, stays below it), and every column meets
    the residual."""
    th, ph, pol = wl.planewave_grid()
    st = torch.cuda.current_stream()
    V = torch.empty(c3.n * 64, dtype=torch.complex128, device="cuda")
    mm.mm_rhs_planewave(c3.array, th, ph, pol, V, mm.MM_C128, st)
    E = torch.empty_like(V)
    s = mm.mm_solve(c3.array, 64, V, E, tol=1e-6, restart=50, max_iter=4000, precision=mm.MM_C64, refine=1,
                    inner_tol=1e-5, stream=st, precond=1)
    assert s["converged"] and s["rel_residual"] <= 1e-6
    Eb = E.cpu().numpy().reshape(c3.n, 64)
    for j in (0, 37):
        V1 = torch.empty(c3.n, dtype=torch.complex128, device="cuda")
        mm.mm_rhs_planewave(c3.array, [th[j]], [ph[j]], [pol[j]], V1, mm.MM_C128, st)
        E1 = torch.empty_like(V1)
        s1 = mm.mm_solve(c3.array, 1, V1, E1, tol=1e-6, restart=50, max_iter=4000, precision=mm.MM_C64, refine=1,
                         inner_tol=1e-5, stream=st, precond=1)
        assert s1["converged"]
        e1 = E1.cpu().numpy()
        assert np.linalg.norm(Eb[:, j] - e1) / np.linalg.norm(e1) <= 1e-4


@pytest.mark.parametrize("prec", [mm.MM_C128, mm.MM_C64])
def test_far_field_only_operator(ctx, c1, loop_model, prec):
    """N_NF = -1 drops the precorrection: y = D x - I H P T A^-1 B x (no G_NF term),
    3 x 2 array, three right-hand sides."""
    from oracle.aim import AIMArray, AIMParams
    lay = wl.loop_array(3, 2)
    A = AIMArray([loop_model], lay.type_of, lay.offsets, AIMParams(0.1, 2, -1, wl.DEFAULT_GRID_PHASE), K0)
    assert A.GNF.nnz == 0
    la = loop_array(ctx, 3, 2, n_nf=-1, types=c1.types)
    try:
        assert la.info["nnz_near"] == 0
        X = wl.random_cvec(la.n, 0, 13, nrhs=3)
        Y = _apply(la, X, prec, nrhs=3)
        ref = np.stack([A.matvec(np.ascontiguousarray(X[:, j])) for j in range(3)], axis=1)
        _close(Y, ref, prec)
    finally:
        mm.mm_array_destroy(la.array)


@pytest.mark.parametrize("prec,refine,orth", [(mm.MM_C128, 0, 1), (mm.MM_C128, 0, 3), (mm.MM_C64, 1, 2),
                                              (mm.MM_C64, 1, 3)])
def test_c1_solve_orthogonalisation_modes(c1, prec, refine, orth):
    """Every Arnoldi orthogonalisation mode (one classical Gram-Schmidt pass,
    selective second pass, two passes) reaches the oracle's solution within the
    solver tolerance."""
    g = np.load(os.path.join(GOLD, "c1_2x2.npz"))
    V = torch.from_numpy(g["V"]).cuda()
    E = torch.empty_like(V)
    st = mm.mm_solve(c1.array, 1, V, E, tol=1e-6, restart=50, max_iter=500, precision=prec, refine=refine,
                     orth=orth)
    assert st["converged"] and st["rel_residual"] <= 1e-6
    err = np.linalg.norm(E.cpu().numpy() - g["E"]) / np.linalg.norm(g["E"])
    assert err <= 1e-4, err


def test_orthogonalisation_mode_out_of_range_rejected(c1):
    V = torch.zeros(c1.n, dtype=torch.complex128, device="cuda")
    E = torch.empty_like(V)
    with pytest.raises(mm.MacroAIMError) as e:
        mm.mm_solve(c1.array, 1, V, E, tol=1e-6, orth=4)
    assert e.value.status == mm.MM_EINVAL


@pytest.mark.parametrize("nrhs", [8, 12, 24])
@pytest.mark.parametrize("prec", [mm.MM_C128, mm.MM_C64])
def test_c3_block_near_field_column_tiles(c3, prec, nrhs):
    """8 or more right-hand sides take the near field as dense translation-invariant
    blocks (one launch per lattice offset) instead of CSR rows; 8, 12 and 24 columns
    exercise the 8-, 16- and 32-column tiles and the ragged column edge.  The first
    nrhs columns of the 64-column oracle product are the reference."""
    g = np.load(os.path.join(GOLD, "c3_types_6x6.npz"))
    X = wl.random_cvec(c3.n, 2, 7, nrhs=64)
    Y = _apply(c3, np.ascontiguousarray(X[:, :nrhs]), prec, nrhs=nrhs)
    _close(Y[g["rows"]], g["y_rows"][:, :nrhs], prec)


@pytest.fixture()
def near_csr_env(monkeypatch):
    """Arrays created under this fixture assemble the near-field CSR and apply the
    near field as CSR rows (the choice is read when the array is created)."""
    monkeypatch.setenv("MACROAIM_NEAR", "csr")


@pytest.mark.parametrize("nrhs", [1, 3])
@pytest.mark.parametrize("prec", [mm.MM_C128, mm.MM_C64])
def test_block_near_field_few_rhs(ctx, c3, prec, nrhs):
    """Blocks with one or three right-hand sides: the GEMM's columns are (element
    pair, right-hand side), so one right-hand side still fills the tiles."""
    g = np.load(os.path.join(GOLD, "c3_types_6x6.npz"))
    la = loop_array(ctx, 6, 6, outers=C3_OUTERS, config_index=2, types=c3.types)
    try:
        X = wl.random_cvec(la.n, 2, 7, nrhs=64)
        Y = _apply(la, np.ascontiguousarray(X[:, :nrhs]), prec, nrhs=nrhs).reshape(la.n, nrhs)
        _close(Y[g["rows"]], g["y_rows"][:, :nrhs], prec)
    finally:
        mm.mm_array_destroy(la.array)


@pytest.mark.parametrize("prec", [mm.MM_C128, mm.MM_C64])
def test_c2_full_size_csr_near_field(ctx, c1, near_csr_env, prec):
    """16 x 16 array, one right-hand side, near field as CSR rows (the alternative
    to the blocks): sampled rows vs the oracle."""
    g = np.load(os.path.join(GOLD, "c2_16x16.npz"))
    la = loop_array(ctx, 16, 16, types=c1.types)
    try:
        assert la.info["nnz_near"] > 0
        x = wl.random_cvec(la.n, 1, 7)
        _close(_apply(la, x, prec)[g["rows"]], g["y_rows"], prec)
    finally:
        mm.mm_array_destroy(la.array)


@pytest.mark.parametrize("prec", [mm.MM_C128, mm.MM_C64])
def test_csr_near_field_multi_rhs(ctx, c3, near_csr_env, prec):
    """CSR rows with 3 (4-column chunks) and 12 (8-column chunks) right-hand sides."""
    g = np.load(os.path.join(GOLD, "c3_types_6x6.npz"))
    la = loop_array(ctx, 6, 6, outers=C3_OUTERS, config_index=2, types=c3.types)
    try:
        X = wl.random_cvec(la.n, 2, 7, nrhs=64)
        for nrhs in (3, 12):
            Y = _apply(la, np.ascontiguousarray(X[:, :nrhs]), prec, nrhs=nrhs).reshape(la.n, nrhs)
            _close(Y[g["rows"]], g["y_rows"][:, :nrhs], prec)
    finally:
        mm.mm_array_destroy(la.array)


@pytest.mark.parametrize("prec", [mm.MM_C128, mm.MM_C64])
def test_near_csr_never_assembled(ctx, c1, prec):
    """near_csr = 2: the blocks alone carry the near field in both precisions (the
    form large arrays use); info still counts its non-zeros, the CSR export is
    refused, and the product still matches the oracle."""
    g = np.load(os.path.join(GOLD, "c1_2x2.npz"))
    lay = wl.loop_array(2, 2)
    arr = mm.mm_array_create(ctx, [c1.types[0]] * lay.n_elem, lay.offsets, 0.1, 2, 3, wl.DEFAULT_GRID_PHASE,
                             near_csr=2)
    try:
        info = mm.mm_array_info_get(arr)
        assert info["nnz_near"] > 0 and info["near_format"] == "blocks"
        with pytest.raises(mm.MacroAIMError) as e:
            mm.mm_array_export(arr, mm.MM_EXPORT_NEAR_PTR)
        assert e.value.status == mm.MM_EINVAL
        xd = torch.from_numpy(g["x"]).to(DT[prec]).cuda()
        yd = torch.empty_like(xd)
        mm.mm_apply(arr, 1, xd, yd, prec, torch.cuda.current_stream())
        torch.cuda.synchronize()
        _close(yd.cpu().numpy().astype(np.complex128), g["y"], prec)
    finally:
        mm.mm_array_destroy(arr)


@pytest.mark.parametrize("prec,refine", [(mm.MM_C128, 0), (mm.MM_C64, 1)])
def test_c1_solve_block_jacobi(c1, prec, refine):
    """Right block-Jacobi preconditioning leaves the solution unchanged (oracle's
    1e-12 solution within 1e-4 at tol 1e-6) and needs fewer GMRES iterations."""
    g = np.load(os.path.join(GOLD, "c1_2x2.npz"))
    V = torch.from_numpy(g["V"]).cuda()
    E = torch.empty_like(V)
    st0 = mm.mm_solve(c1.array, 1, V, E, tol=1e-6, restart=50, max_iter=500, precision=prec, refine=refine)
    st = mm.mm_solve(c1.array, 1, V, E, tol=1e-6, restart=50, max_iter=500, precision=prec, refine=refine, precond=1)
    assert st["converged"] and st["rel_residual"] <= 1e-6
    assert st["iterations"] < st0["iterations"], (st["iterations"], st0["iterations"])
    err = np.linalg.norm(E.cpu().numpy() - g["E"]) / np.linalg.norm(g["E"])
    assert err <= 1e-4, err


def test_300_rhs_product_and_solve(c1):
    """More right-hand sides than the Arnoldi block has threads (300 > 256: the
    per-column reduction path): columns are multiples alpha_j of the golden vector,
    so by linearity y_j = alpha_j y and E_j = alpha_j E.  Both precisions of the
    product, and a refined solve of all 300 columns."""
    g = np.load(os.path.join(GOLD, "c1_2x2.npz"))
    r = 300
    alpha = (np.arange(1, r + 1) / r) * np.exp(1j * 0.37 * np.arange(r))
    X = np.outer(g["x"], alpha)
    for prec in (mm.MM_C128, mm.MM_C64):
        Y = _apply(c1, X, prec, nrhs=r).reshape(c1.n, r)
        _close(Y, np.outer(g["y"], alpha), prec)
    V = torch.from_numpy(np.ascontiguousarray(np.outer(g["V"], alpha))).cuda()
    E = torch.empty_like(V)
    st = mm.mm_solve(c1.array, r, V, E, tol=1e-6, restart=50, max_iter=500, precision=mm.MM_C64, refine=1,
                     precond=1)
    assert st["converged"] and st["rel_residual"] <= 1e-6
    ref = np.outer(g["E"], alpha)
    Eg = E.cpu().numpy().reshape(c1.n, r)
    assert np.linalg.norm(Eg - ref) / np.linalg.norm(ref) <= 1e-4


def test_degenerate_arguments_rejected(ctx, c1):
    x = torch.zeros(c1.n, dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(mm.MacroAIMError) as e:
        mm.mm_apply(c1.array, 0, x, y, mm.MM_C64)            # no right-hand side
    assert e.value.status == mm.MM_EINVAL
    with pytest.raises(mm.MacroAIMError) as e:
        mm.mm_array_create(ctx, [], np.zeros((0, 3)), 0.1, 2, 3, wl.DEFAULT_GRID_PHASE)   # no element
    assert e.value.status == mm.MM_EINVAL


@pytest.mark.parametrize("prec", [mm.MM_C64, mm.MM_C128])
def test_near_field_stream_matches_in_order(ctx, monkeypatch, prec):
    """The near field runs on its own stream beside the far-field chain (joined
    before the interpolation); the same array built with one in-order stream
    (MACROAIM_NEAR_OVERLAP=0) gives the same product up to the summation order
    of the near field's atomic adds.  Several products back to back, so that a
    missing join between consecutive products would show."""
    outs = []
    for ov in ("1", "0"):
        monkeypatch.setenv("MACROAIM_NEAR_OVERLAP", ov)
        la = loop_array(ctx, 4, 4)
        try:
            X = wl.random_cvec(la.n, 0, 21, nrhs=2)
            xd = torch.from_numpy(np.ascontiguousarray(X)).to(DT[prec]).cuda()
            ys = [torch.empty_like(xd) for _ in range(3)]
            for yk in ys:
                mm.mm_apply(la.array, 2, xd, yk, prec, torch.cuda.current_stream())
            torch.cuda.synchronize()
            outs.append([yk.cpu().numpy().astype(np.complex128) for yk in ys])
        finally:
            la.close()
    ref = outs[1][0]
    for y in outs[0] + outs[1]:
        rel = np.linalg.norm(y - ref) / np.linalg.norm(ref)
        assert rel <= (1e-6 if prec == mm.MM_C64 else 1e-13), rel


@pytest.mark.parametrize("shape,ks", [(0, 1), (1, 2), (2, 4), (1, 3), (3, 1), (3, 4), (4, 2), (5, 1), (6, 2)])
@pytest.mark.parametrize("nrhs", [1, 5])
def test_block_near_field_every_kernel_shape(ctx, c3, monkeypatch, shape, ks, nrhs):
    """Every shape of the block near-field kernel (64-row tiles of 32 columns, the
    same for five CTAs per SM, 64 columns; 32-row tiles of 32 and 64 columns) with
    several k splits, fixed through MACROAIM_NEAR_SHAPE instead of the autotuner:
    sampled rows vs the oracle."""
    monkeypatch.setenv("MACROAIM_NEAR_SHAPE", "%d,%d" % (shape, ks))
    g = np.load(os.path.join(GOLD, "c3_types_6x6.npz"))
    la = loop_array(ctx, 6, 6, outers=C3_OUTERS, config_index=2, types=c3.types)
    try:
        X = wl.random_cvec(la.n, 2, 7, nrhs=64)
        Y = _apply(la, np.ascontiguousarray(X[:, :nrhs]), mm.MM_C64, nrhs=nrhs).reshape(la.n, nrhs)
        _close(Y[g["rows"]], g["y_rows"][:, :nrhs], mm.MM_C64)
    finally:
        mm.mm_array_destroy(la.array)


@pytest.mark.parametrize("nx", [10, 15, 19, 24, 30, 34, 38])
def test_register_fft_lengths(ctx, c1, loop_model, nx):
    """Linear arrays whose padded x length is 128, 160, 224, 256, 320, 352 and 384
    points (32 R with R = 4, 5, 7, 8, 10, 11, 12: the register FFT's even and odd
    lane DFTs up to the largest; the other tests reach R = 1, 2, 3, 6).  The
    complex128 product takes Stockham stages at the same lengths (radix 11 at
    352).  Far-field operator only (N_NF = -1), whole product vs the oracle,
    complex64 and complex128."""
    from oracle.aim import AIMArray, AIMParams
    lay = wl.loop_array(nx, 1)
    A = AIMArray([loop_model], lay.type_of, lay.offsets, AIMParams(0.1, 2, -1, wl.DEFAULT_GRID_PHASE), 2 * np.pi)
    la = loop_array(ctx, nx, 1, n_nf=-1, types=c1.types)
    try:
        assert la.info["fft"][0] == {10: 128, 15: 160, 19: 224, 24: 256, 30: 320, 34: 352, 38: 384}[nx]
        x = wl.random_cvec(la.n, 0, 30 + nx)
        ref = A.matvec(np.ascontiguousarray(x))
        for prec in (mm.MM_C64, mm.MM_C128):
            _close(_apply(la, x, prec), ref, prec)
    finally:
        mm.mm_array_destroy(la.array)
