"""The complex128 product in float-float arithmetic (MM_C128_FF): every stage
(macromodel GEMM, projection, FFT convolution, interpolation, block near field)
carries its values as unevaluated sums of two floats (Dekker 1971) on the FP32
pipe; the stages exchange FP64 vectors and grids.

Bars.  Products are exact (FMA) and the running sums exact (two-sum); what is
lost is the FP32 rounding of the correction term, which holds about ulp(sum)
and takes K additions: about 2^-48 sqrt(K) |a||b| per sum of K terms, some
4e-14 of a random sum of K ~ 300 (GEMM, N^_t terms) to ~540 (a near-field
row) terms.  The product then subtracts the near field from the far field and
the macromodel term (|G_NF u| is several times |y|), which scales the error
relative to |y| by that factor: 2e-13 was measured at 2 x 2.  The bar is
1e-12 relative L2 both against the plain FP64 product (MM_C128) and against the
complex128 oracle (the FP64 product itself is within about 1e-13 of it), the
accuracy the refinement residual is held to.

The refinement residual of a complex64 solve uses this product by default
(mm_solve_opts.fp64 = 0), and the inner solves then keep their Krylov basis
in float-float and take the Arnoldi products on the FP32 pipe: the solutions
of both forms meet the tolerance and agree with the oracle's solve.
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
C3_OUTERS = (0.30, 0.34, 0.38, 0.42)
BAR_ORACLE, BAR_FP64 = 1e-12, 1e-12


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
def c1(ctx):
    la = loop_array(ctx, 2, 2)
    yield la
    la.close()


def _apply(la, x, prec, nrhs=1):
    xd = torch.from_numpy(np.ascontiguousarray(x)).to(torch.complex128).cuda()
    yd = torch.empty_like(xd)
    mm.mm_apply(la.array, nrhs, xd, yd, prec, torch.cuda.current_stream())
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def _both(la, x, nrhs=1):
    return _apply(la, x, mm.MM_C128_FF, nrhs), _apply(la, x, mm.MM_C128, nrhs)


def test_ff_c1_matvec(c1):
    g = np.load(os.path.join(GOLD, "c1_2x2.npz"))
    yf, yd = _both(c1, g["x"])
    assert _rel(yf, yd) <= BAR_FP64, _rel(yf, yd)
    assert _rel(yf, g["y"]) <= BAR_ORACLE, _rel(yf, g["y"])


def test_ff_ragged_multi_rhs(ctx, c1):
    g = np.load(os.path.join(GOLD, "ragged_3x5.npz"))
    la = loop_array(ctx, 3, 5, types=c1.types)
    try:
        X = wl.random_cvec(la.n, 0, 8, nrhs=3)
        yf, yd = _both(la, X, nrhs=3)
        yf = yf.reshape(la.n, 3)
        assert _rel(yf, yd.reshape(la.n, 3)) <= BAR_FP64
        assert _rel(yf, g["y"]) <= BAR_ORACLE
        # a column alone equals its column in the batch
        y1 = _apply(la, np.ascontiguousarray(X[:, 1]), mm.MM_C128_FF)
        assert _rel(y1, yf[:, 1]) <= 1e-14   # FP64 atomics of the near field in another order
    finally:
        mm.mm_array_destroy(la.array)


def test_ff_c2_full_size_sampled_rows(ctx, c1):
    """16 x 16 array, one right-hand side (the refinement residual of the benchmark's solves)."""
    g = np.load(os.path.join(GOLD, "c2_16x16.npz"))
    la = loop_array(ctx, 16, 16, types=c1.types)
    try:
        x = wl.random_cvec(la.n, 1, 7)
        yf, yd = _both(la, x)
        assert _rel(yf, yd) <= BAR_FP64, _rel(yf, yd)
        assert _rel(yf[g["rows"]], g["y_rows"]) <= BAR_ORACLE
    finally:
        mm.mm_array_destroy(la.array)


def test_ff_c3_four_types_64_rhs(ctx):
    g = np.load(os.path.join(GOLD, "c3_types_6x6.npz"))
    la = loop_array(ctx, 6, 6, outers=C3_OUTERS, config_index=2)
    try:
        X = wl.random_cvec(la.n, 2, 7, nrhs=64)
        yf, yd = _both(la, X, nrhs=64)
        yf = yf.reshape(la.n, 64)
        assert _rel(yf, yd.reshape(la.n, 64)) <= BAR_FP64
        assert _rel(yf[g["rows"]], g["y_rows"]) <= BAR_ORACLE
    finally:
        la.close()


def test_ff_far_field_only_operator(ctx, c1, loop_model):
    """No near field (N_NF = -1): only the GEMM takes the float-float form."""
    from oracle.aim import AIMArray, AIMParams
    lay = wl.loop_array(3, 2)
    A = AIMArray([loop_model], lay.type_of, lay.offsets, AIMParams(0.1, 2, -1, wl.DEFAULT_GRID_PHASE), K0)
    la = loop_array(ctx, 3, 2, n_nf=-1, types=c1.types)
    try:
        X = wl.random_cvec(la.n, 0, 13, nrhs=3)
        yf = _apply(la, X, mm.MM_C128_FF, nrhs=3).reshape(la.n, 3)
        ref = np.stack([A.matvec(np.ascontiguousarray(X[:, j])) for j in range(3)], axis=1)
        assert _rel(yf, ref) <= BAR_ORACLE
    finally:
        mm.mm_array_destroy(la.array)


def test_ff_csr_near_field(ctx, c1, monkeypatch):
    """Arrays that apply their near field as CSR rows (MACROAIM_NEAR=csr): the
    float-float GEMM feeds the FP64 three-product SpMV (Re u + Im u from its
    epilogue)."""
    monkeypatch.setenv("MACROAIM_NEAR", "csr")
    g = np.load(os.path.join(GOLD, "c1_2x2.npz"))
    la = loop_array(ctx, 2, 2, types=c1.types)
    try:
        yf, yd = _both(la, g["x"])
        assert _rel(yf, yd) <= BAR_FP64
        assert _rel(yf, g["y"]) <= BAR_ORACLE
    finally:
        mm.mm_array_destroy(la.array)


@pytest.mark.parametrize("residual", [0, 1])
def test_refinement_residual_forms(c1, residual):
    """GMRES to 1e-6 with complex64 inner solves and either refinement residual
    (0: float-float contractions, 1: FP64): converged, residual met, solution
    within the cond * tol bar of the oracle's 1e-12 solve."""
    g = np.load(os.path.join(GOLD, "c1_2x2.npz"))
    V = torch.from_numpy(g["V"]).cuda()
    E = torch.empty_like(V)
    st = mm.mm_solve(c1.array, 1, V, E, tol=1e-6, restart=50, max_iter=500, precision=mm.MM_C64, refine=1,
                     fp64=residual)
    assert st["converged"] and st["rel_residual"] <= 1e-6
    err = _rel(E.cpu().numpy(), g["E"])
    assert err <= 1e-4, err


def test_refinement_residual_forms_agree_at_1e_10(ctx, c1):
    """Tolerance 1e-10, beyond the complex64 operator's own accuracy: only the
    refinement residual makes it reachable.  Both residual forms get there and
    their solutions agree within 1e-7 (each is within cond * 1e-10 of the
    exact solution)."""
    g = np.load(os.path.join(GOLD, "c1_2x2.npz"))
    V = torch.from_numpy(g["V"]).cuda()
    out = []
    for residual in (0, 1):
        E = torch.empty_like(V)
        st = mm.mm_solve(c1.array, 1, V, E, tol=1e-10, restart=50, max_iter=2000, precision=mm.MM_C64, refine=1,
                         inner_tol=1e-4, fp64=residual)
        assert st["converged"] and st["rel_residual"] <= 1e-10
        assert st["refinements"] >= 2
        out.append(E.cpu().numpy())
    assert _rel(out[0], out[1]) <= 1e-7


def test_ff_rejected_where_unsupported(c1):
    x = torch.zeros(c1.n, dtype=torch.complex128, device="cuda")
    with pytest.raises(mm.MacroAIMError) as e:
        mm.mm_solve(c1.array, 1, x, torch.empty_like(x), tol=1e-6, precision=mm.MM_C64, refine=1, fp64=2)
    assert e.value.status == mm.MM_EINVAL


@pytest.mark.parametrize("nx", [10, 15, 19, 34, 38])
def test_ff_fft_lengths(ctx, c1, loop_model, nx):
    """The float-float FFT stages (Stockham radices 4, 2, 3, 5, 7 and 11 on CF
    values) at padded x lengths 128, 160, 224, 352 and 384: linear arrays, far
    field only (N_NF = -1), whole product against the oracle and the FP64 product."""
    from oracle.aim import AIMArray, AIMParams
    lay = wl.loop_array(nx, 1)
    A = AIMArray([loop_model], lay.type_of, lay.offsets, AIMParams(0.1, 2, -1, wl.DEFAULT_GRID_PHASE), K0)
    la = loop_array(ctx, nx, 1, n_nf=-1, types=c1.types)
    try:
        assert la.info["fft"][0] == {10: 128, 15: 160, 19: 224, 34: 352, 38: 384}[nx]
        x = wl.random_cvec(la.n, 0, 30 + nx)
        yf, yd = _both(la, x)
        assert _rel(yf, yd) <= BAR_FP64
        assert _rel(yf, A.matvec(np.ascontiguousarray(x))) <= BAR_ORACLE
    finally:
        mm.mm_array_destroy(la.array)
