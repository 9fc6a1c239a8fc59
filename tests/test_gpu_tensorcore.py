"""Macromodel contraction on tensor cores (tcgen05, BF16 / FP16 inputs, FP32
accumulation) and its accuracy recovered by FP64 iterative refinement.

Tolerances from the input rounding: BF16 keeps 8 significant bits (relative
rounding 2^-9 ~ 2e-3 per entry of [M; D] and x), so products of a few hundred
terms carry ~2e-3 relative error: bar 2e-2 relative L2 on y.  FP16 keeps 11 bits
(2^-12 ~ 2.4e-4): bar 3e-3.  After refinement the solution must meet the same
bar as the complex64 path (error vs the oracle's solution <= 1e-4)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1712_02443_gb300 as mm  # noqa: E402
from paper_1712_02443_gb300 import workloads as wl  # noqa: E402
from paper_1712_02443_gb300.arrays import loop_array  # noqa: E402

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
BAR = {mm.MM_C64_BF16: 2e-2, mm.MM_C64_F16: 3e-3}


@pytest.fixture(scope="module")
def c1():
    from paper_1712_02443_gb300.build import build
    build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = mm.mm_ctx_create(0)
    la = loop_array(ctx, 2, 2)
    yield la
    la.close()
    mm.mm_ctx_destroy(ctx)


def _apply(la, x, prec, nrhs=1):
    xd = torch.from_numpy(np.ascontiguousarray(x)).to(torch.complex64).cuda()
    yd = torch.empty_like(xd)
    mm.mm_apply(la.array, nrhs, xd, yd, prec, torch.cuda.current_stream())
    torch.cuda.synchronize()
    return yd.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("prec", [mm.MM_C64_F16, mm.MM_C64_BF16])
def test_tensorcore_matvec(c1, prec):
    g = np.load(os.path.join(GOLD, "c1_2x2.npz"))
    y = _apply(c1, g["x"], prec)
    rel = np.linalg.norm(y - g["y"]) / np.linalg.norm(g["y"])
    assert rel <= BAR[prec], rel
    # the same product in complex64 on CUDA cores is much closer; the tensor-core
    # error must come from the 16-bit inputs, not from a wrong layout
    y64 = _apply(c1, g["x"], mm.MM_C64)
    assert rel > 10 * np.linalg.norm(y64 - g["y"]) / np.linalg.norm(g["y"])


@pytest.mark.parametrize("prec", [mm.MM_C64_F16, mm.MM_C64_BF16])
def test_tensorcore_multi_rhs_ragged(c1, prec):
    ctx = c1.ctx
    g = np.load(os.path.join(GOLD, "ragged_3x5.npz"))
    la = loop_array(ctx, 3, 5, types=c1.types)
    try:
        X = wl.random_cvec(la.n, 0, 8, nrhs=3)
        Y = _apply(la, X, prec, nrhs=3)
        rel = np.linalg.norm(Y - g["y"]) / np.linalg.norm(g["y"])
        assert rel <= BAR[prec], rel
    finally:
        mm.mm_array_destroy(la.array)


@pytest.mark.parametrize("prec", [mm.MM_C64_F16, mm.MM_C64_BF16])
def test_tensorcore_solve_refined(c1, prec):
    g = np.load(os.path.join(GOLD, "c1_2x2.npz"))
    V = torch.from_numpy(g["V"]).cuda()
    E = torch.empty_like(V)
    st = mm.mm_solve(c1.array, 1, V, E, tol=1e-6, restart=50, max_iter=1000, precision=prec, refine=1,
                     inner_tol=1e-2)
    assert st["converged"] and st["rel_residual"] <= 1e-6
    err = np.linalg.norm(E.cpu().numpy() - g["E"]) / np.linalg.norm(g["E"])
    assert err <= 1e-4, err


C3_OUTERS = (0.30, 0.34, 0.38, 0.42)


@pytest.mark.parametrize("prec", [mm.MM_C64_F16, mm.MM_C64_BF16])
def test_tensorcore_four_types_64_rhs(c1, prec):
    """Four element types, 64 right-hand sides (whole-element 8-column output
    groups): sampled rows of all 64 columns vs the oracle."""
    g = np.load(os.path.join(GOLD, "c3_types_6x6.npz"))
    la = loop_array(c1.ctx, 6, 6, outers=C3_OUTERS, config_index=2)
    try:
        X = wl.random_cvec(la.n, 2, 7, nrhs=64)
        Y = _apply(la, X, prec, nrhs=64)[g["rows"]]
        rel = np.linalg.norm(Y - g["y_rows"]) / np.linalg.norm(g["y_rows"])
        assert rel <= BAR[prec], rel
    finally:
        la.close()


def test_tensorcore_many_tiles_per_cta(c1, loop_model):
    """32 x 32 array, 16 right-hand sides: 16384 columns, 576 output tiles of
    128 x 256, about four per CTA of the persistent kernel, so each CTA reuses
    both accumulators.  Far-field operator only (N_NF = -1) so that the
    oracle's full product is cheap; columns 8-15 are 1j times columns 0-7, whose
    products follow by linearity.  The whole product is compared, both formats."""
    from oracle.aim import AIMArray, AIMParams
    lay = wl.loop_array(32, 32)
    A = AIMArray([loop_model], lay.type_of, lay.offsets, AIMParams(0.1, 2, -1, wl.DEFAULT_GRID_PHASE), 2 * np.pi)
    la = loop_array(c1.ctx, 32, 32, n_nf=-1, types=c1.types)
    try:
        X8 = wl.random_cvec(la.n, 0, 14, nrhs=8)
        ref8 = np.stack([A.matvec(np.ascontiguousarray(X8[:, j])) for j in range(8)], axis=1)
        X = np.concatenate([X8, 1j * X8], axis=1)
        ref = np.concatenate([ref8, 1j * ref8], axis=1)
        for prec in (mm.MM_C64_F16, mm.MM_C64_BF16):
            Y = _apply(la, X, prec, nrhs=16)
            rel = np.linalg.norm(Y - ref) / np.linalg.norm(ref)
            assert rel <= BAR[prec], (prec, rel)
    finally:
        mm.mm_array_destroy(la.array)


@pytest.mark.parametrize("prec", [mm.MM_C64_F16, mm.MM_C64_BF16])
def test_tensorcore_wait_limit_reports_timeout(c1, prec):
    """The failure path of the bounded waits, with no GPU fault: the testing
    hook makes the GEMM issue no products, so its waits run out after 20 ms;
    the call returns MM_ETIMEOUT, and the next product (hook off) is correct."""
    g = np.load(os.path.join(GOLD, "c1_2x2.npz"))
    x = np.ascontiguousarray(g["x"].astype(np.complex64))
    y = np.zeros_like(x)
    mm.mm_test_tc_stall(20)
    try:
        with pytest.raises(mm.MacroAIMError) as e:
            mm.mm_apply_host(c1.array, 1, x, y, prec)
        assert e.value.status == mm.MM_ETIMEOUT
    finally:
        mm.mm_test_tc_stall(0)
    mm.mm_apply_host(c1.array, 1, x, y, prec)
    rel = np.linalg.norm(y.astype(np.complex128) - g["y"]) / np.linalg.norm(g["y"])
    assert rel <= BAR[prec], rel
