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
