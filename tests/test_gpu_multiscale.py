"""Multiscale element (square loop with a meandered inner trace) on the GPU: the
product in every precision and refined solves against the oracle.

The reduced element (workloads.MEANDER_REDUCED, 535 scatterer RWG, 288 box RWG)
keeps the oracle's fills within seconds; the 2x2 array with 8 right-hand sides
takes the block near field and the tensor-core GEMM.  Tolerances as in the other
parity files: complex128 rounding (1e-11 L2), complex64 (1e-5), BF16 / FP16
input rounding (2e-2 / 3e-3); solutions of the refined solves to 1e-6 must be
within 1e-4 of the oracle's 1e-12 solution."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1712_02443_gb300 as mm  # noqa: E402
from paper_1712_02443_gb300 import workloads as wl  # noqa: E402
from paper_1712_02443_gb300.arrays import multiscale_array  # noqa: E402

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
BAR = {mm.MM_C128: 1e-11, mm.MM_C64: 1e-5, mm.MM_C64_F16: 3e-3, mm.MM_C64_BF16: 2e-2}


@pytest.fixture(scope="module")
def c4():
    from paper_1712_02443_gb300.build import build
    build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = mm.mm_ctx_create(0)
    la = multiscale_array(ctx, 2, 2, meander=wl.MEANDER_REDUCED, box_div=wl.MEANDER_REDUCED_BOX)
    yield la
    la.close()
    mm.mm_ctx_destroy(ctx)


@pytest.mark.parametrize("prec", [mm.MM_C128, mm.MM_C64, mm.MM_C64_F16, mm.MM_C64_BF16])
def test_multiscale_product_8_rhs(c4, prec):
    g = np.load(os.path.join(GOLD, "c4_meander_2x2.npz"))
    X = wl.random_cvec(c4.n, 3, 7, nrhs=8)
    assert np.allclose([X.sum(), (np.abs(X) ** 2).sum()], g["x_check"])
    dt = torch.complex128 if prec == mm.MM_C128 else torch.complex64
    xd = torch.from_numpy(np.ascontiguousarray(X)).to(dt).cuda()
    yd = torch.empty_like(xd)
    mm.mm_apply(c4.array, 8, xd, yd, prec, torch.cuda.current_stream())
    torch.cuda.synchronize()
    Y = yd.cpu().numpy().astype(np.complex128)
    rel = np.linalg.norm(Y - g["y"]) / np.linalg.norm(g["y"])
    assert rel <= BAR[prec], rel


@pytest.mark.parametrize("prec", [mm.MM_C64_F16, mm.MM_C64_BF16, mm.MM_C64])
def test_multiscale_refined_solve(c4, prec):
    """The per-result error of the mixed-precision solve against the oracle's
    FP64 solution: 16-bit macromodel GEMM, FP32 FFT and near field, FP64 Arnoldi
    and refinement."""
    g = np.load(os.path.join(GOLD, "c4_meander_2x2.npz"))
    V = torch.from_numpy(g["V"]).cuda()
    E = torch.empty_like(V)
    st = mm.mm_solve(c4.array, 1, V, E, tol=1e-6, restart=50, max_iter=2000, precision=prec, refine=1,
                     inner_tol=1e-3 if prec != mm.MM_C64 else 1e-5)
    assert st["converged"] and st["rel_residual"] <= 1e-6
    err = np.linalg.norm(E.cpu().numpy() - g["E"]) / np.linalg.norm(g["E"])
    assert err <= 1e-4, err


@pytest.mark.parametrize("prec", [mm.MM_C64_F16, mm.MM_C64_BF16])
def test_multiscale_refined_solve_block_jacobi(c4, prec):
    g = np.load(os.path.join(GOLD, "c4_meander_2x2.npz"))
    V = torch.from_numpy(g["V"]).cuda()
    E = torch.empty_like(V)
    st = mm.mm_solve(c4.array, 1, V, E, tol=1e-6, restart=50, max_iter=2000, precision=prec, refine=1,
                     inner_tol=1e-3, precond=1)
    assert st["converged"] and st["rel_residual"] <= 1e-6
    err = np.linalg.norm(E.cpu().numpy() - g["E"]) / np.linalg.norm(g["E"])
    assert err <= 1e-4, err
