"""mm_apply_noalloc: the product for callers that cannot allocate device memory
(their framework owns the memory pool, or an allocation would stall a real-time
loop).  It must give the same result as mm_apply, call after call, while using
only the library's static scratch array.  Collected last on purpose."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1712_02443_gb300 as mm  # noqa: E402
from paper_1712_02443_gb300.arrays import loop_array  # noqa: E402

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
# same bars as the other GPU parity tests (the complex64 product bar of 1e-5
# relative L2; FP64 rounding for complex128)
TOL = {mm.MM_C64: 1e-5, mm.MM_C128: 1e-11}
DT = {mm.MM_C64: torch.complex64, mm.MM_C128: torch.complex128}


@pytest.fixture(scope="module")
def arr():
    from paper_1712_02443_gb300.build import build
    build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = mm.mm_ctx_create(0)
    la = loop_array(ctx, 2, 2)
    yield la
    la.close()
    mm.mm_ctx_destroy(ctx)


@pytest.mark.parametrize("prec", [mm.MM_C64, mm.MM_C128])
def test_noalloc_matches_apply_twice(arr, prec):
    g = np.load(os.path.join(GOLD, "c1_2x2.npz"))
    st = torch.cuda.current_stream()
    x = torch.from_numpy(g["x"]).to(DT[prec]).cuda()
    y_ref = torch.empty_like(x)
    mm.mm_apply(arr.array, 1, x, y_ref, prec, st)      # also makes the complex128 operator resident
    ref = y_ref.cpu().numpy().astype(np.complex128)
    for _ in range(2):                                  # two calls in a row share the scratch
        y = torch.full_like(x, float("nan"))
        mm.mm_apply_noalloc(arr.array, 1, x, y, prec, st)
        torch.cuda.synchronize()
        got = y.cpu().numpy().astype(np.complex128)
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel <= TOL[prec], rel
        # and both agree with the oracle's expected values
        assert np.linalg.norm(got - g["y"]) / np.linalg.norm(g["y"]) <= TOL[prec]


@pytest.mark.parametrize("prec", [mm.MM_C128, mm.MM_C64])
def test_noalloc_16x16_fits_the_scratch(prec):
    """The 16x16 loop array (73,728 unknowns, one right-hand side) fits the
    16 MiB scratch at either precision: two calls in a row match mm_apply."""
    from paper_1712_02443_gb300.build import build
    build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = mm.mm_ctx_create(0)
    la = loop_array(ctx, 16, 16)
    try:
        rng = np.random.default_rng(20171206)
        xh = rng.standard_normal(la.n) + 1j * rng.standard_normal(la.n)
        st = torch.cuda.current_stream()
        x = torch.from_numpy(xh).to(DT[prec]).cuda()
        y_ref = torch.empty_like(x)
        mm.mm_apply(la.array, 1, x, y_ref, prec, st)
        ref = y_ref.cpu().numpy().astype(np.complex128)
        for _ in range(2):
            y = torch.full_like(x, float("nan"))
            mm.mm_apply_noalloc(la.array, 1, x, y, prec, st)
            torch.cuda.synchronize()
            got = y.cpu().numpy().astype(np.complex128)
            rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert rel <= TOL[prec], rel
    finally:
        la.close()
        mm.mm_ctx_destroy(ctx)


def test_noalloc_rejects_oversized_requests(arr):
    nrhs = 256
    x = torch.zeros(arr.n * nrhs, dtype=torch.complex64, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(mm.MacroAIMError) as e:
        mm.mm_apply_noalloc(arr.array, nrhs, x, y, mm.MM_C64)
    assert e.value.status == mm.MM_EINVAL
    assert "static maximum" in str(e.value)
