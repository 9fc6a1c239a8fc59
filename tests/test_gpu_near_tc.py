"""Block near field on tensor cores (TF32 three-product split, FP32 accumulation
in tensor memory) against the oracle, for every tile shape, k split and
right-hand-side count.

The split keeps about 2^-22 of each product (hi*hi + hi*lo + lo*hi with TF32
hi = rn(x), lo = rn(x - hi)), so the whole product must meet the complex64
bar of the other parity tests: relative L2 <= 1e-5, worst element <= 1e-4 of
max |y|.  MACROAIM_NEAR_SHAPE fixes the shape (5: 32 complex columns per tile,
6: 64) instead of the autotuner.  The products go into per-pair slices of a
partial-sum buffer, which a reduction kernel subtracts from v.  Shapes 7 and 8
(and 9, two stages) are the direct form (32 or 64 right-hand sides of one element per tile, the
element's pairs accumulated in tensor memory and subtracted from v in place);
it takes even right-hand-side counts of 16 or more, and other counts fall back
to the CUDA-core kernel."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1712_02443_gb300 as mm  # noqa: E402
from paper_1712_02443_gb300 import workloads as wl  # noqa: E402
from paper_1712_02443_gb300.arrays import loop_array  # noqa: E402

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
C3_OUTERS = (0.30, 0.34, 0.38, 0.42)


def _close(got, ref, l2=1e-5, worst=1e-4):
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    w = np.abs(got - ref).max() / np.abs(ref).max()
    assert rel <= l2 and w <= worst, (rel, w)
    return rel


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
def c3_types(ctx):
    la = loop_array(ctx, 6, 6, outers=C3_OUTERS, config_index=2)
    yield la.types
    la.close()


def _apply(la, X, nrhs, prec=mm.MM_C64):
    xd = torch.from_numpy(np.ascontiguousarray(X)).to(torch.complex64).cuda()
    yd = torch.empty_like(xd)
    mm.mm_apply(la.array, nrhs, xd, yd, prec, torch.cuda.current_stream())
    torch.cuda.synchronize()
    return yd.cpu().numpy().astype(np.complex128).reshape(la.n, nrhs)


@pytest.mark.parametrize("shape,ks", [(5, 1), (6, 1), (5, 2), (6, 2)])
@pytest.mark.parametrize("nrhs", [1, 3, 5, 8, 12, 24, 64])
def test_tensor_core_near_field_c3(ctx, c3_types, monkeypatch, shape, ks, nrhs):
    """6 x 6 array of the four loop types (16 x 9 type and offset blocks, ragged
    column tiles): sampled rows of every column vs the oracle."""
    monkeypatch.setenv("MACROAIM_NEAR_SHAPE", "%d,%d" % (shape, ks))
    g = np.load(os.path.join(GOLD, "c3_types_6x6.npz"))
    la = loop_array(ctx, 6, 6, outers=C3_OUTERS, config_index=2, types=c3_types)
    try:
        X = wl.random_cvec(la.n, 2, 7, nrhs=64)
        Y = _apply(la, X[:, :nrhs], nrhs)
        _close(Y[g["rows"]], g["y_rows"][:, :nrhs])
    finally:
        mm.mm_array_destroy(la.array)


@pytest.mark.parametrize("shape", [7, 8, 9])
@pytest.mark.parametrize("nrhs", [5, 8, 16, 24, 40, 64])
def test_tensor_core_direct_near_field_c3(ctx, c3_types, monkeypatch, shape, nrhs):
    """Direct form on the 6 x 6 four-type array: ragged right-hand-side tiles
    (24 and 40 against 32 or 64 per tile), and counts it does not take (odd, or
    below 16: the CUDA-core fallback), sampled rows vs the oracle."""
    monkeypatch.setenv("MACROAIM_NEAR_SHAPE", "%d,1" % shape)
    g = np.load(os.path.join(GOLD, "c3_types_6x6.npz"))
    la = loop_array(ctx, 6, 6, outers=C3_OUTERS, config_index=2, types=c3_types)
    try:
        X = wl.random_cvec(la.n, 2, 7, nrhs=64)
        Y = _apply(la, X[:, :nrhs], nrhs)
        _close(Y[g["rows"]], g["y_rows"][:, :nrhs])
    finally:
        mm.mm_array_destroy(la.array)


@pytest.mark.parametrize("shape,ks", [(5, 1), (6, 1), (5, 2), (6, 2)])
def test_tensor_core_near_field_c1_full(ctx, monkeypatch, shape, ks):
    """2 x 2 loop array, one right-hand side: every entry vs the oracle (k split 2:
    each unit's k tiles over two units, their partial sums in two planes)."""
    monkeypatch.setenv("MACROAIM_NEAR_SHAPE", "%d,%d" % (shape, ks))
    g = np.load(os.path.join(GOLD, "c1_2x2.npz"))
    la = loop_array(ctx, 2, 2)
    try:
        _close(_apply(la, g["x"], 1)[:, 0], g["y"])
    finally:
        la.close()


@pytest.mark.parametrize("shape,ks", [(5, 1), (6, 1), (6, 2)])
def test_tensor_core_near_field_c2_sampled(ctx, monkeypatch, shape, ks):
    """16 x 16 loop array (the benchmark workload), one right-hand side."""
    monkeypatch.setenv("MACROAIM_NEAR_SHAPE", "%d,%d" % (shape, ks))
    g = np.load(os.path.join(GOLD, "c2_16x16.npz"))
    la = loop_array(ctx, 16, 16)
    try:
        x = wl.random_cvec(la.n, 1, 7)
        y = _apply(la, x, 1)[:, 0]
        _close(y[g["rows"]], g["y_rows"])
    finally:
        la.close()


@pytest.mark.parametrize("nrhs,shapes", [(8, (0, 5)), (64, (0, 6, 8)), (32, (5, 7))])
def test_tensor_core_and_cuda_core_near_fields_agree(ctx, c3_types, monkeypatch, nrhs, shapes):
    """The tensor-core (partial-sum and direct) and CUDA-core block kernels on
    the same array and input: all FP32-level, so they agree well below the
    oracle bar.  Each row sums about 2,600 products (nine blocks of 288
    columns) in FP32 in a different order, so the two results differ by about
    sqrt(2600) x 2^-24 = 3e-6 of the near-field terms: bar 5e-6."""
    outs = []
    for shape in shapes:
        monkeypatch.setenv("MACROAIM_NEAR_SHAPE", "%d,1" % shape)
        la = loop_array(ctx, 6, 6, outers=C3_OUTERS, config_index=2, types=c3_types)
        try:
            X = wl.random_cvec(la.n, 2, 7, nrhs=nrhs)
            outs.append(_apply(la, X, nrhs))
        finally:
            mm.mm_array_destroy(la.array)
    for o in outs[1:]:
        rel = np.linalg.norm(o - outs[0]) / np.linalg.norm(outs[0])
        assert rel <= 5e-6, rel


def test_tensor_core_near_field_wait_limit(ctx, monkeypatch):
    """Bounded waits of the tensor-core near field, with no GPU fault: the
    testing hook makes it issue no products, its waits run out after 20 ms, the
    synchronising call returns MM_ETIMEOUT and the next product is correct."""
    monkeypatch.setenv("MACROAIM_NEAR_SHAPE", "5,1")
    g = np.load(os.path.join(GOLD, "c1_2x2.npz"))
    la = loop_array(ctx, 2, 2)
    try:
        x = np.ascontiguousarray(g["x"].astype(np.complex64))
        y = np.zeros_like(x)
        mm.mm_test_tc_stall(20)
        try:
            with pytest.raises(mm.MacroAIMError) as e:
                mm.mm_apply_host(la.array, 1, x, y, mm.MM_C64)
            assert e.value.status == mm.MM_ETIMEOUT
        finally:
            mm.mm_test_tc_stall(0)
        mm.mm_apply_host(la.array, 1, x, y, mm.MM_C64)
        _close(y.astype(np.complex128), g["y"])
    finally:
        la.close()


def test_tensor_core_direct_near_field_wait_limit(ctx, monkeypatch):
    """The direct form's bounded waits: no products issued, every wait runs out
    after 20 ms, MM_ETIMEOUT, and the next product (16 copies of the golden
    column) is correct."""
    monkeypatch.setenv("MACROAIM_NEAR_SHAPE", "7,1")
    g = np.load(os.path.join(GOLD, "c1_2x2.npz"))
    la = loop_array(ctx, 2, 2)
    try:
        X = np.ascontiguousarray(np.repeat(g["x"].astype(np.complex64)[:, None], 16, axis=1))
        Y = np.zeros_like(X)
        mm.mm_test_tc_stall(20)
        try:
            with pytest.raises(mm.MacroAIMError) as e:
                mm.mm_apply_host(la.array, 16, X.reshape(-1), Y.reshape(-1), mm.MM_C64)
            assert e.value.status == mm.MM_ETIMEOUT
        finally:
            mm.mm_test_tc_stall(0)
        mm.mm_apply_host(la.array, 16, X.reshape(-1), Y.reshape(-1), mm.MM_C64)
        for c in range(16):
            _close(Y[:, c].astype(np.complex128), g["y"])
    finally:
        la.close()
