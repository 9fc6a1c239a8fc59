"""Several arrays in one product call (mm_apply_batch) and the grid-stage
launch schedules chosen by the tuner.

* One call over three arrays of different sizes, element types and
  right-hand-side counts: each array's columns equal its product alone and
  the oracle's, within the complex64 product bar (1e-5 relative L2).
* Every projection / interpolation schedule (fixed through MACROAIM_GRID_SCHED)
  gives the oracle's product within the same bar; the tuner records its
  choices and timings (mm_array_tuning)."""
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


def test_batch_of_uneven_arrays(ctx):
    g1 = np.load(os.path.join(GOLD, "c1_2x2.npz"))
    g2 = np.load(os.path.join(GOLD, "ragged_3x5.npz"))
    g3 = np.load(os.path.join(GOLD, "c3_types_6x6.npz"))
    a1 = loop_array(ctx, 2, 2)
    a2 = loop_array(ctx, 3, 5, types=a1.types)
    a3 = loop_array(ctx, 6, 6, outers=C3_OUTERS, config_index=2)
    try:
        xs = [g1["x"], wl.random_cvec(a2.n, 0, 8, nrhs=3), wl.random_cvec(a3.n, 2, 7, nrhs=64)]
        nr = [1, 3, 64]
        X = [torch.from_numpy(np.ascontiguousarray(x).reshape(-1)).to(torch.complex64).cuda() for x in xs]
        Y = [torch.empty_like(x) for x in X]
        st = torch.cuda.current_stream()
        mm.mm_apply_batch([a1.array, a2.array, a3.array], nr, X, Y, mm.MM_C64, st)
        torch.cuda.synchronize()
        out = [y.cpu().numpy().astype(np.complex128) for y in Y]
        for la, x, y, r in zip((a1, a2, a3), X, out, nr):
            y1 = torch.empty_like(x)
            mm.mm_apply(la.array, r, x, y1, mm.MM_C64, st)
            torch.cuda.synchronize()
            assert _rel(y, y1.cpu().numpy().astype(np.complex128)) <= 1e-6
        assert _rel(out[0], g1["y"]) <= 1e-5
        assert _rel(out[1].reshape(a2.n, 3), g2["y"]) <= 1e-5
        assert _rel(out[2].reshape(a3.n, 64)[g3["rows"]], g3["y_rows"]) <= 1e-5
        for la, r in zip((a1, a2, a3), nr):
            t = mm.mm_array_tuning(la.array, r)
            assert t is not None and t["project"] >= 0 and t["interp"] >= 0
            assert len(t["project_ms"]) >= 2 and len(t["interp_ms"]) >= 2
    finally:
        a3.close()
        mm.mm_array_destroy(a2.array)
        a1.close()


@pytest.mark.parametrize("prec", [mm.MM_C64, mm.MM_C64_F16, mm.MM_C128, mm.MM_C128_FF])
def test_batch_graph_replay(ctx, prec):
    """From the second call with the same arrays, widths, buffers and precision
    (the float-float complex128 product included) the batch is captured into one
    CUDA graph and replayed: new inputs in the
    same buffers give the new products (each equal to mm_apply alone), and
    destroying an array of a captured batch drops its graph (a later batch with a
    new array of the same size is computed afresh)."""
    a1 = loop_array(ctx, 2, 2)
    a2 = loop_array(ctx, 6, 6, outers=C3_OUTERS, config_index=2)
    wide = prec in (mm.MM_C128, mm.MM_C128_FF)
    dt = torch.complex128 if wide else torch.complex64
    tol = 1e-11 if wide else 1e-5
    try:
        nr = [1, 16]
        X = [torch.empty(la.n * r, dtype=dt, device="cuda") for la, r in zip((a1, a2), nr)]
        Y = [torch.empty_like(x) for x in X]
        st = torch.cuda.current_stream()
        for call in range(4):   # call 0: tuned; 1: captured and replayed; 2, 3: replayed
            xs = [wl.random_cvec(a1.n, 0, 40 + call), wl.random_cvec(a2.n, 2, 50 + call, nrhs=16)]
            for x, h in zip(X, xs):
                x.copy_(torch.from_numpy(np.ascontiguousarray(h).reshape(-1)).to(dt))
            mm.mm_apply_batch([a1.array, a2.array], nr, X, Y, prec, st)
            torch.cuda.synchronize()
            for la, x, y, r in zip((a1, a2), X, Y, nr):
                y1 = torch.empty_like(x)
                mm.mm_apply(la.array, r, x, y1, prec, st)
                torch.cuda.synchronize()
                assert _rel(y.cpu().numpy().astype(np.complex128), y1.cpu().numpy().astype(np.complex128)) <= tol
            assert mm.mm_batch_graphs(a2.array) == (0 if call == 0 else 1)
        a3 = loop_array(ctx, 2, 2, types=a1.types)
        mm.mm_array_destroy(a1.array)
        assert mm.mm_batch_graphs(a2.array) == 0
        a1.array = a3.array
        g1 = np.load(os.path.join(GOLD, "c1_2x2.npz"))
        X[0].copy_(torch.from_numpy(g1["x"]).to(dt))
        for _ in range(3):
            mm.mm_apply_batch([a1.array, a2.array], nr, X, Y, prec, st)
            torch.cuda.synchronize()
            # the 16-bit bar of the GEMM tests; the float-float bar of tests/test_gpu_ff.py
            bar = {mm.MM_C128: 1e-10, mm.MM_C128_FF: 1e-12, mm.MM_C64: 1e-5, mm.MM_C64_F16: 3e-3}[prec]
            assert _rel(Y[0].cpu().numpy().astype(np.complex128), g1["y"]) <= bar
    finally:
        a2.close()
        a1.close()


def test_batch_rejects_an_array_twice(ctx):
    la = loop_array(ctx, 2, 2)
    try:
        x = torch.zeros(la.n, dtype=torch.complex64, device="cuda")
        y1, y2 = torch.zeros_like(x), torch.zeros_like(x)
        with pytest.raises(mm.MacroAIMError) as e:
            mm.mm_apply_batch([la.array, la.array], [1, 1], [x, x], [y1, y2], mm.MM_C64)
        assert e.value.status == mm.MM_EINVAL
    finally:
        la.close()


@pytest.mark.parametrize("sched", ["0,0", "1,1", "2,2", "0,2", "2,0", "3,0", "3,2"])
def test_every_grid_schedule_one_rhs(ctx, monkeypatch, sched):
    monkeypatch.setenv("MACROAIM_GRID_SCHED", sched)
    g = np.load(os.path.join(GOLD, "c1_2x2.npz"))
    la = loop_array(ctx, 2, 2)
    try:
        x = torch.from_numpy(g["x"]).to(torch.complex64).cuda()
        y = torch.empty_like(x)
        mm.mm_apply(la.array, 1, x, y, mm.MM_C64, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert _rel(y.cpu().numpy().astype(np.complex128), g["y"]) <= 1e-5
    finally:
        la.close()


@pytest.mark.parametrize("sched", ["0,0", "1,1", "0,1", "1,0", "2,0", "2,1", "3,0", "3,1", "0,2", "3,2", "0,3", "3,3"])
@pytest.mark.parametrize("prec", [mm.MM_C64, mm.MM_C128])
def test_every_grid_schedule_64_rhs(ctx, monkeypatch, sched, prec):
    monkeypatch.setenv("MACROAIM_GRID_SCHED", sched)
    g = np.load(os.path.join(GOLD, "c3_types_6x6.npz"))
    la = loop_array(ctx, 6, 6, outers=C3_OUTERS, config_index=2)
    try:
        X = wl.random_cvec(la.n, 2, 7, nrhs=64)
        dt = torch.complex128 if prec == mm.MM_C128 else torch.complex64
        x = torch.from_numpy(np.ascontiguousarray(X).reshape(-1)).to(dt).cuda()
        y = torch.empty_like(x)
        mm.mm_apply(la.array, 64, x, y, prec, torch.cuda.current_stream())
        torch.cuda.synchronize()
        Y = y.cpu().numpy().astype(np.complex128).reshape(la.n, 64)
        assert _rel(Y[g["rows"]], g["y_rows"]) <= (1e-11 if prec == mm.MM_C128 else 1e-5)
    finally:
        la.close()


@pytest.mark.parametrize("nrhs", [8, 12, 20])
@pytest.mark.parametrize("sched", ["3,0", "0,2", "3,2", "3,3"])
def test_table_projection_ragged_chunks(ctx, monkeypatch, nrhs, sched):
    """Table-driven projection (projection schedule 3) and the
    right-hand-side-lane interpolation (interpolation schedule 2), eight
    right-hand sides per pass: counts that leave a partial last pass,
    complex64, sampled rows vs the oracle."""
    monkeypatch.setenv("MACROAIM_GRID_SCHED", sched)
    g = np.load(os.path.join(GOLD, "c3_types_6x6.npz"))
    la = loop_array(ctx, 6, 6, outers=C3_OUTERS, config_index=2)
    try:
        X = wl.random_cvec(la.n, 2, 7, nrhs=64)[:, :nrhs]
        x = torch.from_numpy(np.ascontiguousarray(X).reshape(-1)).to(torch.complex64).cuda()
        y = torch.empty_like(x)
        mm.mm_apply(la.array, nrhs, x, y, mm.MM_C64, torch.cuda.current_stream())
        torch.cuda.synchronize()
        Y = y.cpu().numpy().astype(np.complex128).reshape(la.n, nrhs)
        assert _rel(Y[g["rows"]], g["y_rows"][:, :nrhs]) <= 1e-5
    finally:
        la.close()
