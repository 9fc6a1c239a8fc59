"""Macromodel build with its dense FP64 steps on the GPU (blocked LU with partial
pivoting, triangular solves, ZGEMM products; taken for scatterers of at least
1024 RWG functions) against the host build of the same element (host-only
context): every matrix of the type within 1e-10 relative (Frobenius) -- the
two differ only in the order of FP64 rounding.  Elements: the loop (384
scatterer RWG, host path on both), the reduced multiscale element (535, host
path on both) and the full multiscale element (2,547 / 576, device path).

Near-field blocks filled on the GPU (exact EFIE Galerkin entries of the near
pairs minus the grid part, FP64) against the host fill of the same array
(MACROAIM_NEAR_FILL=host, fresh element types so that no block comes from the
cache): the assembled near-field CSR (pattern identical, values within 1e-12
relative) for one loop type and for four types (blocks between different
meshes), and the arrays' products agree."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1712_02443_gb300 as mm  # noqa: E402
from paper_1712_02443_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu
MATS = {"M": mm.MM_MAT_M, "D": mm.MM_MAT_D, "T": mm.MM_MAT_T, "A": mm.MM_MAT_A, "B": mm.MM_MAT_B,
        "GHH": mm.MM_MAT_GHH, "GHE": mm.MM_MAT_GHE, "PJ": mm.MM_MAT_PJ}


def _type(ctx, et):
    ms = mm.mm_mesh_create(ctx, et.scatterer.xyz, et.scatterer.tri)
    me = mm.mm_mesh_create(ctx, et.equiv.xyz, et.equiv.tri)
    t0 = time.perf_counter()
    ty = mm.mm_element_type_create(ctx, ms, me, 2 * np.pi)
    return ty, [ms, me], time.perf_counter() - t0


@pytest.mark.parametrize("name", ["loop", "multiscale_reduced", "multiscale"])
def test_device_build_matches_host_build(name):
    from paper_1712_02443_gb300.build import build
    build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    et = {"loop": lambda: wl.loop_element(),
          "multiscale_reduced": lambda: wl.multiscale_element(meander=wl.MEANDER_REDUCED,
                                                              box_div=wl.MEANDER_REDUCED_BOX),
          "multiscale": lambda: wl.multiscale_element()}[name]()
    hctx, dctx = mm.mm_ctx_create(-1), mm.mm_ctx_create(0)
    th, hm, t_host = _type(hctx, et)
    td, dm, t_dev = _type(dctx, et)
    try:
        for key, which in MATS.items():
            a, b = mm.mm_type_matrix(th, which), mm.mm_type_matrix(td, which)
            assert a.shape == b.shape
            rel = np.linalg.norm(b - a) / np.linalg.norm(a)
            assert rel <= 1e-10, (key, rel)
        print("%s: host build %.2f s, device build %.2f s" % (name, t_host, t_dev))
    finally:
        for t in (th, td):
            mm.mm_type_destroy(t)
        for m in hm + dm:
            mm.mm_mesh_destroy(m)
        mm.mm_ctx_destroy(hctx)
        mm.mm_ctx_destroy(dctx)


@pytest.mark.parametrize("outers,cfg", [((0.4,), 0), ((0.30, 0.34, 0.38, 0.42), 2)])
def test_device_near_fill_matches_host_fill(monkeypatch, outers, cfg):
    from paper_1712_02443_gb300.build import build
    from paper_1712_02443_gb300.arrays import loop_array
    build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = mm.mm_ctx_create(0)
    try:
        monkeypatch.setenv("MACROAIM_NEAR_FILL", "host")
        t0 = time.perf_counter()
        la_h = loop_array(ctx, 4, 3, outers=outers, config_index=cfg)
        t_host = time.perf_counter() - t0
        monkeypatch.delenv("MACROAIM_NEAR_FILL")
        t0 = time.perf_counter()
        la_d = loop_array(ctx, 4, 3, outers=outers, config_index=cfg)
        t_dev = time.perf_counter() - t0
        try:
            ex = {w: (mm.mm_array_export(la_h.array, w), mm.mm_array_export(la_d.array, w))
                  for w in (mm.MM_EXPORT_NEAR_PTR, mm.MM_EXPORT_NEAR_COL, mm.MM_EXPORT_NEAR_VAL)}
            for w in (mm.MM_EXPORT_NEAR_PTR, mm.MM_EXPORT_NEAR_COL):
                assert np.array_equal(ex[w][0], ex[w][1])
            vh, vd = ex[mm.MM_EXPORT_NEAR_VAL]
            assert vh.size > 0
            rel = np.linalg.norm(vd - vh) / np.linalg.norm(vh)
            assert rel <= 1e-12, rel
            x = wl.random_cvec(la_h.n, 0, 5)
            yh = np.zeros_like(x)
            yd = np.zeros_like(x)
            mm.mm_apply_host(la_h.array, 1, np.ascontiguousarray(x.astype(np.complex128)), yh, mm.MM_C128)
            mm.mm_apply_host(la_d.array, 1, np.ascontiguousarray(x.astype(np.complex128)), yd, mm.MM_C128)
            assert np.linalg.norm(yd - yh) / np.linalg.norm(yh) <= 1e-11
            print("near fill: host %.2f s, device %.2f s (array set-up incl. types)" % (t_host, t_dev))
        finally:
            la_h.close()
            la_d.close()
    finally:
        mm.mm_ctx_destroy(ctx)
