"""Macromodel build with its dense FP64 steps on the GPU (blocked LU with partial
pivoting, triangular solves, ZGEMM products; taken for scatterers of at least
1024 RWG functions) against the host build of the same element (host-only
context): every matrix of the type within 1e-10 relative (Frobenius) -- the
two differ only in the order of FP64 rounding.  Elements: the loop (384
scatterer RWG, host path on both), the reduced multiscale element (535, host
path on both) and the full multiscale element (2,547 / 576, device path)."""
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
