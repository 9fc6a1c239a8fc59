"""Repeated products of a loop array, for profiling one stage with ncu.

  python -m paper_1712_02443_gb300.profile_run --side 16 --nrhs 1 --reps 3 [--types 1|4]
      [--precision c64|c128|ff|bf16|f16] [--stages]

The array is the seeded loop array of the benchmark (one loop type; four loop
types drawn per cell with --types 4), built on cuda:0; the near-field kernel
shape can be fixed with MACROAIM_NEAR_SHAPE as for any product.  Prints the
unknown count and the shape the array chose; with --stages, also the stage
profiler's device time per product and stage over the repetitions (after one
untimed product).
"""
from __future__ import annotations

import argparse

import numpy as np


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--side", type=int, default=16)
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--types", type=int, default=1, choices=[1, 4])
    ap.add_argument("--precision", default="c64", choices=["c64", "c128", "ff", "bf16", "f16"])
    ap.add_argument("--stages", action="store_true")
    a = ap.parse_args()
    import torch

    from . import _binding as mm
    from . import workloads as wl
    from .arrays import loop_array
    from .build import build
    build()
    prec = {"c64": mm.MM_C64, "c128": mm.MM_C128, "ff": mm.MM_C128_FF, "bf16": mm.MM_C64_BF16,
            "f16": mm.MM_C64_F16}[a.precision]
    wide = prec in (mm.MM_C128, mm.MM_C128_FF)
    outers = (0.4,) if a.types == 1 else (0.30, 0.34, 0.38, 0.42)
    ctx = mm.mm_ctx_create(0)
    la = loop_array(ctx, a.side, a.side, outers=outers, config_index=0 if a.types == 1 else 2)
    dt = torch.complex128 if wide else torch.complex64
    x = torch.from_numpy(np.ascontiguousarray(wl.random_cvec(la.n, 1, 7, nrhs=a.nrhs)).reshape(-1)).to(dt).cuda()
    y = torch.empty_like(x)
    if a.stages:
        mm.mm_apply(la.array, a.nrhs, x, y, prec, torch.cuda.current_stream())
        mm.mm_profile_enable(la.array, True)
    for _ in range(a.reps):
        mm.mm_apply(la.array, a.nrhs, x, y, prec, torch.cuda.current_stream())
    torch.cuda.synchronize()
    print("unknowns", la.n, "near shape", mm.mm_array_near_shape(la.array, a.nrhs,
                                                                 mm.MM_C128 if wide else mm.MM_C64))
    if a.stages:
        tab = mm.mm_profile_read(la.array, mm.MM_C128 if wide else mm.MM_C64)
        mm.mm_profile_enable(la.array, False)
        print("us per product:", {k: round(1e3 * v["ms"] / a.reps, 1) for k, v in tab.items() if v["launches"]})
    la.close()
    mm.mm_ctx_destroy(ctx)


if __name__ == "__main__":
    main()
