"""Convenience constructors: library handles for the seeded loop arrays (marshalling only)."""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import _binding as b
from . import workloads as wl

K0 = 2.0 * np.pi
H, ORDER, N_NF = 0.1, 2, 3


@dataclass
class LibArray:
    ctx: object
    array: object
    layout: wl.ArrayLayout
    types: list
    meshes: list = field(default_factory=list)
    info: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.info["n_unknowns"]

    def close(self):
        b.mm_array_destroy(self.array)
        for t in self.types:
            b.mm_type_destroy(t)
        for m in self.meshes:
            b.mm_mesh_destroy(m)
        self.types, self.meshes = [], []


def build_types(ctx, layout: wl.ArrayLayout, k0: float = K0):
    meshes, types = [], []
    for et in layout.types:
        ms = b.mm_mesh_create(ctx, et.scatterer.xyz, et.scatterer.tri)
        me = b.mm_mesh_create(ctx, et.equiv.xyz, et.equiv.tri)
        meshes += [ms, me]
        types.append(b.mm_element_type_create(ctx, ms, me, k0))
    return meshes, types


def loop_array(ctx, nx: int, ny: int, outers=(0.4,), config_index: int = 0, h: float = H, order: int = ORDER,
               n_nf: int = N_NF, phase=wl.DEFAULT_GRID_PHASE, types=None) -> LibArray:
    layout = wl.loop_array(nx, ny, outers=outers, config_index=config_index)
    meshes = []
    if types is None:
        meshes, types = build_types(ctx, layout)
    per_elem = [types[t] for t in layout.type_of]
    arr = b.mm_array_create(ctx, per_elem, layout.offsets, h, order, n_nf, phase)
    la = LibArray(ctx, arr, layout, list(types), meshes)
    la.info = b.mm_array_info_get(arr)
    return la


def multiscale_array(ctx, nx: int, ny: int, meander=None, box_div=(8, 8, 2), h: float = H, order: int = ORDER,
                     n_nf: int = N_NF, phase=wl.DEFAULT_GRID_PHASE, types=None, near_csr: int = 0) -> LibArray:
    """nx x ny array of the multiscale element (loop with a meandered inner trace)."""
    layout = wl.multiscale_array(nx, ny, meander=meander, box_div=box_div)
    meshes = []
    if types is None:
        meshes, types = build_types(ctx, layout)
    arr = b.mm_array_create(ctx, [types[0]] * layout.n_elem, layout.offsets, h, order, n_nf, phase, near_csr)
    la = LibArray(ctx, arr, layout, list(types), meshes)
    la.info = b.mm_array_info_get(arr)
    return la
