"""The C-ABI library on the host: it loads, exports every declared symbol, and its
FP64 set-up (run in a host-only context) equals the oracle's."""
import os
import re

import numpy as np
import pytest

import paper_1712_02443_gb300 as mm
from paper_1712_02443_gb300 import workloads as wl
from paper_1712_02443_gb300.arrays import loop_array

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
K0 = 2.0 * np.pi


@pytest.fixture(scope="module")
def lib():
    from paper_1712_02443_gb300.build import build
    build()
    return mm.load()


def test_library_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "macroaim.h")).read()
    declared = set(re.findall(r"^\s*(?:mm_status|void|const char\*)\s+(mm_\w+)\s*\(", hdr, re.M))
    assert len(declared) >= 18
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(mm.exported_symbols())


@pytest.fixture(scope="module")
def host_ctx(lib):
    ctx = mm.mm_ctx_create(-1)
    yield ctx
    mm.mm_ctx_destroy(ctx)


@pytest.fixture(scope="module")
def lib_c1(host_ctx):
    la = loop_array(host_ctx, 2, 2)
    yield la
    la.close()


def test_type_matrices_match_oracle(lib_c1, loop_model):
    ty = lib_c1.types[0]
    ref = {mm.MM_MAT_M: loop_model.M, mm.MM_MAT_D: loop_model.D, mm.MM_MAT_T: loop_model.T, mm.MM_MAT_A: loop_model.A,
           mm.MM_MAT_B: loop_model.B, mm.MM_MAT_GHH: loop_model.G_hEH, mm.MM_MAT_GHE: loop_model.G_hEE}
    for which, R in ref.items():
        L = mm.mm_type_matrix(ty, which)
        assert L.shape == R.shape
        assert np.abs(L - R).max() <= 1e-11 * np.abs(R).max(), which


@pytest.fixture(scope="module")
def oracle_c1(loop_model, c1_layout):
    from oracle.aim import AIMArray, AIMParams
    return AIMArray([loop_model], c1_layout.type_of, c1_layout.offsets, AIMParams(0.1, 2, 3, wl.DEFAULT_GRID_PHASE), K0)


def test_aim_setup_matches_oracle(lib_c1, oracle_c1):
    A = oracle_c1
    arr = lib_c1.array
    info = lib_c1.info
    assert tuple(info["grid"]) == A.N
    anc = mm.mm_array_export(arr, mm.MM_EXPORT_ANCHORS).reshape(-1, 3)
    assert np.array_equal(anc, A.anc)                      # integer work: bit-exact
    Pi = mm.mm_array_export(arr, mm.MM_EXPORT_PI).reshape(A.Pi.shape)
    assert np.abs(Pi - A.Pi).max() <= 1e-13 * np.abs(A.Pi).max()
    G = A.GNF.tocsr()
    G.sort_indices()
    ptr = mm.mm_array_export(arr, mm.MM_EXPORT_NEAR_PTR)
    col = mm.mm_array_export(arr, mm.MM_EXPORT_NEAR_COL)
    val = mm.mm_array_export(arr, mm.MM_EXPORT_NEAR_VAL)
    assert np.array_equal(ptr, G.indptr) and np.array_equal(col, G.indices)
    assert np.abs(val - G.data).max() <= 1e-12 * np.abs(G.data).max()


def test_green_spectrum_matches_numpy_fft(lib_c1, oracle_c1):
    """Library Green's spectrum (its own padded sizes) vs numpy FFT of the same embedding."""
    from oracle.aim import grid_green
    N = oracle_c1.N
    P = tuple(lib_c1.info["fft"])
    assert all(P[a] >= 2 * N[a] - 1 for a in range(3))
    idx = []
    for a in range(3):
        i = np.arange(P[a])
        d = np.where(i < N[a], i, np.where(i > P[a] - N[a], i - P[a], 10 ** 6))
        idx.append(d)
    D = np.stack(np.meshgrid(*idx, indexing="ij"), axis=-1)
    K = grid_green(np.where(np.abs(D) >= 10 ** 6, 0, D), 0.1, K0)
    K[(np.abs(D) >= 10 ** 6).any(axis=-1)] = 0.0
    ref = np.fft.fftn(K) / np.prod(P)
    got = mm.mm_array_export(lib_c1.array, mm.MM_EXPORT_GHAT).reshape(P)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_device_calls_refused_on_host_context(lib_c1):
    with pytest.raises(mm.MacroAIMError) as e:
        mm.mm_apply(lib_c1.array, 1, 1, 2, mm.MM_C64)
    assert e.value.status == mm.MM_EINVAL


def test_invalid_inputs_are_rejected(host_ctx):
    with pytest.raises(mm.MacroAIMError):
        mm.mm_mesh_create(host_ctx, np.zeros((3, 3)), np.array([[0, 1, 5]]))   # index out of range
    with pytest.raises(mm.MacroAIMError):
        mm.mm_mesh_create(host_ctx, np.zeros((3, 3)), np.array([[0, 1, 2]]))   # degenerate triangle
    open_mesh = wl.square_loop_mesh()
    ms = mm.mm_mesh_create(host_ctx, open_mesh.xyz, open_mesh.tri)
    assert mm.mm_mesh_info(ms)[1] is False
    with pytest.raises(mm.MacroAIMError):                                     # equivalent surface not closed
        mm.mm_element_type_create(host_ctx, ms, ms, K0)
    mm.mm_mesh_destroy(ms)


def test_off_lattice_offsets_rejected(host_ctx, lib_c1):
    ty = lib_c1.types[0]
    with pytest.raises(mm.MacroAIMError) as e:
        mm.mm_array_create(host_ctx, [ty, ty], np.array([[0, 0, 0], [0.5123, 0, 0]]), 0.1, 2, 3,
                           wl.DEFAULT_GRID_PHASE)
    assert "integer multiples" in str(e.value)


def test_rounding_tie_rejected(host_ctx, lib_c1):
    # phase that puts the top-face centroids (z = 0.05) exactly on a rounding tie
    ty = lib_c1.types[0]
    with pytest.raises(mm.MacroAIMError):
        mm.mm_array_create(host_ctx, [ty], np.zeros((1, 3)), 0.1, 2, 3, (0.0137, 0.0291, 0.0))


def test_near_field_radius_options(host_ctx, lib_c1):
    """N_NF = -1 builds the far-field-only operator (no near-field rows); below -1 is refused."""
    ty = lib_c1.types[0]
    arr = mm.mm_array_create(host_ctx, [ty, ty], np.array([[0, 0, 0], [0.5, 0, 0]]), 0.1, 2, -1,
                             wl.DEFAULT_GRID_PHASE)
    assert mm.mm_array_info_get(arr)["nnz_near"] == 0
    mm.mm_array_destroy(arr)
    with pytest.raises(mm.MacroAIMError) as e:
        mm.mm_array_create(host_ctx, [ty], np.zeros((1, 3)), 0.1, 2, -2, wl.DEFAULT_GRID_PHASE)
    assert e.value.status == mm.MM_EINVAL


def test_near_blocks_reused_across_arrays_are_identical(host_ctx, lib_c1):
    """A second array over the same types takes its near-field blocks from the types'
    cache; its near field must equal the first array's (and the first array of a
    different size shares the blocks of the offsets they both hold)."""
    ty = lib_c1.types[0]
    lay2 = wl.loop_array(2, 3)
    fresh = mm.mm_array_create(host_ctx, [ty] * lay2.n_elem, lay2.offsets, 0.1, 2, 3, wl.DEFAULT_GRID_PHASE,
                               near_csr=1)
    again = mm.mm_array_create(host_ctx, [ty] * lay2.n_elem, lay2.offsets, 0.1, 2, 3, wl.DEFAULT_GRID_PHASE,
                               near_csr=1)
    try:
        for which in (mm.MM_EXPORT_NEAR_PTR, mm.MM_EXPORT_NEAR_COL, mm.MM_EXPORT_NEAR_VAL):
            assert np.array_equal(mm.mm_array_export(fresh, which), mm.mm_array_export(again, which))
        # the 2 x 2 array's first element row block equals the 2 x 3 array's for the same neighbours
        a_ptr = mm.mm_array_export(lib_c1.array, mm.MM_EXPORT_NEAR_PTR)
        a_val = mm.mm_array_export(lib_c1.array, mm.MM_EXPORT_NEAR_VAL)
        assert a_ptr[-1] > 0 and np.all(np.isfinite(a_val))
    finally:
        mm.mm_array_destroy(fresh)
        mm.mm_array_destroy(again)


def test_multiscale_type_matrices_match_oracle(host_ctx, meander_model):
    """The multiscale element (two conductors: the loop and a meandered trace with
    gaps as narrow as its cells) through the library's FP64 element build."""
    from paper_1712_02443_gb300.arrays import multiscale_array
    la = multiscale_array(host_ctx, 1, 1, meander=wl.MEANDER_REDUCED, box_div=wl.MEANDER_REDUCED_BOX)
    try:
        ty = la.types[0]
        assert mm.mm_type_info(ty) == (meander_model.rwg_s.n, meander_model.rwg_e.n)
        for which, R in ((mm.MM_MAT_M, meander_model.M), (mm.MM_MAT_D, meander_model.D),
                         (mm.MM_MAT_T, meander_model.T)):
            L = mm.mm_type_matrix(ty, which)
            assert np.abs(L - R).max() <= 1e-10 * np.abs(R).max(), which
    finally:
        la.close()


def test_block_jacobi_operator_matches_oracle(lib_c1, loop_model):
    """MM_MAT_PJ is the inverse of the element's own block D - G^(E^,H^) M, formed
    from the oracle's matrices by numpy's inverse."""
    ref = np.linalg.inv(loop_model.D - loop_model.G_hEH @ loop_model.M)
    L = mm.mm_type_matrix(lib_c1.types[0], mm.MM_MAT_PJ)
    assert np.abs(L - ref).max() <= 1e-9 * np.abs(ref).max()
