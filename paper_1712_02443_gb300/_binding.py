"""ctypes binding of libmacroaim (argument marshalling only; every step runs in the library).

Each function has the name and argument order of its C entry point in
include/macroaim.h.  Handles are returned as ctypes void pointers; numpy arrays
are passed as host pointers, device buffers as integers (e.g. torch
``tensor.data_ptr()``), streams as integers (``torch.cuda.current_stream().cuda_stream``)
or None for the default stream.  A non-zero status raises MacroAIMError with the
context's message.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmacroaim.so")

MM_OK, MM_EINVAL, MM_ENOMEM, MM_ECUDA, MM_ENOCONV, MM_EBREAKDOWN, MM_ETIMEOUT, MM_EBUSY, MM_EINTERNAL = range(9)
STATUS_NAMES = ["MM_OK", "MM_EINVAL", "MM_ENOMEM", "MM_ECUDA", "MM_ENOCONV", "MM_EBREAKDOWN", "MM_ETIMEOUT",
                "MM_EBUSY", "MM_EINTERNAL"]
MM_C64, MM_C128, MM_C64_BF16, MM_C64_F16, MM_C128_FF = 0, 1, 2, 3, 4
MM_MAT_M, MM_MAT_D, MM_MAT_T, MM_MAT_A, MM_MAT_B, MM_MAT_GHH, MM_MAT_GHE, MM_MAT_PJ = range(8)
STAGES = ["gemm", "project", "fft_fwd", "fft_conv", "fft_inv", "interp", "near", "krylov"]
MM_EXPORT_ANCHORS, MM_EXPORT_PI, MM_EXPORT_NEAR_PTR, MM_EXPORT_NEAR_COL, MM_EXPORT_NEAR_VAL, MM_EXPORT_GHAT = range(6)


class MacroAIMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status, msg))


class mm_em_opts(ct.Structure):
    _fields_ = [("k0", ct.c_double), ("eta0", ct.c_double)]


class mm_aim_opts(ct.Structure):
    _fields_ = [("h", ct.c_double), ("order", ct.c_int32), ("n_nf", ct.c_int32), ("phase", ct.c_double * 3),
                ("near_csr", ct.c_int32)]


class mm_array_info(ct.Structure):
    _fields_ = [("n_unknowns", ct.c_int64), ("n_elem", ct.c_int64), ("n_types", ct.c_int64),
                ("grid", ct.c_int64 * 3), ("fft", ct.c_int64 * 3), ("nnz_near", ct.c_int64),
                ("device_bytes", ct.c_int64), ("n_scat_unknowns", ct.c_int64), ("n_near_blocks", ct.c_int64),
                ("near_block_entries", ct.c_int64), ("near_format", ct.c_int32)]


class mm_solve_opts(ct.Structure):
    _fields_ = [("tol", ct.c_double), ("restart", ct.c_int32), ("max_iter", ct.c_int32), ("precision", ct.c_int32),
                ("refine", ct.c_int32), ("inner_tol", ct.c_double), ("orth", ct.c_int32), ("precond", ct.c_int32),
                ("fp64", ct.c_int32)]


class mm_solve_stats(ct.Structure):
    _fields_ = [("iterations", ct.c_int32), ("matvecs", ct.c_int32), ("refinements", ct.c_int32),
                ("converged", ct.c_int32), ("rel_residual", ct.c_double)]


class mm_request(ct.Structure):
    _fields_ = [("n_elem", ct.c_int64), ("types", ct.POINTER(ct.c_void_p)), ("offsets_xyz", ct.c_void_p),
                ("aim", mm_aim_opts), ("nrhs", ct.c_int32), ("theta", ct.c_void_p), ("phi", ct.c_void_p),
                ("pol", ct.c_void_p), ("solve", mm_solve_opts)]


class mm_result(ct.Structure):
    _fields_ = [("done", ct.c_int32), ("status", ct.c_int32), ("n_unknowns", ct.c_int64),
                ("stats", mm_solve_stats), ("queue_s", ct.c_double), ("setup_s", ct.c_double),
                ("solve_s", ct.c_double), ("latency_s", ct.c_double), ("message", ct.c_char * 160),
                ("group_requests", ct.c_int32), ("group_columns", ct.c_int32)]


P = ct.c_void_p
PP = ct.POINTER(ct.c_void_p)
I64P = ct.POINTER(ct.c_int64)

_SIGS = {
    "mm_ctx_create": (ct.c_int, [ct.c_int, PP]),
    "mm_ctx_destroy": (None, [P]),
    "mm_last_error": (ct.c_char_p, [P]),
    "mm_ctx_set_threads": (ct.c_int, [P, ct.c_int]),
    "mm_mesh_create": (ct.c_int, [P, P, ct.c_int64, P, ct.c_int64, PP]),
    "mm_mesh_info": (ct.c_int, [P, I64P, ct.POINTER(ct.c_int32)]),
    "mm_mesh_destroy": (None, [P]),
    "mm_element_type_create": (ct.c_int, [P, P, P, ct.POINTER(mm_em_opts), PP]),
    "mm_type_matrix": (ct.c_int, [P, ct.c_int32, P, I64P, I64P]),
    "mm_type_info": (ct.c_int, [P, I64P, I64P]),
    "mm_type_destroy": (None, [P]),
    "mm_array_create": (ct.c_int, [P, ct.c_int64, PP, P, ct.POINTER(mm_aim_opts), PP]),
    "mm_array_info_get": (ct.c_int, [P, ct.POINTER(mm_array_info)]),
    "mm_array_footprint": (ct.c_int, [P, ct.c_int32, ct.c_int32, ct.c_int32, ct.POINTER(ct.c_size_t)]),
    "mm_array_export": (ct.c_int, [P, ct.c_int32, P, I64P]),
    "mm_array_destroy": (None, [P]),
    "mm_apply": (ct.c_int, [P, ct.c_int32, P, P, ct.c_int32, P]),
    "mm_apply_host": (ct.c_int, [P, ct.c_int32, P, P, ct.c_int32]),
    "mm_apply_noalloc": (ct.c_int, [P, ct.c_int32, P, P, ct.c_int32, P]),
    "mm_rhs_planewave": (ct.c_int, [P, ct.c_int32, P, P, P, P, ct.c_int32, P]),
    "mm_solve": (ct.c_int, [P, ct.c_int32, P, P, ct.POINTER(mm_solve_opts), ct.POINTER(mm_solve_stats), P]),
    "mm_currents": (ct.c_int, [P, ct.c_int32, P, P, P, P]),
    "mm_farfield": (ct.c_int, [P, ct.c_int32, P, ct.c_int64, P, P, P, P]),
    "mm_rcs": (ct.c_int, [P, ct.c_int32, P, ct.c_int64, P, P, P]),
    "mm_server_create": (ct.c_int, [ct.c_int, ct.c_int32, ct.c_size_t, PP]),
    "mm_server_submit": (ct.c_int, [P, ct.POINTER(mm_request), ct.POINTER(ct.c_uint64)]),
    "mm_server_poll": (ct.c_int, [P, ct.c_uint64, ct.c_int32, ct.POINTER(mm_result), P, ct.c_int64]),
    "mm_server_release": (ct.c_int, [P, ct.c_uint64]),
    "mm_server_destroy": (None, [P]),
    "mm_profile_enable": (ct.c_int, [P, ct.c_int32]),
    "mm_profile_stages": (ct.c_int, [P, ct.c_uint32]),
    "mm_profile_read": (ct.c_int, [P, ct.c_int32, ct.POINTER(ct.c_double), ct.POINTER(ct.c_int64)]),
    "mm_test_tc_stall": (ct.c_int, [ct.c_int32]),
    "mm_solve_planewave_host": (ct.c_int, [P, ct.c_int32, P, P, P, P, ct.POINTER(mm_solve_opts),
                                           ct.POINTER(mm_solve_stats)]),
    "mm_type_set_feed": (ct.c_int, [P, ct.c_int32, P, P]),
    "mm_apply_batch": (ct.c_int, [P, ct.c_int32, P, P, P, ct.c_int32, P]),
    "mm_batch_graphs": (ct.c_int, [P, P]),
    "mm_array_tuning": (ct.c_int, [P, ct.c_int32, ct.c_int32, P, P, P]),
    "mm_rhs_deltagap": (ct.c_int, [P, ct.c_int32, P, P, P]),
    "mm_currents_fed": (ct.c_int, [P, ct.c_int32, P, P, P, P, P]),
    "mm_rhs_planewave_ground": (ct.c_int, [P, ct.c_int32, P, P, P, ct.c_double, P, ct.c_int32, P]),
    "mm_array_near_shape": (ct.c_int, [P, ct.c_int32, ct.c_int32, ct.POINTER(ct.c_int32), ct.POINTER(ct.c_int32)]),
}

_lib = None


def load() -> ct.CDLL:
    """Loads the in-tree library; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libmacroaim.so is not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ct.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def exported_symbols():
    return list(_SIGS)


_ctx_of: dict = {}


def _check(status: int, ctx) -> None:
    if status != MM_OK:
        msg = load().mm_last_error(ctx).decode() if ctx else ""
        raise MacroAIMError(status, msg)


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, int):
        return ct.c_void_p(a)
    if hasattr(a, "data_ptr"):
        return ct.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous")
        return a.ctypes.data_as(ct.c_void_p)
    raise TypeError("unsupported buffer type %r" % type(a))


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return ct.c_void_p(s)
    return ct.c_void_p(s.cuda_stream)


# ---------------------------------------------------------------------------- entry points
def mm_ctx_create(device: int):
    h = ct.c_void_p()
    _check(load().mm_ctx_create(device, ct.byref(h)), None)
    return h


def mm_ctx_destroy(ctx) -> None:
    load().mm_ctx_destroy(ctx)


def mm_last_error(ctx) -> str:
    return load().mm_last_error(ctx).decode()


def mm_ctx_set_threads(ctx, n: int) -> None:
    _check(load().mm_ctx_set_threads(ctx, n), ctx)


def mm_mesh_create(ctx, xyz, tri):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    h = ct.c_void_p()
    _check(load().mm_mesh_create(ctx, _ptr(xyz), len(xyz), _ptr(tri), len(tri), ct.byref(h)), ctx)
    _ctx_of[h.value] = ctx
    return h


def mm_mesh_info(mesh):
    n = ct.c_int64()
    c = ct.c_int32()
    _check(load().mm_mesh_info(mesh, ct.byref(n), ct.byref(c)), _ctx_of.get(mesh.value))
    return n.value, bool(c.value)


def mm_mesh_destroy(mesh) -> None:
    load().mm_mesh_destroy(mesh)


def mm_element_type_create(ctx, scatterer, equiv, k0: float, eta0: float = 0.0):
    o = mm_em_opts(k0, eta0)
    h = ct.c_void_p()
    _check(load().mm_element_type_create(ctx, scatterer, equiv, ct.byref(o), ct.byref(h)), ctx)
    _ctx_of[h.value] = ctx
    return h


def mm_type_matrix(typ, which: int) -> np.ndarray:
    r, c = ct.c_int64(), ct.c_int64()
    ctx = _ctx_of.get(typ.value)
    _check(load().mm_type_matrix(typ, which, None, ct.byref(r), ct.byref(c)), ctx)
    out = np.zeros((r.value, c.value), dtype=np.complex128)
    _check(load().mm_type_matrix(typ, which, _ptr(out), ct.byref(r), ct.byref(c)), ctx)
    return out


def mm_type_info(typ):
    a, b = ct.c_int64(), ct.c_int64()
    _check(load().mm_type_info(typ, ct.byref(a), ct.byref(b)), _ctx_of.get(typ.value))
    return a.value, b.value


def mm_type_destroy(typ) -> None:
    load().mm_type_destroy(typ)


def mm_array_create(ctx, types, offsets, h: float, order: int, n_nf: int, phase, near_csr: int = 0):
    offsets = np.ascontiguousarray(offsets, dtype=np.float64).reshape(-1, 3)
    arr = (ct.c_void_p * len(types))(*[t.value for t in types])
    o = mm_aim_opts(h, order, n_nf, (ct.c_double * 3)(*phase), near_csr)
    hnd = ct.c_void_p()
    _check(load().mm_array_create(ctx, len(types), ct.cast(arr, PP), _ptr(offsets), ct.byref(o), ct.byref(hnd)), ctx)
    _ctx_of[hnd.value] = ctx
    return hnd


def mm_array_info_get(array) -> dict:
    i = mm_array_info()
    _check(load().mm_array_info_get(array, ct.byref(i)), _ctx_of.get(array.value))
    return {"n_unknowns": i.n_unknowns, "n_elem": i.n_elem, "n_types": i.n_types, "grid": tuple(i.grid),
            "fft": tuple(i.fft), "nnz_near": i.nnz_near, "device_bytes": i.device_bytes,
            "n_near_blocks": i.n_near_blocks, "near_block_entries": i.near_block_entries,
            "near_format": "csr" if i.near_format == 1 else "blocks",
            "n_scat_unknowns": i.n_scat_unknowns}


def mm_array_footprint(array, nrhs: int, precision: int, restart: int) -> int:
    b = ct.c_size_t()
    _check(load().mm_array_footprint(array, nrhs, precision, restart, ct.byref(b)), _ctx_of.get(array.value))
    return b.value


_EXPORT_DTYPE = {MM_EXPORT_ANCHORS: np.int64, MM_EXPORT_PI: np.float64, MM_EXPORT_NEAR_PTR: np.int64,
                 MM_EXPORT_NEAR_COL: np.int32, MM_EXPORT_NEAR_VAL: np.float64, MM_EXPORT_GHAT: np.float64}


def mm_array_export(array, which: int) -> np.ndarray:
    n = ct.c_int64()
    ctx = _ctx_of.get(array.value)
    _check(load().mm_array_export(array, which, None, ct.byref(n)), ctx)
    out = np.zeros(n.value, dtype=_EXPORT_DTYPE[which])
    _check(load().mm_array_export(array, which, _ptr(out), ct.byref(n)), ctx)
    if which in (MM_EXPORT_NEAR_VAL, MM_EXPORT_GHAT):
        out = out.view(np.complex128)
    return out


def mm_array_destroy(array) -> None:
    load().mm_array_destroy(array)


def mm_apply(array, nrhs: int, x_dev, y_dev, precision: int, stream=None) -> None:
    _check(load().mm_apply(array, nrhs, _ptr(x_dev), _ptr(y_dev), precision, _stream(stream)),
           _ctx_of.get(array.value))


def mm_apply_batch(arrays, nrhs, xs, ys, precision: int, stream=None) -> None:
    """Products of several arrays in one call; entry i: ys[i] = Z_i xs[i] with nrhs[i] columns."""
    n = len(arrays)
    ar = (ct.c_void_p * n)(*[a.value for a in arrays])
    nr = np.ascontiguousarray(nrhs, dtype=np.int32)
    xp = (ct.c_void_p * n)(*[_ptr(x) for x in xs])
    yp = (ct.c_void_p * n)(*[_ptr(y) for y in ys])
    _check(load().mm_apply_batch(ar, n, _ptr(nr), xp, yp, precision, _stream(stream)), _ctx_of.get(arrays[0].value))


def mm_batch_graphs(array=None) -> int:
    """Number of CUDA graphs mm_apply_batch holds for the array (None: all)."""
    n = ct.c_int32()
    _check(load().mm_batch_graphs(array, ct.byref(n)), _ctx_of.get(array.value) if array is not None else None)
    return n.value


def mm_apply_noalloc(array, nrhs: int, x_dev, y_dev, precision: int, stream=None) -> None:
    """mm_apply without any device allocation (shared static scratch of at most 16 MiB)."""
    _check(load().mm_apply_noalloc(array, nrhs, _ptr(x_dev), _ptr(y_dev), precision, _stream(stream)),
           _ctx_of.get(array.value))


def mm_test_tc_stall(ms: int) -> None:
    """Testing hook: ms > 0 makes tensor-core GEMMs issue no products and give up their waits after ms ms."""
    _check(load().mm_test_tc_stall(int(ms)), None)


def mm_apply_host(array, nrhs: int, x_host: np.ndarray, y_host: np.ndarray, precision: int) -> None:
    _check(load().mm_apply_host(array, nrhs, _ptr(x_host), _ptr(y_host), precision), _ctx_of.get(array.value))


def mm_rhs_planewave(array, theta, phi, pol, V_dev, precision: int, stream=None) -> None:
    th = np.ascontiguousarray(theta, dtype=np.float64).ravel()
    ph = np.ascontiguousarray(phi, dtype=np.float64).ravel()
    po = np.ascontiguousarray(pol, dtype=np.int32).ravel()
    _check(load().mm_rhs_planewave(array, len(th), _ptr(th), _ptr(ph), _ptr(po), _ptr(V_dev), precision,
                                   _stream(stream)), _ctx_of.get(array.value))


def mm_type_set_feed(type_, rwg, direction) -> None:
    """Delta-gap feed across the scatterer RWG edges `rwg` along `direction`."""
    r = np.ascontiguousarray(rwg, dtype=np.int64).ravel()
    d = np.ascontiguousarray(direction, dtype=np.float64).ravel()
    _check(load().mm_type_set_feed(type_, len(r), _ptr(r), _ptr(d)), _ctx_of.get(type_.value))


def mm_rhs_deltagap(array, volts, V_dev, stream=None) -> None:
    """V^_eff of the driven elements; volts (n_elem, nrhs) complex."""
    v = np.ascontiguousarray(volts, dtype=np.complex128)
    nrhs = v.shape[1] if v.ndim == 2 else 1
    _check(load().mm_rhs_deltagap(array, nrhs, _ptr(v), _ptr(V_dev), _stream(stream)), _ctx_of.get(array.value))


def mm_currents_fed(array, nrhs: int, E_dev, volts, J_dev=None, Jhat_dev=None, stream=None) -> None:
    v = np.ascontiguousarray(volts, dtype=np.complex128)
    _check(load().mm_currents_fed(array, nrhs, _ptr(E_dev), _ptr(v), _ptr(J_dev), _ptr(Jhat_dev), _stream(stream)),
           _ctx_of.get(array.value))


def mm_rhs_planewave_ground(array, theta, phi, pol, z_ground: float, V_dev, precision: int, stream=None) -> None:
    th = np.ascontiguousarray(theta, dtype=np.float64).ravel()
    ph = np.ascontiguousarray(phi, dtype=np.float64).ravel()
    po = np.ascontiguousarray(pol, dtype=np.int32).ravel()
    _check(load().mm_rhs_planewave_ground(array, len(th), _ptr(th), _ptr(ph), _ptr(po), float(z_ground), _ptr(V_dev),
                                          precision, _stream(stream)), _ctx_of.get(array.value))


def mm_currents(array, nrhs: int, E_dev, J_dev=None, Jhat_dev=None, stream=None) -> None:
    _check(load().mm_currents(array, nrhs, _ptr(E_dev), _ptr(J_dev), _ptr(Jhat_dev), _stream(stream)),
           _ctx_of.get(array.value))


def mm_farfield(array, nrhs: int, Jhat_dev, theta, phi, F_dev, stream=None) -> None:
    th = np.ascontiguousarray(theta, dtype=np.float64).ravel()
    ph = np.ascontiguousarray(phi, dtype=np.float64).ravel()
    _check(load().mm_farfield(array, nrhs, _ptr(Jhat_dev), len(th), _ptr(th), _ptr(ph), _ptr(F_dev), _stream(stream)),
           _ctx_of.get(array.value))


def mm_rcs(array, nrhs: int, Jhat_dev, theta, phi) -> np.ndarray:
    th = np.ascontiguousarray(theta, dtype=np.float64).ravel()
    ph = np.ascontiguousarray(phi, dtype=np.float64).ravel()
    out = np.zeros((len(th), nrhs), dtype=np.float64)
    _check(load().mm_rcs(array, nrhs, _ptr(Jhat_dev), len(th), _ptr(th), _ptr(ph), _ptr(out)),
           _ctx_of.get(array.value))
    return out


def mm_solve(array, nrhs: int, V_dev, E_dev, tol: float, restart: int = 50, max_iter: int = 1000,
             precision: int = MM_C64, refine: int = 1, inner_tol: float = 1e-2, stream=None, check: bool = True,
             orth: int = 0, precond: int = 0, fp64: int = 0):
    o = mm_solve_opts(tol, restart, max_iter, precision, refine, inner_tol, orth, precond, fp64)
    s = mm_solve_stats()
    st = load().mm_solve(array, nrhs, _ptr(V_dev), _ptr(E_dev), ct.byref(o), ct.byref(s), _stream(stream))
    stats = {"iterations": s.iterations, "matvecs": s.matvecs, "refinements": s.refinements,
             "converged": bool(s.converged), "rel_residual": s.rel_residual, "status": st}
    if check:
        _check(st, _ctx_of.get(array.value))
    return stats


def mm_solve_planewave_host(array, theta, phi, pol, E_host: np.ndarray, tol: float, restart: int = 50,
                            max_iter: int = 1000, precision: int = MM_C64, refine: int = 1, inner_tol: float = 1e-2,
                            orth: int = 0, precond: int = 0, check: bool = True, fp64: int = 0):
    """Excitation, solve and the solution copied into E_host (complex128, N x nrhs), all in the library."""
    th = np.ascontiguousarray(theta, dtype=np.float64).ravel()
    ph = np.ascontiguousarray(phi, dtype=np.float64).ravel()
    po = np.ascontiguousarray(pol, dtype=np.int32).ravel()
    if E_host.dtype != np.complex128 or not E_host.flags.c_contiguous:
        raise ValueError("E_host must be a C-contiguous complex128 array")
    o = mm_solve_opts(tol, restart, max_iter, precision, refine, inner_tol, orth, precond, fp64)
    s = mm_solve_stats()
    st = load().mm_solve_planewave_host(array, len(th), _ptr(th), _ptr(ph), _ptr(po), _ptr(E_host), ct.byref(o),
                                        ct.byref(s))
    stats = {"iterations": s.iterations, "matvecs": s.matvecs, "refinements": s.refinements,
             "converged": bool(s.converged), "rel_residual": s.rel_residual, "status": st}
    if check:
        _check(st, _ctx_of.get(array.value))
    return stats


def mm_array_near_shape(array, nrhs: int, precision: int = MM_C64):
    """(shape, ksplit) of the block near-field kernel chosen for nrhs columns, or None before the first product."""
    sh, ks = ct.c_int32(), ct.c_int32()
    st = load().mm_array_near_shape(array, nrhs, precision, ct.byref(sh), ct.byref(ks))
    return (sh.value, ks.value) if st == MM_OK else None


def mm_array_tuning(array, nrhs: int, precision: int = MM_C64):
    """The array's launch choices for nrhs columns (near shape, k split, projection and
    interpolation schedules) and the grid tuner's timings, or None before the first product."""
    ch = np.zeros(4, dtype=np.int32)
    pm = np.zeros(4, dtype=np.float32)
    im = np.zeros(4, dtype=np.float32)
    st = load().mm_array_tuning(array, nrhs, precision, _ptr(ch), _ptr(pm), _ptr(im))
    if st != MM_OK:
        return None

    def times(a):   # per variant, None where the variant was not timed; trailing untimed ones dropped
        t = [float(x) if x >= 0 else None for x in a]
        while t and t[-1] is None:
            t.pop()
        return t
    return {"near_shape": int(ch[0]), "near_ksplit": int(ch[1]), "project": int(ch[2]), "interp": int(ch[3]),
            "project_ms": times(pm), "interp_ms": times(im)}


def mm_profile_enable(array, enable: bool = True) -> None:
    _check(load().mm_profile_enable(array, 1 if enable else 0), _ctx_of.get(array.value))


def mm_profile_stages(array, stages=None) -> None:
    """Record only the named stages (None: all)."""
    mask = 0xFF if stages is None else sum(1 << STAGES.index(s) for s in stages)
    _check(load().mm_profile_stages(array, mask), _ctx_of.get(array.value))


def mm_profile_read(array, precision: int = -1) -> dict:
    ms = (ct.c_double * len(STAGES))()
    nl = (ct.c_int64 * len(STAGES))()
    _check(load().mm_profile_read(array, precision, ms, nl), _ctx_of.get(array.value))
    return {name: {"ms": ms[i], "launches": nl[i]} for i, name in enumerate(STAGES)}


# ---------------------------------------------------------------------------- server
def mm_server_create(device: int = 0, workers: int = 2, hbm_budget_bytes: int = 0):
    h = ct.c_void_p()
    _check(load().mm_server_create(device, workers, hbm_budget_bytes, ct.byref(h)), None)
    return h


def mm_server_submit(server, types, offsets, theta, phi, pol, tol: float, h: float = 0.1, order: int = 2,
                     n_nf: int = 3, phase=(0.0137, 0.0291, 0.0913), restart: int = 50, max_iter: int = 2000,
                     precision: int = MM_C64, refine: int = 1, inner_tol: float = 1e-5, precond: int = 0,
                     near_csr: int = 0) -> int:
    """Submits one request; its inputs are copied before this returns."""
    offsets = np.ascontiguousarray(offsets, dtype=np.float64).reshape(-1, 3)
    th = np.ascontiguousarray(theta, dtype=np.float64).ravel()
    ph = np.ascontiguousarray(phi, dtype=np.float64).ravel()
    po = np.ascontiguousarray(pol, dtype=np.int32).ravel()
    arr = (ct.c_void_p * len(types))(*[t.value for t in types])
    q = mm_request(len(types), ct.cast(arr, ct.POINTER(ct.c_void_p)), offsets.ctypes.data_as(ct.c_void_p),
                   mm_aim_opts(h, order, n_nf, (ct.c_double * 3)(*phase), near_csr), len(th),
                   th.ctypes.data_as(ct.c_void_p),
                   ph.ctypes.data_as(ct.c_void_p), po.ctypes.data_as(ct.c_void_p),
                   mm_solve_opts(tol, restart, max_iter, precision, refine, inner_tol, 0, precond))
    t = ct.c_uint64()
    _check(load().mm_server_submit(server, ct.byref(q), ct.byref(t)), None)
    return t.value


def mm_server_poll(server, ticket: int, wait: bool = True, nrhs: int = 1, want_solution: bool = True):
    """Returns (result dict, E or None); result['done'] is False while it runs."""
    r = mm_result()
    st = load().mm_server_poll(server, ticket, 1 if wait else 0, ct.byref(r), None, 0)
    if st == MM_EBUSY:
        return {"done": False}, None
    _check(st, None)
    E = None
    if want_solution and r.status in (MM_OK, MM_ENOCONV):
        buf = np.zeros(2 * r.n_unknowns * nrhs, dtype=np.float64)
        _check(load().mm_server_poll(server, ticket, 1, ct.byref(r), buf.ctypes.data_as(ct.c_void_p), len(buf)), None)
        E = buf.view(np.complex128).reshape(r.n_unknowns, nrhs)
    res = {"done": True, "status": r.status, "n_unknowns": r.n_unknowns, "iterations": r.stats.iterations,
           "matvecs": r.stats.matvecs, "converged": bool(r.stats.converged), "rel_residual": r.stats.rel_residual,
           "queue_s": r.queue_s, "setup_s": r.setup_s, "solve_s": r.solve_s, "latency_s": r.latency_s,
           "message": r.message.decode(errors="replace"), "group_requests": r.group_requests,
           "group_columns": r.group_columns}
    return res, E


def mm_server_release(server, ticket: int) -> None:
    _check(load().mm_server_release(server, ticket), None)


def mm_server_destroy(server) -> None:
    load().mm_server_destroy(server)
