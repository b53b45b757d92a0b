"""ctypes binding of libeikonal.so: the C structs of include/eikonal.h and the
entry points with the same names.  Argument marshalling only -- every step
of the solve runs in the CUDA library.  Loading fails loudly when the
library is missing or does not load; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libeikonal.so")
# the same library with device-side index and NaN checks (compiled with -DEIK_DEBUG)
LIB_DEBUG_PATH = os.path.join(HERE, "libeikonal_debug.so")

EIK_OK = 0
EIK_ERR_ARG = 1
EIK_ERR_NOCONVERGE = 2
EIK_ERR_CUDA = 3
EIK_ERR_DEVICE = 4

TILES = {"auto": 0, "8x8x8": 1, "4x4x4": 2, "8x8x4": 3, "16x16x1": 4, "8x4x4": 5, "8x8x1": 6}
SCHEDULES = {"auto": 0, "persistent": 1, "hostloop": 2, "async": 3}
PRECISIONS = {"fp32": 0, "fp64": 1}
CONVERGE = {"auto": 0, "confirm": 1, "sweep": 2}
METHODS = {"ifim": 0, "fim": 1}


class eik_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64),
                ("h", ctypes.c_double), ("hy", ctypes.c_double), ("hz", ctypes.c_double)]


class eik_options(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("max_iters", ctypes.c_int64), ("precision", ctypes.c_int32),
                ("skip_remedy", ctypes.c_int32), ("order", ctypes.c_float),
                ("converge", ctypes.c_int32), ("method", ctypes.c_int32), ("wait_limit_us", ctypes.c_int32),
                ("remedy_order", ctypes.c_float)]


class eik_stats(ctypes.Structure):
    _fields_ = [("iters_update", ctypes.c_int64), ("iters_remedy", ctypes.c_int64),
                ("tiles_update", ctypes.c_int64), ("tiles_flagged", ctypes.c_int64),
                ("tiles_remedy", ctypes.c_int64), ("sweeps", ctypes.c_int64),
                ("tiles_deferred", ctypes.c_int64),
                ("status", ctypes.c_int32), ("device_flags", ctypes.c_int32),
                ("ms_total", ctypes.c_double), ("ms_loop", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class EikonalError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"eikonal error {code}: {msg}")
        self.code = code


_lib = None
_lib_debug = None
_vp = ctypes.c_void_p
_sz = ctypes.c_size_t
_i64 = ctypes.c_int64
_pi64 = ctypes.POINTER(ctypes.c_int64)


def load():
    """Load libeikonal.so (built in-tree by paper_2106_15869_b300.build)."""
    global _lib
    if _lib is None:
        _lib = _open(LIB_PATH)
    return _lib


def load_debug():
    """Load libeikonal_debug.so: the same entry points, with the device-side checks of the
    debug build (a tile id out of range or a NaN in phi/lambda raises a device flag and
    the call returns EIK_ERR_DEVICE; nothing traps).  For tests and diagnosis."""
    global _lib_debug
    if _lib_debug is None:
        _lib_debug = _open(LIB_DEBUG_PATH)
    return _lib_debug


def _open(path):
    if not os.path.exists(path):
        raise ImportError(f"{os.path.basename(path)} is not built ({path}); run "
                          "`python -m paper_2106_15869_b300.build` (needs nvcc)")
    lib = ctypes.CDLL(path)
    G = ctypes.POINTER(eik_grid)
    O = ctypes.POINTER(eik_options)
    S = ctypes.POINTER(eik_stats)
    lib.eik_workspace_size.restype = _sz
    lib.eik_workspace_size.argtypes = [G, O]
    lib.eik_workspace_size_batched.restype = _sz
    lib.eik_workspace_size_batched.argtypes = [_i64, G, O]
    lib.eik_solve.restype = ctypes.c_int
    lib.eik_solve.argtypes = [G, _vp, _vp, _vp, _i64, _vp, _vp, _sz, _vp, O, S]
    lib.eik_solve_batched.restype = ctypes.c_int
    lib.eik_solve_batched.argtypes = [_i64, G, _vp, _pi64, _vp, _vp, _pi64, _vp, _pi64, _vp, _sz,
                                      _vp, O, S]
    lib.eik_last_error.restype = ctypes.c_char_p
    lib.eik_last_error.argtypes = []
    lib.eik_version.restype = ctypes.c_char_p
    lib.eik_version.argtypes = []
    _optional_symbols(lib)
    return lib


def _optional_symbols(lib):
    """Declare signatures of entry points added after the forward solve."""
    G = ctypes.POINTER(eik_grid)
    O = ctypes.POINTER(eik_options)
    S = ctypes.POINTER(eik_stats)
    if hasattr(lib, "eik_set_trace"):
        lib.eik_set_trace.restype = ctypes.c_int
        lib.eik_set_trace.argtypes = [_vp, _i64]
    if hasattr(lib, "eik_solve_noalloc"):
        lib.eik_solve_noalloc.restype = ctypes.c_int
        lib.eik_solve_noalloc.argtypes = [G, _vp, _vp, _vp, _i64, _vp, _vp, O, S]
    if hasattr(lib, "eik_adjoint_workspace_size_batched"):
        lib.eik_adjoint_workspace_size_batched.restype = _sz
        lib.eik_adjoint_workspace_size_batched.argtypes = [_i64, G, O]
    if hasattr(lib, "eik_adjoint_batched"):
        lib.eik_adjoint_batched.restype = ctypes.c_int
        lib.eik_adjoint_batched.argtypes = [_i64, G, _vp, _pi64, _vp, _pi64, _vp, _pi64, _vp, _vp, _pi64,
                                            _vp, _sz, _vp, O, S]
    if hasattr(lib, "eik_adjoint"):
        lib.eik_adjoint.restype = ctypes.c_int
        lib.eik_adjoint.argtypes = [G, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _sz, _vp, O, S]
    if hasattr(lib, "eik_backtrace"):
        lib.eik_backtrace.restype = ctypes.c_int
        lib.eik_backtrace.argtypes = [G, ctypes.c_int, _vp, _vp, _i64, _i64, _vp, _vp, _vp]


def check(rc: int, lib=None):
    if rc != EIK_OK:
        msg = (lib or load()).eik_last_error().decode(errors="replace")
        raise EikonalError(rc, msg)


def make_options(tile="auto", schedule="auto", precision="fp32", skip_remedy=False,
                 max_iters=0, order=0.0, converge="auto", method="ifim", wait_limit_us=0,
                 remedy_order=0.0) -> eik_options:
    o = eik_options()
    o.tile = TILES[tile] if isinstance(tile, str) else int(tile)
    o.schedule = SCHEDULES[schedule] if isinstance(schedule, str) else int(schedule)
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.skip_remedy = int(bool(skip_remedy))
    o.max_iters = int(max_iters)
    o.order = float(order)
    o.converge = CONVERGE[converge] if isinstance(converge, str) else int(converge)
    o.method = METHODS[method] if isinstance(method, str) else int(method)
    o.wait_limit_us = int(wait_limit_us)
    o.remedy_order = float(remedy_order)
    return o


def spacing(h):
    """h as a number or per axis (hx, hy[, hz]) -> (h, hy, hz) of eik_grid (0 = same as h)."""
    if isinstance(h, (int, float)) or getattr(h, "ndim", 1) == 0:
        return float(h), 0.0, 0.0
    hs = [float(v) for v in h]
    if len(hs) == 2:
        hs.append(0.0)
    if len(hs) != 3:
        raise ValueError("h must be a number or (hx, hy[, hz])")
    return hs[0], hs[1], hs[2]


def grids_array(dims_h):
    """[(nx, ny, nz, h), ...] -> ctypes array of eik_grid; h a number or (hx, hy[, hz])."""
    arr = (eik_grid * len(dims_h))()
    for q, (nx, ny, nz, h) in enumerate(dims_h):
        arr[q].nx, arr[q].ny, arr[q].nz = int(nx), int(ny), int(nz)
        arr[q].h, arr[q].hy, arr[q].hz = spacing(h)
    return arr


def i64_array(vals):
    arr = (ctypes.c_int64 * len(vals))()
    for q, v in enumerate(vals):
        arr[q] = int(v)
    return arr
