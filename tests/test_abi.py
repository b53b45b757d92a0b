"""CPU checks of the C ABI: the library builds, loads, exports every function
declared in include/*.h, and rejects bad arguments on the host before any
device work (no compute call needs a GPU here)."""
import ctypes
import glob
import os
import re

import pytest

from paper_2106_15869_b300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*(eik_[a-z_0-9]+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_builds_and_loads():
    build.build()
    lib = _lib.load()
    assert b"sm_103a" in lib.eik_version()


def test_every_declared_symbol_is_exported():
    lib = _lib.load()
    names = _declared_functions()
    assert {"eik_solve", "eik_solve_batched", "eik_workspace_size", "eik_last_error", "eik_adjoint",
            "eik_adjoint_batched", "eik_adjoint_workspace_size_batched", "eik_solve_noalloc",
            "eik_set_trace"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_struct_sizes_match_header_layout():
    # int64 x3 + double; int32,int32,int64,int32,int32,float,int32[3],float; 7 int64 + 2 int32 + 2 double
    assert ctypes.sizeof(_lib.eik_grid) == 48
    assert ctypes.sizeof(_lib.eik_options) == 48
    assert ctypes.sizeof(_lib.eik_stats) == 7 * 8 + 2 * 4 + 2 * 8


def _ws_size(dims, **kw):
    lib = _lib.load()
    g = _lib.grids_array([dims])
    o = _lib.make_options(**kw)
    return lib.eik_workspace_size(g, ctypes.byref(o))


def test_workspace_size_rules():
    n8 = _ws_size((256, 256, 256, 1 / 255))
    # phi and tau bricks dominate: 2 x 4 B per (padded) node, plus per-tile
    # state and the work queue (about 100 B per 4^3 tile)
    assert 2 * 4 * 256**3 <= n8 < 2 * 4 * 256**3 * 1.25
    assert _ws_size((256, 256, 256, 1 / 255), schedule="persistent") < n8
    assert _ws_size((256, 256, 256, 1 / 255), precision="fp64") > 1.7 * n8
    assert _ws_size((100, 50, 1, 0.1)) > 0                       # 2D -> 16x16x1 tiles
    assert _ws_size((100, 50, 3, 0.1), tile="16x16x1") == 0      # 2D tile on a 3D grid
    assert _ws_size((0, 5, 5, 0.1)) == 0
    assert _ws_size((5, 5, 5, 0.0)) == 0
    assert _ws_size((5, 5, 5, float("nan"))) == 0
    assert _ws_size((5, 5, 5, 1.0), precision=7) == 0
    # unequal spacings: hy, hz must be 0 (= h) or finite and > 0
    assert _ws_size((5, 5, 5, (1.0, 2.0, 3.0))) > 0
    assert _ws_size((5, 5, 5, (1.0, -2.0, 3.0))) == 0
    assert _ws_size((5, 5, 5, (1.0, 2.0, float("nan")))) == 0
    assert _ws_size((5, 5, 5, (1.0, 2.0, float("inf")))) == 0


def test_spacing_ratio_rules():
    lib = _lib.load()
    o = _lib.make_options()
    # every grid of one call shares hy/h and hz/h (the axis weights are per call)
    same = _lib.grids_array([(8, 8, 8, (0.1, 0.2, 0.3)), (9, 7, 5, (0.2, 0.4, 0.6))])
    assert lib.eik_workspace_size_batched(2, same, ctypes.byref(o)) > 0
    diff = _lib.grids_array([(8, 8, 8, (0.1, 0.2, 0.3)), (9, 7, 5, (0.2, 0.2, 0.6))])
    assert lib.eik_workspace_size_batched(2, diff, ctypes.byref(o)) == 0
    # a 2D grid has no z axis: its hz does not enter the comparison
    mixed = _lib.grids_array([(8, 8, 1, (0.1, 0.2, 5.0)), (9, 7, 5, (0.2, 0.4, 0.6))])
    assert lib.eik_workspace_size_batched(2, mixed, ctypes.byref(o)) > 0
    # equal spacings given explicitly are the isotropic case; the adjoint takes only those
    iso = _lib.grids_array([(8, 8, 8, (0.1, 0.1, 0.1))])
    assert lib.eik_adjoint_workspace_size_batched(1, iso, ctypes.byref(o)) > 0
    aniso = _lib.grids_array([(8, 8, 8, (0.1, 0.2, 0.1))])
    assert lib.eik_adjoint_workspace_size_batched(1, aniso, ctypes.byref(o)) == 0


def test_host_argument_errors_before_device_work():
    lib = _lib.load()
    g = _lib.grids_array([(8, 8, 8, 0.1)])
    o = _lib.make_options()
    st = _lib.eik_stats()
    # NULL workspace -> EIK_ERR_ARG without touching a device
    rc = lib.eik_solve(g, 1, None, None, 0, 1, None, 0, None, ctypes.byref(o), ctypes.byref(st))
    assert rc == _lib.EIK_ERR_ARG
    assert b"workspace" in lib.eik_last_error()
    # misaligned workspace
    rc = lib.eik_solve(g, 1, None, None, 0, 1, 4096 + 8, 1 << 30, None, ctypes.byref(o), None)
    assert rc == _lib.EIK_ERR_ARG and b"aligned" in lib.eik_last_error()
    # too small
    rc = lib.eik_solve(g, 1, None, None, 0, 1, 4096, 16, None, ctypes.byref(o), None)
    assert rc == _lib.EIK_ERR_ARG and b"too small" in lib.eik_last_error()
    # negative source count, bad dims
    assert lib.eik_solve(g, 1, None, None, -1, 1, 4096, 1 << 30, None, None, None) == _lib.EIK_ERR_ARG
    bad = _lib.grids_array([(8, 0, 8, 0.1)])
    assert lib.eik_solve(bad, 1, None, None, 0, 1, 4096, 1 << 30, None, None, None) == _lib.EIK_ERR_ARG
    # a negative wait limit is rejected; the method must be a known one
    o2 = _lib.make_options(wait_limit_us=-1)
    assert lib.eik_solve(g, 1, None, None, 0, 1, 4096, 1 << 30, None, ctypes.byref(o2), None) == _lib.EIK_ERR_ARG
    for m in (-1, 2):
        o3 = _lib.make_options(method=m)
        assert lib.eik_solve(g, 1, None, None, 0, 1, 4096, 1 << 30, None, ctypes.byref(o3), None) == _lib.EIK_ERR_ARG
        assert lib.eik_workspace_size(g, ctypes.byref(o3)) == 0
    assert lib.eik_workspace_size(g, ctypes.byref(_lib.make_options(method="fim"))) > 0
    # the Step-3 width: any number, not NaN
    assert lib.eik_workspace_size(g, ctypes.byref(_lib.make_options(remedy_order=float("nan")))) == 0
    for w in (-1.0, 2.0):
        assert lib.eik_workspace_size(g, ctypes.byref(_lib.make_options(remedy_order=w))) > 0
    # batched: decreasing source offsets
    gb = _lib.grids_array([(8, 8, 8, 0.1), (8, 8, 8, 0.1)])
    rc = lib.eik_solve_batched(2, gb, 1, _lib.i64_array([0, 0]), 1, 1, _lib.i64_array([0, 3, 2]), 1,
                               _lib.i64_array([0, 512]), 4096, 1 << 30, None, None, None)
    assert rc == _lib.EIK_ERR_ARG and b"non-decreasing" in lib.eik_last_error()


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libeikonal.so"))
    with pytest.raises(ImportError):
        _lib.load()


def test_backtrace_argument_errors_before_device_work():
    lib = _lib.load()
    g = _lib.grids_array([(8, 8, 8, 0.1)])
    E = _lib.EIK_ERR_ARG
    assert lib.eik_backtrace(g, 0, None, 1, 1, 4, 1, 1, None) == E                     # null phi
    assert lib.eik_backtrace(g, 7, 1, 1, 1, 4, 1, 1, None) == E                        # precision
    assert lib.eik_backtrace(g, 0, 1, 1, -1, 4, 1, 1, None) == E                       # n_paths
    assert lib.eik_backtrace(g, 0, 1, 1, 1, 0, 1, 1, None) == E                        # max_len
    assert lib.eik_backtrace(g, 0, 1, None, 1, 4, 1, 1, None) == E                     # null starts
    assert lib.eik_backtrace(g, 0, 1, 1, 1 << 20, 1 << 20, 1, 1, None) == E            # buffer too large
    bad = _lib.grids_array([(8, 8, 8, (0.1, -1.0, 0.1))])
    assert lib.eik_backtrace(bad, 0, 1, 1, 1, 4, 1, 1, None) == E                      # spacing
    assert lib.eik_backtrace(g, 0, 1, None, 0, 4, None, None, None) == _lib.EIK_OK     # nothing to do


def test_adjoint_gradient_blocks_equal_or_disjoint():
    """eik_adjoint_batched rejects gradient blocks that partly overlap, or that
    share an offset with different dims, before any device work."""
    lib = _lib.load()
    o = _lib.make_options()
    so = _lib.i64_array([0, 0, 0])
    zero = _lib.i64_array([0, 0])
    for dims, goff in (([(8, 8, 8, 0.1), (8, 8, 8, 0.1)], [0, 100]),
                       ([(8, 8, 8, 0.1), (8, 8, 4, 0.1)], [0, 0]),
                       ([(8, 8, 8, 0.1), (8, 8, 8, 0.1)], [600, 100])):
        g = _lib.grids_array(dims)
        rc = lib.eik_adjoint_batched(2, g, 4096, zero, 4096, zero, None, so, 4096, 4096, _lib.i64_array(goff),
                                     4096, 1 << 40, None, ctypes.byref(o), None)
        assert rc == _lib.EIK_ERR_ARG and b"gradient blocks" in lib.eik_last_error(), (dims, goff)
