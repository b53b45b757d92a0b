"""The allocation-free solve entry point (eik_solve_noalloc), through the C ABI.

It serves callers that must not allocate device memory while solving; its
scratch is a fixed static array inside the library.  Its results must match
the ordinary eik_solve (caller workspace) within the FP32 tolerance of the
other parity tests, on two calls in a row (the second call reuses the array
left behind by the first), and the oracle's fast marching within the same
tolerance.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2106_15869_b300 import _lib
from paper_2106_15869_b300 import workloads as W

TOL32 = 1e-4


def _solve_both(inst):
    import torch
    lib = _lib.load()
    F = torch.as_tensor(inst.F, dtype=torch.float32).cuda().contiguous()
    idx = torch.as_tensor(inst.src_idx, dtype=torch.int64).cuda()
    val = torch.as_tensor(inst.src_val, dtype=torch.float32).cuda()
    nx, ny, nz = inst.dims
    g = _lib.grids_array([(nx, ny, nz, inst.h)])
    opt = _lib.make_options()
    stream = torch.cuda.current_stream().cuda_stream
    phi_na = torch.full_like(F, -1.0)
    st = _lib.eik_stats()
    rc = lib.eik_solve_noalloc(g, F.data_ptr(), idx.data_ptr(), val.data_ptr(), idx.numel(), phi_na.data_ptr(),
                               stream, ctypes.byref(opt), ctypes.byref(st))
    _lib.check(rc)
    nbytes = lib.eik_workspace_size(g, ctypes.byref(opt))
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    phi_ws = torch.full_like(F, -1.0)
    st2 = _lib.eik_stats()
    rc = lib.eik_solve(g, F.data_ptr(), idx.data_ptr(), val.data_ptr(), idx.numel(), phi_ws.data_ptr(),
                       ws.data_ptr(), nbytes, stream, ctypes.byref(opt), ctypes.byref(st2))
    _lib.check(rc)
    return phi_na.cpu().double().numpy(), phi_ws.cpu().double().numpy()


def _assert_close(a, b):
    fin = np.isfinite(b)
    assert np.array_equal(fin, np.isfinite(a))
    scale = float(np.max(np.abs(b[fin])))
    assert float(np.max(np.abs(a[fin] - b[fin]))) <= TOL32 * scale


@pytest.mark.gpu
def test_noalloc_matches_workspace_solve_twice():
    first = W.maze_3d(64, seed=3, n_slabs=4, gap=10, n_src=3)
    second = W.oscillating_3d(96)
    for inst in (first, second):
        a, b = _solve_both(inst)
        _assert_close(a, b)
        ref = oracle.fmm(inst.F.astype(np.float32).astype(np.float64), inst.h, inst.src_idx,
                         np.asarray(inst.src_val, np.float32).astype(np.float64))
        _assert_close(a, ref)


@pytest.mark.gpu
def test_noalloc_rejects_grids_beyond_the_static_scratch():
    import torch
    lib = _lib.load()
    g = _lib.grids_array([(512, 512, 512, 1.0 / 511)])
    opt = _lib.make_options()
    F = torch.ones(1, device="cuda")          # never read: the size check comes first
    rc = lib.eik_solve_noalloc(g, F.data_ptr(), None, None, 0, F.data_ptr(),
                               torch.cuda.current_stream().cuda_stream, ctypes.byref(opt), None)
    assert rc == _lib.EIK_ERR_ARG
    assert b"static scratch" in lib.eik_last_error()
