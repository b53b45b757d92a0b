"""The checked build (libeikonal_debug.so, compiled with -DEIK_DEBUG) on the small
odd-shaped and random parity cases, through the C ABI.

In that build every tile id read from a list, a visit record or the work queue
is checked against the tile count before use, and every value written back to
phi or lambda is checked for NaN; a failed check raises a device flag and makes
the call return EIK_ERR_DEVICE (nothing traps).  These cases must pass every
check (status EIK_OK, device flags 0) and still match the oracle: FP64 within
1e-10 of max phi, FP32 within 1e-4.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2106_15869_b300 import _lib
from paper_2106_15869_b300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = {"fp32": 1e-4, "fp64": 1e-10}


def _solve_debug(inst, dtype, **opts):
    import torch
    lib = _lib.load_debug()
    tdt = torch.float32 if dtype == "fp32" else torch.float64
    F = torch.as_tensor(inst.F, dtype=tdt).cuda().contiguous()
    idx = torch.as_tensor(np.asarray(inst.src_idx, np.int64)).cuda()
    val = torch.as_tensor(np.asarray(inst.src_val, np.float64), dtype=tdt).cuda()
    nx, ny, nz = inst.dims
    g = _lib.grids_array([(nx, ny, nz, inst.h)])
    opt = _lib.make_options(precision=dtype, **opts)
    nbytes = lib.eik_workspace_size(g, ctypes.byref(opt))
    assert nbytes > 0
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    phi = torch.full_like(F, -1.0)
    st = _lib.eik_stats()
    rc = lib.eik_solve(g, F.data_ptr(), idx.data_ptr() if idx.numel() else None,
                       val.data_ptr() if idx.numel() else None, idx.numel(), phi.data_ptr(), ws.data_ptr(), nbytes,
                       torch.cuda.current_stream().cuda_stream, ctypes.byref(opt), ctypes.byref(st))
    _lib.check(rc, lib)
    assert st.status == 0 and st.device_flags == 0, (st.status, st.device_flags)
    return phi.cpu().double().numpy()


def _oracle(inst, dtype):
    F = inst.F.astype(np.float32).astype(np.float64) if dtype == "fp32" else inst.F
    val = np.asarray(inst.src_val, np.float32).astype(np.float64) if dtype == "fp32" else inst.src_val
    return oracle.fmm(F, inst.h, inst.src_idx, val)


def _parity(got, ref, tol):
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(got))
    if fin.any():
        assert np.max(np.abs(got[fin] - ref[fin])) <= tol * np.max(np.abs(ref[fin]))


@pytest.mark.parametrize("dims", [(1, 1, 1), (1, 1, 9), (17, 1, 1), (9, 9, 1), (3, 5, 7), (9, 8, 8), (16, 16, 17),
                                  (13, 7, 5)])
@pytest.mark.parametrize("dtype", ["fp64", "fp32"])
def test_debug_build_odd_shapes(dims, dtype):
    inst = W.random_small(31, dims=dims, three_d=dims[2] > 1)
    _parity(_solve_debug(inst, dtype), _oracle(inst, dtype), TOL[dtype])


@pytest.mark.parametrize("seed", range(6))
def test_debug_build_random_grids_every_schedule_and_method(seed):
    inst = W.random_small(300 + seed, max_edge=23, p_barrier=0.08 if seed % 2 else 0.0)
    ref = _oracle(inst, "fp64")
    for opts in (dict(), dict(schedule="hostloop"), dict(schedule="async"), dict(method="fim"),
                 dict(tile="4x4x4", order=-1.0), dict(tile="8x8x4")):
        if opts.get("tile") and inst.dims[2] == 1:
            continue
        _parity(_solve_debug(inst, "fp64", **opts), ref, TOL["fp64"])


def test_debug_build_multi_source_two_phase_and_2d_example():
    base = W.oscillating_3d(96)
    rng = np.random.default_rng(3)
    idx = np.unique(rng.integers(0, base.F.size, size=12)).astype(np.int64)
    inst = W.Instance("osc96_multi", base.F, base.h, idx, np.zeros(idx.size))
    _parity(_solve_debug(inst, "fp32"), _oracle(inst, "fp32"), TOL["fp32"])
    ex = W.paper_example_2d(5, n=300)
    _parity(_solve_debug(ex, "fp32"), _oracle(ex, "fp32"), TOL["fp32"])


def test_debug_build_adjoint():
    import torch
    lib = _lib.load_debug()
    inst = W.random_small(808, dims=(19, 14, 11), three_d=True, f_lo=0.3, f_hi=3.0)
    inst.src_val[:] = 0.0
    phi = oracle.fmm(inst.F, inst.h, inst.src_idx)
    rng = np.random.default_rng(8)
    r = np.where(np.isfinite(phi) & (rng.random(phi.shape) < 0.3), rng.standard_normal(phi.shape), 0.0)
    want = oracle.adjoint(inst.F, inst.h, inst.src_idx, phi, r)
    nx, ny, nz = inst.dims
    g = _lib.grids_array([(nx, ny, nz, inst.h)])
    opt = _lib.make_options(precision="fp64")
    nbytes = lib.eik_adjoint_workspace_size_batched(1, g, ctypes.byref(opt))
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    F_d = torch.as_tensor(inst.F).cuda()
    phi_d = torch.as_tensor(phi).cuda()
    r_d = torch.as_tensor(r).cuda()
    out = torch.zeros_like(F_d)
    idx = torch.as_tensor(np.asarray(inst.src_idx, np.int64)).cuda()
    st = _lib.eik_stats()
    rc = lib.eik_adjoint(g, F_d.data_ptr(), phi_d.data_ptr(), idx.data_ptr(), idx.numel(), r_d.data_ptr(),
                         out.data_ptr(), ws.data_ptr(), nbytes, torch.cuda.current_stream().cuda_stream,
                         ctypes.byref(opt), ctypes.byref(st))
    _lib.check(rc, lib)
    assert st.device_flags == 0
    got = out.cpu().numpy()
    assert np.max(np.abs(got - want)) <= 1e-10 * np.max(np.abs(want))
