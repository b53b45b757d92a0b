"""Failure detection without a GPU fault: every device-side wait of a call (grid
barriers of the persistent kernels, slots of the asynchronous work queue) is
bounded by eik_options.wait_limit_us.  A limit of 1 us is far below one tile
visit (several us of staging and sweeps), so the thread blocks that wait at the
first barrier for the block visiting the source tile give up: the call must
report EIK_ERR_DEVICE with device flag bit 1 (wait timeout), every block leaves
the launch, and phi holds valid upper bounds of the solution (the values are
relaxations from +inf, never below the discrete solution).  The next call on the
same workspace must solve normally: the failure leaves nothing behind.  Nothing
here traps, faults or hangs a GPU: the waits end by their own limit.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2106_15869_b300 import workloads as W

pytestmark = pytest.mark.gpu
TOL32 = 1e-4


def _ref(inst):
    return oracle.fmm(inst.F.astype(np.float32).astype(np.float64), inst.h, inst.src_idx,
                      np.asarray(inst.src_val, np.float32).astype(np.float64))


@pytest.mark.parametrize("schedule", ["persistent", "async"])
@pytest.mark.parametrize("method", ["ifim", "fim"])
def test_wait_limit_runs_out_and_the_next_call_recovers(schedule, method):
    import torch
    from paper_2106_15869_b300 import api, _lib
    inst = W.oscillating_3d(40)
    ref = _ref(inst)
    fin = np.isfinite(ref)
    scale = float(ref[fin].max())
    F = torch.as_tensor(inst.F, dtype=torch.float32).cuda()
    ws = api.Workspace()
    with pytest.raises(_lib.EikonalError) as e:
        api.solve(F, inst.src_idx, inst.h, schedule=schedule, method=method, wait_limit_us=1, workspace=ws,
                  return_stats=True)
    assert e.value.code == _lib.EIK_ERR_DEVICE
    assert "timed out" in str(e.value)
    # the same call through the C ABI, to read its flags and the phi it leaves behind
    out = torch.full_like(F, -1.0)
    lib = _lib.load()
    nx, ny, nz = inst.dims
    g = _lib.grids_array([(nx, ny, nz, inst.h)])
    opt = _lib.make_options(schedule=schedule, method=method, wait_limit_us=1)
    nbytes = lib.eik_workspace_size(g, ctypes.byref(opt))
    buf = ws.get(nbytes)
    idx = torch.as_tensor(inst.src_idx).cuda()
    val = torch.zeros(idx.numel(), device="cuda")
    stt = _lib.eik_stats()
    rc = lib.eik_solve(g, F.data_ptr(), idx.data_ptr(), val.data_ptr(), idx.numel(), out.data_ptr(), buf.data_ptr(),
                       buf.numel(), torch.cuda.current_stream().cuda_stream, ctypes.byref(opt), ctypes.byref(stt))
    assert rc == _lib.EIK_ERR_DEVICE
    assert stt.device_flags & 2, stt.device_flags
    got = out.cpu().double().numpy()
    assert not np.any(got == -1.0)                       # the output was written completely
    assert np.all(got[fin] >= ref[fin] - TOL32 * scale)  # upper bounds of the solution
    assert np.any(np.isinf(got[fin]))                    # the launch ended before the front reached everything
    # the next call on the same workspace, default limit: a normal solve
    phi2, st2 = api.solve(F, inst.src_idx, inst.h, schedule=schedule, method=method, workspace=ws,
                          return_stats=True)
    assert st2["status"] == 0 and st2["device_flags"] == 0
    got2 = phi2.cpu().double().numpy()
    assert np.array_equal(np.isfinite(got2), fin)
    assert np.max(np.abs(got2[fin] - ref[fin])) <= TOL32 * scale


def test_wait_limit_in_the_adjoint():
    import torch
    from paper_2106_15869_b300 import api, _lib
    inst = W.oscillating_3d(40)
    F = torch.as_tensor(inst.F, dtype=torch.float64).cuda()
    phi = api.solve(F, inst.src_idx, inst.h)
    r = torch.zeros_like(phi)
    r[-1] = 1.0
    ws = api.Workspace()
    with pytest.raises(_lib.EikonalError) as e:
        api.adjoint_batched([(F, inst.src_idx, inst.h)], [phi], [r], wait_limit_us=1, workspace=ws,
                            return_stats=True)
    assert e.value.code == _lib.EIK_ERR_DEVICE
    # the next call recovers and matches the oracle's adjoint on the same phi
    g = api.adjoint_batched([(F, inst.src_idx, inst.h)], [phi], [r], workspace=ws)[0]
    want = oracle.adjoint(inst.F, inst.h, inst.src_idx, phi.cpu().numpy(), r.cpu().numpy())
    got = g.cpu().numpy()
    assert np.max(np.abs(got - want)) <= 1e-10 * np.max(np.abs(want))


def test_negative_wait_limit_is_an_argument_error():
    import torch
    from paper_2106_15869_b300 import api, _lib
    F = torch.ones(8, 8, 8, device="cuda")
    with pytest.raises(_lib.EikonalError) as e:
        api.solve(F, [0], 0.1, wait_limit_us=-5)
    assert e.value.code == _lib.EIK_ERR_ARG
