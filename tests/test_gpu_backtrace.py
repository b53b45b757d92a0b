"""GPU parity of the shortest-path back-trace (Example 4): the CUDA kernel and
the oracle's eko_backtrace follow the same steepest-descent rule on the same
phi array (the GPU solve's output), so the paths must be identical node for
node (integer output; the float decision is taken in double on both sides)."""
import numpy as np
import pytest

import oracle
from paper_2106_15869_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _run(inst, h, dtype, starts, max_len=4096, **kw):
    import torch
    from paper_2106_15869_b300 import api
    tdt = torch.float32 if dtype == "fp32" else torch.float64
    F = torch.as_tensor(inst.F, dtype=tdt).cuda()
    phi = api.solve(F, inst.src_idx, h, inst.src_val, **kw)
    path, length = api.backtrace(phi, starts, h, max_len=max_len)
    return phi.cpu().numpy(), path.cpu().numpy(), length.cpu().numpy()


def _check_same(phi, h, starts, path, length, max_len=4096):
    ref = oracle.backtrace(phi, h, starts, max_len=max_len)
    for q, r in enumerate(ref):
        assert length[q] == r.size, (q, length[q], r.size)
        assert np.array_equal(path[q, :r.size], r), q
        assert np.all(path[q, r.size:] == -1)
    return ref


@pytest.mark.parametrize("dtype", ["fp32", "fp64"])
def test_backtrace_maze_3d(dtype):
    inst = W.maze_3d(48, seed=7, n_slabs=3, gap=10, n_src=2)
    rng = np.random.default_rng(1)
    starts = rng.integers(0, inst.F.size, size=300)
    phi, path, length = _run(inst, inst.h, dtype, starts)
    ref = _check_same(phi, inst.h, starts, path, length)
    src = set(int(s) for s in inst.src_idx)
    flat = phi.reshape(-1)
    for q, r in enumerate(ref):
        if r.size:
            assert int(r[-1]) in src and np.all(np.diff(flat[r].astype(np.float64)) < 0)


def test_backtrace_paper_example_2d_and_unreachable():
    inst = W.paper_example_2d(3, n=150)
    F = inst.F.copy()
    F[70:80, 70:80] = 0.0                     # an impassable block: starts inside are unreachable
    inst.F = F
    starts = np.array([75 * 150 + 75, 0, 149 * 150 + 149, 10 * 150 + 140, 77 * 150 + 72], dtype=np.int64)
    phi, path, length = _run(inst, inst.h, "fp32", starts)
    _check_same(phi, inst.h, starts, path, length)
    assert length[0] == 0 and length[4] == 0 and np.all(length[1:4] > 1)


def test_backtrace_unequal_spacings_and_short_rows():
    inst = W.random_small(91, dims=(40, 33, 17), three_d=True, f_lo=0.3, f_hi=3.0)
    hs = (0.2, 0.05, 0.6)
    starts = np.arange(0, inst.F.size, 97, dtype=np.int64)
    phi, path, length = _run(inst, hs, "fp64", starts, max_len=8)
    _check_same(phi, hs, starts, path, length, max_len=8)
    assert np.all(length <= 8)


def test_backtrace_start_out_of_range():
    import torch
    from paper_2106_15869_b300 import api
    phi = torch.zeros((6, 7), dtype=torch.float32, device="cuda")
    path, length = api.backtrace(phi, [3, 42, -1, 41], 1.0, max_len=4)
    assert length.cpu().tolist() == [1, -1, -1, 1]
    assert path.cpu().tolist()[1] == [-1] * 4
