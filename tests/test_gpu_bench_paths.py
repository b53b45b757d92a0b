"""Parity on the paths bench.py times, at the sizes it times them.

* Examples 1, 2, 3 and 5 of Sec. 4.1 at 1000^2 and Examples 2 and 5 at 2000^2
  and 4000^2 with the solver's default options (the 16x16x1 tile, whose
  persistent kernel takes an iteration either as a thread group per tile or,
  for lists longer than 8 entries per group, as a warp per tile: the
  throughput mode).  The per-iteration traces must show iterations in the
  throughput mode (Example 2's two fronts at 4000^2 list enough tiles;
  Example 5's single front may not), so that mode is compared with the
  oracle too.
* A 256^3 oscillating speed with eight sources on the non-default 8x8x4 tile
  (the same two-mode kernel in 3D), with throughput-mode iterations.

Every node is compared with the oracle's fast marching (FP64, fed the
FP32-rounded speeds and source values): FP32 within 1e-4 max phi, +inf exactly.
The oracle solves run in a thread pool on the host cores.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_2106_15869_b300 import workloads as W

pytestmark = pytest.mark.gpu
TOL32 = 1e-4


def _oracle32(inst):
    return oracle.fmm(inst.F.astype(np.float32).astype(np.float64), inst.h, inst.src_idx,
                      np.asarray(inst.src_val, np.float32).astype(np.float64))


def _gpu(inst, **kw):
    import torch
    from paper_2106_15869_b300 import api
    F = torch.as_tensor(inst.F, dtype=torch.float32).cuda()
    val = torch.as_tensor(np.asarray(inst.src_val, np.float64), dtype=torch.float32).cuda()
    with api.Trace() as tr:
        phi, st = api.solve(F, inst.src_idx, inst.h, val, return_stats=True, **kw)
    assert st["status"] == 0, st
    return phi.cpu().double().numpy(), tr


def _parity(got, ref):
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(got)), "reachability differs"
    scale = float(np.max(ref[fin]))
    err = float(np.max(np.abs(got[fin] - ref[fin])))
    assert err <= TOL32 * scale, (err, scale)
    return err / scale


def _throughput_iterations(tr) -> int:
    return int(np.sum((tr.records[1:, 1] & 256) != 0))


@pytest.mark.parametrize("ex", [1, 2, 3, 5])
def test_paper_examples_at_1000(ex):
    inst = W.paper_example_2d(ex, n=1000)
    got, _ = _gpu(inst)
    _parity(got, _oracle32(inst))


def test_paper_examples_at_2000_and_4000_throughput_mode():
    insts = [W.paper_example_2d(ex, n=n) for ex in (2, 5) for n in (2000, 4000)]
    with ThreadPoolExecutor(max_workers=4) as pool:
        refs = pool.map(_oracle32, insts)
        outs = [_gpu(i) for i in insts]
        refs = list(refs)
    thr = []
    for inst, (got, tr), ref in zip(insts, outs, refs):
        err = _parity(got, ref)
        thr.append(_throughput_iterations(tr))
        print(f"{inst.name}: max rel err {err:.2e}, throughput-mode iterations {thr[-1]}")
    # iterations in the throughput mode (a warp per tile) were compared with the oracle
    assert sum(thr) > 0, [tr.summary() for _, tr in outs]


def test_oscillating_256_tile_8x8x4_throughput_mode():
    base = W.oscillating_3d(256)
    rng = np.random.default_rng(17)
    idx = np.unique(rng.integers(0, base.F.size, size=8)).astype(np.int64)
    inst = W.Instance("osc256_8src", base.F, base.h, idx, np.zeros(idx.size))
    with ThreadPoolExecutor(max_workers=1) as pool:
        fut = pool.submit(_oracle32, inst)
        got, tr = _gpu(inst, tile="8x8x4")
        ref = fut.result()
    err = _parity(got, ref)
    assert _throughput_iterations(tr) > 0, tr.summary()
    print(f"osc256 8 sources, 8x8x4: max rel err {err:.2e}, {tr.summary()}")
