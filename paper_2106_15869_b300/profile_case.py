"""Run one named workload a fixed number of times, for a profiler to capture.

    python -m paper_2106_15869_b300.profile_case CASE [--calls N] [--stats] [--converge auto|confirm|sweep]
                                                 [--remedy-order W]

The cases are the benchmark workloads and smaller cases built by the same
recipes (for captures that replay a kernel many times, which want a few GB on
the device at most):

    maze_512, maze_256        the maze (16 / 8 slabs per axis), one solve per call
    oscillating_256           the 256^3 oscillating speed, one solve per call
    batch64, batch16          the lognormal batch (64 / first 16 instances), one batched solve per call
    tomo192_forward           16 shots of the 192^3 tomography, one batched forward per call
    tomo192_adjoint, tomo192_adjoint4
                              the batched adjoint of the 16 (4) shots, one call each (the forward
                              runs once before the calls)

Each call runs the library's kernels for that case once, so that e.g. ncu
`-k regex:k_persistent -s 2 -c 1` captures the third call's loop kernel.
With --stats every call also prints its statistics (this synchronises).
"""
from __future__ import annotations

import argparse
import json

import torch

from . import api, workloads as W


def _single(inst, dev, **kw):
    F = torch.as_tensor(inst.F, dtype=torch.float32).to(dev)
    val = torch.as_tensor(inst.src_val, dtype=torch.float32).to(dev)
    ws = api.Workspace(dev)
    phi = torch.empty_like(F)
    return lambda stats: api.solve(F, inst.src_idx, inst.h, val, workspace=ws, out=phi, return_stats=stats, **kw)


def _batch(insts, dev, **kw):
    probs = [(torch.as_tensor(i.F, dtype=torch.float32).to(dev), i.src_idx, i.h) for i in insts]
    ws = api.Workspace(dev)
    return lambda stats: api.solve_batched(probs, workspace=ws, return_stats=stats, **kw)


def _tomo(dev, shots: int, adjoint: bool):
    t = W.tomography_3d(192)
    F = torch.as_tensor(1.0 / t["s_init"], dtype=torch.float32).to(dev)
    probs = [(F, [int(s)], t["h"]) for s in t["sources"][:shots]]
    ws = api.Workspace(dev)
    if not adjoint:
        return lambda stats: api.solve_batched(probs, shared_F=True, workspace=ws, return_stats=stats)
    phis = api.solve_batched(probs, shared_F=True)
    rec = torch.as_tensor(t["receivers"]).to(dev)
    rs = []
    for ph in phis:
        r = torch.zeros_like(ph).reshape(-1)
        r[rec] = 1.0
        rs.append(r.view(ph.shape))
    return lambda stats: api.adjoint_batched(probs, phis, rs, shared_F=True, sum_instances=True, workspace=ws,
                                             return_stats=stats)


def make_case(name: str, dev, converge: str = "auto", remedy_order: float = 0.0):
    kw = dict(converge=converge, remedy_order=remedy_order)
    if name == "maze_512":
        return _single(W.maze_3d(512), dev, **kw)
    if name == "maze_256":
        return _single(W.maze_3d(256, n_slabs=8), dev, **kw)
    if name == "oscillating_256":
        return _single(W.oscillating_3d(256), dev, **kw)
    if name == "batch64":
        return _batch(W.lognormal_batch(64), dev, **kw)
    if name == "batch16":
        return _batch(W.lognormal_batch(64)[:16], dev, **kw)
    if name == "tomo192_forward":
        return _tomo(dev, 16, False)
    if name == "tomo192_adjoint":
        return _tomo(dev, 16, True)
    if name == "tomo192_adjoint4":
        return _tomo(dev, 4, True)
    raise SystemExit(f"unknown case {name}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case")
    ap.add_argument("--calls", type=int, default=3)
    ap.add_argument("--stats", action="store_true")
    ap.add_argument("--converge", default="auto", choices=["auto", "confirm", "sweep"],
                    help="Step-2 convergence test of the forward cases (the tomography keeps the default)")
    ap.add_argument("--remedy-order", type=float, default=0.0,
                    help="Step-3 list order of the forward cases (0 default, > 0 bucket width, < 0 unordered)")
    a = ap.parse_args()
    dev = torch.device("cuda", torch.cuda.current_device())
    run = make_case(a.case, dev, a.converge, a.remedy_order)
    for q in range(a.calls):
        out = run(a.stats)
        if a.stats:
            st = out[1]
            print(json.dumps({"case": a.case, "call": q, **st}), flush=True)
    torch.cuda.synchronize()


if __name__ == "__main__":
    main()
