"""Autotuner: cache keys (CPU) and a tuned solve on the GPU."""
import json

import numpy as np
import pytest
import torch

from paper_2106_15869_b300 import autotune
from paper_2106_15869_b300 import workloads as W


def test_problem_key_classes():
    F3 = torch.ones(32, 32, 32)
    F2 = torch.ones(64, 64)
    assert autotune.problem_key(F3).startswith("d3-n15-b0-fp32-low")
    assert autotune.problem_key(F2, 64).startswith("d2-n12-b6-fp32-low")
    maze = torch.ones(16, 16, 16)
    maze[4] = 1e-3
    assert autotune.problem_key(maze).endswith("-high")
    assert autotune.problem_key(F3.double()).split("-")[3] == "fp64"


@pytest.mark.gpu
def test_tune_caches_and_solves(tmp_path):
    import oracle
    from paper_2106_15869_b300 import api
    inst = W.oscillating_3d(48)
    F = torch.as_tensor(inst.F, dtype=torch.float32).cuda()
    path = str(tmp_path / "tune.json")
    opts = autotune.tune([(F, inst.src_idx, inst.h)], cache_path=path, reps=1)
    assert opts["schedule"] in ("persistent", "async")
    assert opts["tile"] in ("8x8x4", "8x4x4", "4x4x4", "8x8x8") and len(opts["_ms"]) >= 4
    assert opts.get("converge", "auto") in ("auto", "sweep")
    assert any("converge=sweep" in k for k in opts["_ms"])
    cached = json.load(open(path))
    assert autotune.problem_key(F) in cached
    again = autotune.tune([(F, inst.src_idx, inst.h)], cache_path=path)      # cache hit, no timing
    assert again == opts
    phi = api.solve(F, inst.src_idx, inst.h, **autotune.tuned_options([(F, inst.src_idx, inst.h)], cache_path=path))
    ref = oracle.fmm(inst.F.astype(np.float32).astype(np.float64), inst.h, inst.src_idx)
    assert np.max(np.abs(phi.cpu().double().numpy() - ref)) <= 1e-4 * ref.max()


@pytest.mark.gpu
def test_tune_2d_tries_the_step3_only_order(tmp_path):
    import oracle
    from paper_2106_15869_b300 import api
    inst = W.paper_example_2d(3, 160)
    F = torch.as_tensor(inst.F, dtype=torch.float32).cuda()
    val = torch.as_tensor(inst.src_val, dtype=torch.float32).cuda()
    path = str(tmp_path / "tune.json")
    opts = autotune.tune([(F, inst.src_idx, inst.h)], cache_path=path, reps=1)
    assert autotune.problem_key(F).startswith("d2")
    assert any("remedy_order=4.0" in k for k in opts["_ms"])
    kw = {k: v for k, v in opts.items() if not k.startswith("_")}
    phi = api.solve(F, inst.src_idx, inst.h, val, **kw)
    ref = oracle.fmm(inst.F.astype(np.float32).astype(np.float64), inst.h, inst.src_idx,
                     inst.src_val.astype(np.float32).astype(np.float64))
    fin = np.isfinite(ref)
    got = phi.cpu().double().numpy()
    assert np.array_equal(fin, np.isfinite(got))
    assert np.max(np.abs(got[fin] - ref[fin])) <= 1e-4 * ref[fin].max()
