"""Autotuner for the tile shape, the list order (with the Step-3 bucket width),
the schedule and the Step-2 convergence test of the solve.

The best tile shape (4x4x4, 8x4x4, 8x8x4, 8x8x8; 16x16x1 or 8x8x1 in 2D),
list order (bucketed or unordered), schedule (the persistent kernel with
its per-iteration list passes, or the asynchronous work queue) and Step-2
convergence test of a tile (a confirming visit that changes nothing, or the
visit's own relaxation reaching the tile's fixed point) depend on the grid
size, the batch size and the speed field (slow walls in a fast medium change
which list order wins; smooth speeds from one corner favour the one-visit
test, many sources on a face the confirming one).  tune()
times each candidate on the caller's own inputs (device time from the
library's CUDA events, median of a few runs) and caches the winner in a JSON
file keyed by

    (dimensionality, log2 bucket of nodes per instance, log2 bucket of the
     batch size, precision, speed-contrast class)

so later problems of the same class reuse it without timing.  Every candidate
solves the same discrete problem, so the choice never changes the result
beyond rounding.
"""
from __future__ import annotations

import json
import math
import os
import statistics
import threading

import torch

from . import api

# persistent schedule with either list order, and the asynchronous queue (which has no order); on
# 8x8x8 tiles also the one-visit Step-2 test (measured on B300: 14 % faster on the 256^3
# oscillating speed and 3 % on the 64-instance lognormal batch, 2x slower on the 16-shot tomography)
# and Step-3 bucket widths beside the default 4 (measured on B300: the 64-instance batch is fastest
# at width 2, the 512^3 maze at 5 to 6, 3 % faster than at 4, where the batch is 8 % slower)
CANDIDATES_3D = ([dict(tile=t, order=o, schedule="persistent") for t in ("8x8x4", "8x4x4", "4x4x4", "8x8x8")
                  for o in (0.0, -1.0)] + [dict(tile=t, order=-1.0, schedule="async") for t in ("8x8x4", "8x8x8")]
                 + [dict(tile="8x8x8", order=0.0, schedule="persistent", converge=c, remedy_order=w)
                    for c in ("auto", "sweep") for w in (0.0, 2.0, 3.0) if (c, w) != ("auto", 0.0)]
                 + [dict(tile="8x8x8", order=0.0, schedule="persistent", remedy_order=w) for w in (5.0, 6.0)])
# 2D: also unordered Step-2 lists with bucketed Step-3 lists (measured at 4000^2: Example 3 9.7 ->
# 5.7 ms and Example 1 6.4 -> 5.5 ms, Example 5 9.6 -> 15.4 ms against the 2D default, which buckets
# both)
CANDIDATES_2D = ([dict(tile=t, order=o, schedule="persistent") for t in ("16x16x1", "8x8x1") for o in (0.0, -1.0)]
                 + [dict(tile="16x16x1", order=-1.0, schedule="async"),
                    dict(tile="16x16x1", order=-1.0, remedy_order=4.0, schedule="persistent")])

_lock = threading.Lock()


def default_cache_path() -> str:
    base = os.environ.get("EIKONAL_TUNE_CACHE")
    if base:
        return base
    return os.path.join(os.path.expanduser("~"), ".cache", "eikonal_b300", "tune.json")


def problem_key(F: torch.Tensor, batch: int = 1) -> str:
    """Cache key of a problem class (see the module docstring)."""
    nd = 2 if F.dim() == 2 or (F.dim() == 3 and F.shape[0] == 1) else 3
    nodes_b = int(math.log2(max(F.numel(), 1)))
    batch_b = int(math.log2(max(batch, 1)))
    pos = F[F > 0]
    contrast = "high" if pos.numel() and float(pos.max()) > 100.0 * float(pos.min()) else "low"
    dt = "fp64" if F.dtype == torch.float64 else "fp32"
    return f"d{nd}-n{nodes_b}-b{batch_b}-{dt}-{contrast}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, data):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time_solve(problems, opts, reps):
    ms = []
    for _ in range(reps):
        if len(problems) == 1:
            F, src, h = problems[0][:3]
            _, st = api.solve(F, src, h, return_stats=True, **opts)
        else:
            _, st = api.solve_batched(problems, return_stats=True, **opts)
        ms.append(st["ms_total"])
    return statistics.median(ms)


def tune(problems, *, cache_path: str | None = None, reps: int = 3, candidates=None, force: bool = False) -> dict:
    """Options (tile, order, schedule, converge, remedy_order) for this problem class, timed on
    `problems` on a cache miss.

    problems: a list of (F, src_idx, h) tuples (one for a single solve) on a CUDA
    device.  Returns a dict usable as keyword arguments of api.solve /
    api.solve_batched, plus the timings under "_ms".
    """
    path = cache_path or default_cache_path()
    F0 = problems[0][0]
    key = problem_key(F0, len(problems))
    with _lock:
        cache = _load(path)
        if key in cache and not force:
            return dict(cache[key])
    if candidates is None:
        candidates = CANDIDATES_2D if key.startswith("d2") else CANDIDATES_3D
    timings = {}
    best, best_ms = None, float("inf")
    for c in candidates:
        try:
            _time_solve(problems, c, 1)                  # warm-up
            t = _time_solve(problems, c, reps)
        except api._lib.EikonalError:
            continue
        name = f"{c['tile']}/order={c['order']}/{c.get('schedule', 'auto')}"
        if c.get("converge", "auto") != "auto":
            name += f"/converge={c['converge']}"
        if c.get("remedy_order", 0.0):
            name += f"/remedy_order={c['remedy_order']}"
        timings[name] = t
        if t < best_ms:
            best, best_ms = c, t
    if best is None:
        raise RuntimeError("no candidate configuration ran")
    entry = dict(best)
    entry["_ms"] = timings
    with _lock:
        cache = _load(path)
        cache[key] = entry
        _store(path, cache)
    return dict(entry)


def tuned_options(problems, **kw) -> dict:
    """The tuned options without the timing record."""
    return {k: v for k, v in tune(problems, **kw).items() if not k.startswith("_")}
