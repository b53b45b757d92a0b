#!/usr/bin/env python
"""Throughput of the improved-FIM Eikonal solve on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload maze_512|oscillating_256|point_source_128|lognormal_batch64]

One step = one complete solve (Steps 1-3 of Algorithm 2 and the output
unpack) of the workload, inputs already resident in HBM.  The default workload
is the largest single grid: the 512^3 maze (134 M nodes, slabs of slow walls
with one gap each, 4 sources).  The metric is converged grid nodes per second,
FP32.  Each step's device time is measured with CUDA events that the library
records on the solve's stream (first to last kernel); L2 is flushed between
steps by a 256 MiB write outside the measured interval.  With N > 1 (torchrun)
every rank solves its own replica (weak scaling, no collective on the data
path); value = nodes over all ranks / max over ranks of the time.

Beside the headline line's own roofline (the Step-2/3 loop kernel of the 512^3
maze) the line carries the other forms, each with its roofline block: the
64-instance lognormal batch on autotuned options, replayed from a CUDA graph;
the 192^3 tomography (16 shots: forward, adjoint, forward + adjoint); the 256^3
oscillating-speed grid; the paper's 2D examples; and the FIM of Sec. 2.3 on the
headline grid.

--impl reference times the FP64 CPU oracle (fast marching) on the host cores
on a bounded sample of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "converged grid nodes/sec and % HBM roofline, FP32 at 1e-4 rel; fwd+adjoint vs plain"
UNIT = "nodes/s"
# algorithmic bytes per node of the Step-2/3 loop kernel (FP32): every node is
# read (phi, tau) and written (phi) at least once in Step 2, and read (phi,
# tau) once by the Step-3 recomputation: 12 + 8 = 20 B.
LOOP_BYTES_PER_NODE = 20
# whole step incl. layout conversion: F read, tau/phi brick writes (12 B),
# the loop (20 B), unpack read + write (8 B)
STEP_BYTES_PER_NODE = 40
# the adjoint's loop kernel: phi, tau and r read once, lambda written once (16 B per node)
ADJ_LOOP_BYTES_PER_NODE = 16
FALLBACK_HBM_GBS = 6400.0
# kernels of one default solve: k_write_desc, k_init, k_scale, k_tile_scale, k_sources,
# k_persistent, k_unpack
LAUNCHES_PER_SOLVE = 7

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the loop kernel
# with the default options (or the ones an entry names), from one-pass ncu captures of that kernel
# on the full workload (the ncu captures summarised with the profiles of this repository);
# reported only for those options and while the kernel sources (comments stripped) hash to the captured version
# (else null).
MEASURED_TRAFFIC = {
    "maze_512": {"hash": "35e2b5e8e7ed3dfa", "bytes": 3460604672 + 908771584},
    "lognormal_batch64": {"hash": "35e2b5e8e7ed3dfa", "bytes": 9066408448 + 1564659456},
    "lognormal_batch64_tuned": {"hash": "35e2b5e8e7ed3dfa", "bytes": 7149655552 + 1437020416,
                                "opts": {"tile": "8x8x8", "order": 0.0, "schedule": "persistent",
                                         "converge": "sweep", "remedy_order": 2.0}},
    "tomography_192_forward": {"hash": "35e2b5e8e7ed3dfa", "bytes": 2011617024 + 463398912},
    "oscillating_256": {"hash": "35e2b5e8e7ed3dfa", "bytes": 349053696 + 82819072},
    "tomography_192_adjoint": {"hash": "d42a46e339bf29bf", "bytes": 2806409216 + 413992704},
}


# The paper's own timings (seconds on an NVIDIA Tesla P100; Tables 1, 2, 3 and 5,
# Sec. 4.1) of its GPU FIM and iFIM for Examples 1, 2, 3 and 5 at N^2 nodes --
# context for the B300 times of the same examples, not a target.  As printed, the FIM
# rows of Tables 3 and 5 share their first four entries; they are kept as printed.
PAPER_SIZES = (200, 500, 1000, 2000, 4000)
PAPER_TIMES_S = {
    1: {"fim": (0.00164, 0.00428, 0.08834, 0.32604, 1.67655), "ifim": (0.00141, 0.00384, 0.03721, 0.11642, 0.80981)},
    2: {"fim": (0.00118, 0.00319, 0.08794, 0.63421, 1.86989), "ifim": (0.00097, 0.00329, 0.0539, 0.35359, 1.09434)},
    3: {"fim": (0.00125, 0.00410, 0.08954, 0.78251, 2.05581), "ifim": (0.00089, 0.00341, 0.0499, 0.36897, 1.48971)},
    5: {"fim": (0.00125, 0.00410, 0.08954, 0.78251, 2.45581), "ifim": (0.00119, 0.00341, 0.0689, 0.56897, 1.098971)},
}


# the sources the forward solve's kernels (and their launch) are built from; the adjoint and
# back-trace headers are left out, so that changing them keeps the captured forward counters
FORWARD_SOURCES = ("eik_api.cu", "eik_async.cuh", "eik_common.cuh", "eik_forward.cuh", "eik_group.cuh",
                   "eik_kernels.cuh")
ADJOINT_SOURCES = FORWARD_SOURCES + ("eik_adjoint.cuh",)


def _code_only(text: str) -> str:
    """C++ source without comments and with whitespace collapsed: a change to a comment
    leaves the hash of the kernel sources as it was (the sources hold no string literal
    with a comment marker in it)."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_hash(files=FORWARD_SOURCES) -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2106_15869_b300", "csrc")
    for f in files:
        h.update(_code_only(open(os.path.join(csrc, f)).read()).encode())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def _norm_opts(o: dict) -> tuple:
    return (o.get("tile", "8x8x8"), float(o.get("order", 0.0)), o.get("schedule", "persistent"),
            o.get("converge", "auto"), float(o.get("remedy_order", 0.0)))


def captured_traffic(key: str, files=FORWARD_SOURCES, opts: dict | None = None):
    """Bytes per launch from MEASURED_TRAFFIC for `key`, or None when absent or stale: the kernel
    sources must hash to the captured version, and the solve options (default ones unless the
    entry names others) must be the captured ones."""
    t = MEASURED_TRAFFIC.get(key)
    if not t or t.get("hash") != kernel_source_hash(files):
        return None
    if _norm_opts(opts or {}) != _norm_opts(t.get("opts", {})):
        return None
    return t["bytes"]


def roofline_block(kernel: str, bytes_per_node: float, nodes: int, loop_ms: float, traffic=None, **extra) -> dict:
    """Roofline of one loop kernel: algorithmic bytes (bytes_per_node x nodes) over its
    device time, against the measured HBM copy bandwidth."""
    peak, peak_kind = measured_peaks()
    achieved = bytes_per_node * nodes / (loop_ms / 1e3) / 1e9
    return {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak, "peak_kind": peak_kind,
            "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
            "algorithmic_bytes_per_node": bytes_per_node, "nodes": nodes, "loop_ms": loop_ms, **extra}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(seconds: float, device=None) -> float:
    """Max of a per-rank time over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return seconds
    t = torch.tensor([seconds], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(nodes_per_rank: int, steps: int, world: int, seconds: float) -> float:
    """Converged nodes per second of the whole job: every rank solves its own replica
    (weak scaling), so the units processed are nodes x steps x ranks over the slowest rank's time."""
    return nodes_per_rank * steps * world / seconds


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def make_workload(name: str):
    from paper_2106_15869_b300 import workloads as W
    if name == "oscillating_256":
        return [W.oscillating_3d(256)]
    if name == "point_source_128":
        return [W.point_source_2d(128, (64, 64))]
    if name == "maze_512":
        return [W.maze_3d(512)]
    if name == "lognormal_batch64":
        return W.lognormal_batch(64)
    raise ValueError(name)


def cpu_sample(name: str):
    """Bounded sample of the workload for the oracle timing (single-threaded fast marching)."""
    from paper_2106_15869_b300 import workloads as W
    if name == "oscillating_256":
        return W.oscillating_3d(256), "full 256^3 oscillating-speed grid, one FMM solve"
    if name == "point_source_128":
        return W.point_source_2d(128, (64, 64)), "full 128^2 grid"
    if name == "maze_512":
        return W.maze_3d(192, n_slabs=6, gap=12), "192^3 maze built by the same recipe (6 slabs/axis, 12^2 gaps)"
    return W.lognormal_batch(4)[0], "first instance of the lognormal batch"


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args, ws, rank):
    import numpy as np
    import oracle
    if rank != 0:
        return 0
    inst, desc = cpu_sample(args.workload)
    F = inst.F.astype(np.float32).astype(np.float64)
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.fmm(F, inst.h, inst.src_idx, inst.src_val)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = inst.n_nodes * len(times) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "sample": desc, "nodes_per_step": inst.n_nodes},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, ws, rank, local):
    import torch
    import torch.distributed as dist
    from paper_2106_15869_b300 import api

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=dev)
    insts = make_workload(args.workload)
    n_nodes = sum(i.n_nodes for i in insts)
    wsp = api.Workspace(dev)
    stream = torch.cuda.current_stream(dev)

    if len(insts) == 1:
        inst = insts[0]
        F = torch.as_tensor(inst.F, dtype=torch.float32).to(dev)
        idx = torch.as_tensor(inst.src_idx).to(dev)
        val = torch.as_tensor(inst.src_val, dtype=torch.float32).to(dev)
        phi = torch.empty_like(F)

        def step(stats=True):
            return api.solve(F, idx, inst.h, val, tile=args.tile, schedule=args.schedule, workspace=wsp,
                             out=phi, return_stats=stats, order=args.order, converge=args.converge,
                             method=args.method)
    else:
        probs = [(torch.as_tensor(i.F, dtype=torch.float32).to(dev), i.src_idx, i.h, i.src_val) for i in insts]

        def step(stats=True):
            return api.solve_batched(probs, tile=args.tile, schedule=args.schedule, workspace=wsp,
                                     return_stats=stats, order=args.order, converge=args.converge,
                                     method=args.method)

    flush_buf = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > L2
    for _ in range(args.warmup):
        _, st = step()
        if st["status"] != 0:
            raise RuntimeError(f"solve failed: {st}")
    sampler = ClockSampler(local)
    sampler.start()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    tot, loop, stats = [], [], []
    for _ in range(args.steps):
        flush_buf.zero_()
        _, st = step()
        tot.append(st["ms_total"])
        loop.append(st["ms_loop"])
        stats.append(st)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    total_s = max_over_ranks(sum(tot) / 1e3, dev if ws > 1 else None)
    value = whole_job_rate(n_nodes, args.steps, ws, total_s)
    ms_step = 1e3 * total_s / args.steps
    loop_ms = statistics.mean(loop)

    # end to end through the public API: pinned host F in, host phi out, every step
    e2e = None
    if len(insts) == 1:
        e2e = bench_e2e(args, inst, F, idx, val, phi, wsp, flush_buf, stream, n_nodes, ws)

    src_hash = kernel_source_hash()
    # the captured traffic belongs to the default options only
    default_opts = (args.method == "ifim" and args.tile == "auto" and args.schedule == "auto"
                    and args.order == 0.0 and args.converge == "auto")
    traffic = captured_traffic(args.workload) if default_opts else None
    roofline = roofline_block("k_persistent (Steps 2-3)", LOOP_BYTES_PER_NODE, n_nodes, loop_ms, traffic,
                              loop_share_of_step=loop_ms / ms_step,
                              step_achieved_gbs=STEP_BYTES_PER_NODE * n_nodes / (ms_step / 1e3) / 1e9)
    s0 = stats[-1]
    # work of the loop: in-tile sweeps x nodes per tile, an upper bound of the local solves (a
    # latency-mode sweep solves every node of its tile; throughput-mode sweeps skip node slots
    # whose neighbours did not change)
    if args.tile == "auto":
        tile_v = 256 if all(i.dims[2] == 1 for i in insts) else 512
    else:
        bx, by, bz = (int(v) for v in args.tile.split("x"))
        tile_v = bx * by * bz
    sweep_nodes = s0["sweeps"] * tile_v
    work = {"sweep_nodes": sweep_nodes, "sweep_nodes_per_node": sweep_nodes / n_nodes,
            "sweep_nodes_per_s": sweep_nodes / (loop_ms / 1e3),
            "tile_visits": s0["tiles_update"] + s0["tiles_remedy"], "tile_nodes": tile_v}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "nodes_per_gpu": n_nodes, "instances": len(insts),
                       "tile": args.tile, "schedule": args.schedule, "order": args.order,
                       "converge": args.converge, "method": args.method,
                       "l2": "flushed between steps (256 MiB write outside the per-step events)",
                       "parallelism": f"replicas x{ws}"},
            "roofline": roofline, "work": work, "e2e": e2e, "clocks": clocks,
            "gpu_launches": LAUNCHES_PER_SOLVE * args.steps,
            "solver_stats": {k: s0[k] for k in ("iters_update", "iters_remedy", "tiles_update",
                                                "tiles_flagged", "tiles_remedy", "sweeps", "tiles_deferred")},
            "wall_s_timed_region": wall, "kernel_source_hash": src_hash}
    # where the loop time goes (per-iteration trace of one more solve, outside the timed region)
    if len(insts) == 1:
        with api.Trace() as tr:
            step(stats=False)
        line["trace"] = tr.summary()
    if not args.no_extras:
        if len(insts) == 1:
            line["fim_vs_ifim"] = bench_methods(args, insts[0], F, idx, val, phi, wsp, flush_buf)
            line["backtrace"] = bench_backtrace(args, insts[0], F, idx, val, phi, wsp, flush_buf)
            line["unequal_spacings"] = bench_spacings(args, insts[0], F, idx, val, phi, wsp, flush_buf)
            del F, phi
        if args.workload != "oscillating_256":
            line["oscillating_256"] = bench_single(dev, wsp, flush_buf, "oscillating_256")
        line["batched"] = bench_batched(args, dev, wsp, flush_buf)
        line["adjoint"] = bench_adjoint(args, dev, wsp, flush_buf)
        line["paper_examples"] = bench_paper_examples(args, dev, wsp, flush_buf)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import numpy as np
        import oracle
        inst_c, desc = cpu_sample(args.workload)
        Fc = inst_c.F.astype(np.float32).astype(np.float64)
        t0 = time.perf_counter()
        oracle.fmm(Fc, inst_c.h, inst_c.src_idx, inst_c.src_val)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": inst_c.n_nodes / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": desc, "seconds": dt}
        if not args.no_extras:
            line["batched"]["cpu_baseline"] = cpu_baseline_batch(64)
            line["adjoint"]["cpu_baseline"] = cpu_baseline_tomography(16)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def bench_e2e(args, inst, F, idx, val, phi, wsp, flush_buf, stream, n_nodes, ws):
    """The same solve end to end through api.solve: every step copies its speeds and
    sources in from pinned host memory and its phi back out.

    serial: one step at a time (copy in, solve, copy out), CUDA events around each.
    value (pipelined, the way a stream of problems is served): the copies run on their own
    streams with two device buffers, so that step k's solve overlaps the copy in of step
    k + 1 and the copy out of step k - 1; the solves stay on one stream (a cooperative
    launch never shares the GPU with another kernel).  Timed from before the first copy in
    to after the last copy out, K steps."""
    import torch
    from paper_2106_15869_b300 import api
    F_h = torch.as_tensor(inst.F, dtype=torch.float32).pin_memory()
    idx_h = torch.as_tensor(inst.src_idx).pin_memory()
    val_h = torch.as_tensor(inst.src_val, dtype=torch.float32).pin_memory()
    phi_h = [torch.empty_like(F_h).pin_memory() for _ in range(2)]
    opts = dict(tile=args.tile, schedule=args.schedule, order=args.order, converge=args.converge, method=args.method)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    serial_ms = []
    for s in range(args.steps + 1):
        flush_buf.zero_()
        ev0.record(stream)
        F.copy_(F_h, non_blocking=True)
        idx.copy_(idx_h, non_blocking=True)
        val.copy_(val_h, non_blocking=True)
        api.solve(F, idx, inst.h, val, workspace=wsp, out=phi, **opts)
        phi_h[0].copy_(phi, non_blocking=True)
        ev1.record(stream)
        ev1.synchronize()
        if s > 0:
            serial_ms.append(ev0.elapsed_time(ev1))
    # pipelined: buffers k % 2; copy-in and copy-out streams, solves on `stream`
    Fd = [F, torch.empty_like(F)]
    idd = [idx, torch.empty_like(idx)]
    vd = [val, torch.empty_like(val)]
    pd = [phi, torch.empty_like(phi)]
    s_in, s_out = torch.cuda.Stream(F.device), torch.cuda.Stream(F.device)
    K = args.steps
    solved = [torch.cuda.Event() for _ in range(K)]
    copied_in = [torch.cuda.Event() for _ in range(K)]
    copied_out = [torch.cuda.Event() for _ in range(K)]
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    s_in.wait_stream(stream)
    for k in range(K):
        b = k % 2
        with torch.cuda.stream(s_in):
            if k >= 2:
                s_in.wait_event(solved[k - 2])          # buffer b was read by solve k - 2
            Fd[b].copy_(F_h, non_blocking=True)
            idd[b].copy_(idx_h, non_blocking=True)
            vd[b].copy_(val_h, non_blocking=True)
            copied_in[k].record(s_in)
        stream.wait_event(copied_in[k])
        if k >= 2:
            stream.wait_event(copied_out[k - 2])        # phi buffer b was read out by step k - 2
        api.solve(Fd[b], idd[b], inst.h, vd[b], workspace=wsp, out=pd[b], **opts)
        solved[k].record(stream)
        with torch.cuda.stream(s_out):
            s_out.wait_event(solved[k])
            phi_h[b].copy_(pd[b], non_blocking=True)
            copied_out[k].record(s_out)
    stream.wait_stream(s_out)
    t1.record(stream)
    t1.synchronize()
    pipe_ms = t0.elapsed_time(t1) / K
    h2d = F_h.numel() * 4 + idx_h.numel() * 8 + val_h.numel() * 4
    out = {"value": n_nodes * ws / (pipe_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(phi_h[0].numel() * 4), "ms_per_step": pipe_ms,
           "mode": "pipelined: step k's solve overlaps the copy in of k + 1 and the copy out of k - 1",
           "serial_ms_per_step": statistics.mean(serial_ms),
           "serial_value": n_nodes * ws / (statistics.mean(serial_ms) / 1e3)}
    del Fd[1], idd[1], vd[1], pd[1]
    return out


def _timed(fn, flush_buf, reps):
    """Median device time (ms) of fn() over reps runs, L2 flushed before each."""
    import torch
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    for _ in range(reps):
        flush_buf.zero_()
        ev0.record(stream)
        fn()
        ev1.record(stream)
        ev1.synchronize()
        ms.append(ev0.elapsed_time(ev1))
    return statistics.median(ms)


def bench_methods(args, inst, F, idx, val, phi, wsp, flush_buf):
    """The same workload by the improved FIM (Algorithm 2) and by the FIM of Sec. 2.3
    (tile-level neighbour checks, no remedy; unordered lists, as that method is
    stated), both to the same discrete solution (cf. the paper's FIM-vs-iFIM
    comparison, Sec. 4.2)."""
    from paper_2106_15869_b300 import api
    out = {}
    for name, kw in (("ifim", dict(method="ifim")), ("fim", dict(method="fim", order=-1.0))):
        run = lambda: api.solve(F, idx, inst.h, val, workspace=wsp, out=phi, **kw)
        run()
        ms = _timed(run, flush_buf, 3)
        _, st = api.solve(F, idx, inst.h, val, workspace=wsp, out=phi, return_stats=True, **kw)
        out[name] = {"ms": ms, "nodes_per_s": inst.n_nodes / (ms / 1e3), "loop_ms": st["ms_loop"],
                     "iterations": st["iters_update"] + st["iters_remedy"],
                     "tile_visits": st["tiles_update"] + st["tiles_remedy"], "sweeps": st["sweeps"]}
    out["fim_speedup_over_ifim"] = out["ifim"]["ms"] / out["fim"]["ms"]
    return out


def bench_spacings(args, inst, F, idx, val, phi, wsp, flush_buf):
    """The same speeds on a stretched grid, spacings (h, 1.25 h, 2 h) (eq. 6 with unequal
    spacings, the 3D form of Alg 1.2), against equal spacings h."""
    from paper_2106_15869_b300 import api
    out = {}
    for name, h in (("equal", inst.h), ("unequal", (inst.h, 1.25 * inst.h, 2.0 * inst.h))):
        run = lambda: api.solve(F, idx, h, val, workspace=wsp, out=phi)
        run()
        ms = _timed(run, flush_buf, 3)
        _, st = api.solve(F, idx, h, val, workspace=wsp, out=phi, return_stats=True)
        out[name] = {"spacings": h if isinstance(h, tuple) else (h, h, h), "ms": ms,
                     "nodes_per_s": inst.n_nodes / (ms / 1e3), "sweeps": st["sweeps"],
                     "tile_visits": st["tiles_update"] + st["tiles_remedy"]}
    out["unequal_over_equal"] = out["unequal"]["ms"] / out["equal"]["ms"]
    return out


def bench_backtrace(args, inst, F, idx, val, phi, wsp, flush_buf):
    """Shortest paths from 4096 seeded destinations back to the source by steepest
    descent on the solved phi (the application of Example 4, Sec. 4.1)."""
    import numpy as np
    import torch
    from paper_2106_15869_b300 import api
    api.solve(F, idx, inst.h, val, workspace=wsp, out=phi)
    starts = torch.as_tensor(np.random.default_rng(11).integers(0, inst.n_nodes, size=4096)).to(phi.device)
    max_len = 4 * sum(F.shape)
    run = lambda: api.backtrace(phi, starts, inst.h, max_len=max_len)
    _, length = run()
    ms = _timed(run, flush_buf, 5)
    steps = int(length.clamp(min=0).sum().item())
    return {"paths": 4096, "max_len": max_len, "ms": ms, "path_nodes": steps,
            "path_nodes_per_s": steps / (ms / 1e3), "mean_length": steps / 4096}


def bench_single(dev, wsp, flush_buf, name):
    """A secondary single-grid workload with the default options: device time per solve and
    the loop kernel's roofline."""
    import torch
    from paper_2106_15869_b300 import api
    inst = make_workload(name)[0]
    F = torch.as_tensor(inst.F, dtype=torch.float32).to(dev)
    idx = torch.as_tensor(inst.src_idx).to(dev)
    val = torch.as_tensor(inst.src_val, dtype=torch.float32).to(dev)
    phi = torch.empty_like(F)
    run = lambda: api.solve(F, idx, inst.h, val, workspace=wsp, out=phi, return_stats=True)
    run()
    loops, tots = [], []
    for _ in range(5):
        flush_buf.zero_()
        _, st = run()
        loops.append(st["ms_loop"])
        tots.append(st["ms_total"])
    loop_ms, ms = statistics.median(loops), statistics.median(tots)
    return {"workload": name, "nodes": inst.n_nodes, "ms": ms, "nodes_per_s": inst.n_nodes / (ms / 1e3),
            "solver_stats": {k: st[k] for k in ("iters_update", "iters_remedy", "tiles_update", "tiles_flagged",
                                                "tiles_remedy", "sweeps")},
            "roofline": roofline_block("k_persistent (Steps 2-3)", LOOP_BYTES_PER_NODE, inst.n_nodes, loop_ms,
                                       captured_traffic(name))}


def bench_paper_examples(args, dev, wsp, flush_buf):
    """Examples 1, 2, 3 and 5 of Sec. 4.1 (2D, [-10, 10]^2, N = 200 .. 4000) by both methods,
    device time per solve, beside the paper's P100 times (Tables 1-3, 5)."""
    import torch
    from paper_2106_15869_b300 import api, workloads as W
    rows = []
    for ex in sorted(PAPER_TIMES_S):
        for q, n in enumerate(PAPER_SIZES):
            inst = W.paper_example_2d(ex, n=n)
            F = torch.as_tensor(inst.F, dtype=torch.float32).to(dev)
            idx = torch.as_tensor(inst.src_idx).to(dev)
            val = torch.as_tensor(inst.src_val, dtype=torch.float32).to(dev)
            phi = torch.empty_like(F)
            row = {"example": ex, "n": n}
            for name, kw in (("ifim", dict(method="ifim")), ("fim", dict(method="fim", order=-1.0))):
                run = lambda: api.solve(F, idx, inst.h, val, workspace=wsp, out=phi, **kw)
                run()
                row[f"{name}_ms"] = _timed(run, flush_buf, 3)
                row[f"paper_p100_{name}_ms"] = 1e3 * PAPER_TIMES_S[ex][name][q]
            rows.append(row)
    return {"unit": "ms per solve (device time, FP32)", "rows": rows}


def bench_batched(args, dev, wsp, flush_buf):
    """64 lognormal instances (edges 64..192): one batched solve on the options the autotuner
    picks for this problem class (tile shape x list order x one-launch schedule), replayed
    from a CUDA graph, vs one default solve per instance."""
    import torch
    from paper_2106_15869_b300 import api, autotune, workloads as W
    insts = W.lognormal_batch(64)
    n = sum(i.n_nodes for i in insts)
    probs = [(torch.as_tensor(i.F, dtype=torch.float32).to(dev), i.src_idx, i.h) for i in insts]
    t0 = time.perf_counter()
    tuned = autotune.tune(probs, reps=2)
    tune_s = time.perf_counter() - t0
    opts = {k: v for k, v in tuned.items() if not k.startswith("_")}
    bs = api.BatchedSolver(probs, graph=True, **opts)     # one cooperative launch, replayed from a CUDA graph
    batched = bs.solve
    plain = lambda: [api.solve(p[0], p[1], p[2], workspace=wsp) for p in probs]
    batched(); plain()
    tb = _timed(batched, flush_buf, 5)
    tp = _timed(plain, flush_buf, 2)
    loops = []
    for _ in range(3):
        flush_buf.zero_()
        st = bs.stats()
        loops.append(st["ms_loop"])
    loop_ms = statistics.median(loops)
    return {"workload": "lognormal_batch64 (64 instances, edges 64..192, F = exp(0.3 g))", "nodes": n,
            "tuned_options": opts, "tuning_ms": tuned.get("_ms"), "tuning_s": tune_s, "graph_replay": True,
            "batched_ms": tb, "batched_nodes_per_s": n / (tb / 1e3), "plain_loop_ms": tp,
            "plain_loop_nodes_per_s": n / (tp / 1e3), "speedup_vs_plain": tp / tb,
            "solver_stats": {k: st[k] for k in ("iters_update", "iters_remedy", "tiles_update", "tiles_flagged",
                                                "tiles_remedy", "sweeps")},
            "roofline": roofline_block(f"k_persistent (Steps 2-3, batch of 64, {opts})", LOOP_BYTES_PER_NODE, n,
                                       loop_ms, captured_traffic("lognormal_batch64", opts=opts)
                                       or captured_traffic("lognormal_batch64_tuned", opts=opts),
                                       loop_share_of_step=loop_ms / tb)}


def bench_adjoint(args, dev, wsp, flush_buf):
    """Tomography 192^3, 16 shots, 256 receivers, at the configured initial slowness s = 1:
    forward (one batched solve of the 16 shots on one slowness model) + adjoint (one batched
    adjoint, gradients summed) vs the forward alone and vs 16 plain single solves; the loop
    kernels' rooflines."""
    import torch
    from paper_2106_15869_b300 import api, workloads as W
    t = W.tomography_3d(192)
    F = torch.as_tensor(1.0 / t["s_init"], dtype=torch.float32).to(dev)
    shots = [[int(s)] for s in t["sources"]]
    rec = torch.as_tensor(t["receivers"]).to(dev)
    probs = [(F, sh, t["h"]) for sh in shots]
    phis = api.solve_batched(probs, shared_F=True, workspace=wsp)
    rs = []
    for ph in phis:
        r = torch.zeros_like(ph).reshape(-1)
        r[rec] = 1.0
        rs.append(r.view(ph.shape))
    fwd = lambda: api.solve_batched(probs, shared_F=True, workspace=wsp)
    adj = lambda: api.adjoint_batched(probs, phis, rs, shared_F=True, sum_instances=True, workspace=wsp)
    both = lambda: (fwd(), adj())
    plain = lambda: [api.solve(F, sh, t["h"], workspace=wsp) for sh in shots]
    both(); plain()
    tf = _timed(fwd, flush_buf, 3)
    ta = _timed(adj, flush_buf, 3)
    tb = _timed(both, flush_buf, 3)
    tp = _timed(plain, flush_buf, 2)
    n = F.numel() * len(shots)
    f_loop, a_loop = [], []
    for _ in range(3):
        flush_buf.zero_()
        _, fst = api.solve_batched(probs, shared_F=True, workspace=wsp, return_stats=True)
        flush_buf.zero_()
        _, ast = api.adjoint_batched(probs, phis, rs, shared_F=True, sum_instances=True, workspace=wsp,
                                     return_stats=True)
        f_loop.append(fst["ms_loop"])
        a_loop.append(ast["ms_loop"])
    fl, al = statistics.median(f_loop), statistics.median(a_loop)
    return {"workload": "tomography 192^3, 16 shots, 256 receivers, s = 1", "nodes_per_pass": n,
            "adjoint_stats": {"iterations": ast["iters_remedy"], "tile_visits": ast["tiles_remedy"],
                              "sweeps": ast["sweeps"], "loop_ms": al},
            "forward_ms": tf, "adjoint_ms": ta, "forward_plus_adjoint_ms": tb,
            "fwd_adj_over_fwd": tb / tf, "plain_16_solves_ms": tp, "forward_speedup_vs_plain": tp / tf,
            "forward_nodes_per_s": n / (tf / 1e3), "fwd_adj_nodes_per_s": n / (tb / 1e3),
            "roofline": {
                "forward": roofline_block("k_persistent (16 shots, shared speeds)", LOOP_BYTES_PER_NODE, n, fl,
                                          captured_traffic("tomography_192_forward")),
                "adjoint": roofline_block("k_adj_persistent (16 shots, gradients summed)", ADJ_LOOP_BYTES_PER_NODE,
                                          n, al, captured_traffic("tomography_192_adjoint", ADJOINT_SOURCES)),
                "forward_plus_adjoint": roofline_block("both loop kernels", LOOP_BYTES_PER_NODE
                                                       + ADJ_LOOP_BYTES_PER_NODE, n, fl + al)}}


def cpu_baseline_batch(k: int) -> dict:
    """The oracle's fast marching on the first k instances of the 64-instance batch (all of
    them by default), one instance per host core at a time (a thread pool; ctypes releases
    the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    import numpy as np
    import oracle
    from paper_2106_15869_b300 import workloads as W
    insts = W.lognormal_batch(64)[:k]
    cores = min(host_cores(), k)
    run = lambda i: oracle.fmm(i.F.astype(np.float32).astype(np.float64), i.h, i.src_idx, i.src_val)
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(run, insts))
    dt = time.perf_counter() - t0
    nodes = sum(i.n_nodes for i in insts)
    return {"value": nodes / dt, "unit": UNIT, "cores": cores, "kind": "oracle", "seconds": dt,
            "sample": f"{k} of the 64 lognormal instances ({nodes} nodes), FMM per instance, "
                      f"one instance per thread"}


def cpu_baseline_tomography(k: int) -> dict:
    """The oracle's forward (fast marching) and adjoint (back substitution) for k of the 16
    shots of the 192^3 tomography at s = 1, one shot per host core."""
    from concurrent.futures import ThreadPoolExecutor
    import numpy as np
    import oracle
    from paper_2106_15869_b300 import workloads as W
    t = W.tomography_3d(192)
    F = 1.0 / np.asarray(t["s_init"], dtype=np.float64)
    rec = t["receivers"]
    shots = [int(s) for s in t["sources"][:k]]
    cores = min(host_cores(), k)

    def one(s):
        phi = oracle.fmm(F, t["h"], [s])
        r = np.zeros(phi.size)
        r[rec] = 1.0
        t1 = time.perf_counter()
        oracle.adjoint(F, t["h"], [s], phi, r.reshape(phi.shape))
        return time.perf_counter() - t1

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        adj_s = list(ex.map(one, shots))
    dt = time.perf_counter() - t0
    nodes = F.size * k
    return {"value": nodes / dt, "unit": "nodes/s (forward + adjoint)", "cores": cores, "kind": "oracle",
            "seconds": dt, "adjoint_share": sum(adj_s) / (dt * cores),
            "sample": f"{k} of the 16 shots, FMM forward + reverse-order adjoint per shot, one shot per thread"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="maze_512",
                    choices=["maze_512", "oscillating_256", "point_source_128", "lognormal_batch64"])
    ap.add_argument("--tile", default="auto")
    ap.add_argument("--schedule", default="auto")
    ap.add_argument("--converge", default="auto", choices=["auto", "confirm", "sweep"])
    ap.add_argument("--method", default="ifim", choices=["ifim", "fim"],
                    help="ifim: Algorithm 2 (the default); fim: the FIM of Sec. 2.3 at tile granularity")
    ap.add_argument("--order", type=float, default=0.0,
                    help="list order: 0 default bucketed, >0 bucket width, <0 unordered")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the secondary workloads, FIM comparison, batched, adjoint and paper examples")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    return run_ours(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
