"""GPU parity of the forward solve (C ABI via the thin Python binding) against
the FP64 CPU oracle, element by element on the same seeded inputs.

Tolerances: FP32 path max|phi_gpu - phi_oracle| <= 1e-4 * max(phi) over finite
nodes, FP64 validation mode <= 1e-10 * max(phi); +inf (unreachable) must
match exactly.  The oracle is fed the float32-rounded speeds so that only the
solver's arithmetic differs.
"""
import numpy as np
import pytest

import oracle
from paper_2106_15869_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL32 = 1e-4
TOL64 = 1e-10


def _torch():
    import torch
    return torch


def gpu_solve(inst, dtype="fp32", **kw):
    torch = _torch()
    from paper_2106_15869_b300 import api
    tdt = torch.float32 if dtype == "fp32" else torch.float64
    F = torch.as_tensor(inst.F, dtype=tdt).cuda()
    phi, st = api.solve(F, inst.src_idx, inst.h, inst.src_val, return_stats=True, **kw)
    assert st["status"] == 0, st
    return phi.cpu().double().numpy(), st


def oracle_phi(inst, dtype="fp32"):
    F = inst.F.astype(np.float32).astype(np.float64) if dtype == "fp32" else inst.F
    val = inst.src_val.astype(np.float32).astype(np.float64) if dtype == "fp32" else inst.src_val
    return oracle.fmm(F, inst.h, inst.src_idx, val)


def assert_parity(got, ref, tol):
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(got)), "reachability differs"
    if not fin.any():
        return 0.0
    scale = float(np.max(np.abs(ref[fin])))
    err = float(np.max(np.abs(got[fin] - ref[fin])))
    assert err <= tol * max(scale, 1e-30), (err, scale, err / max(scale, 1e-30))
    return err / max(scale, 1e-30)


# ------------------------------------------------------------------ workloads
def test_point_source_2d_128():
    inst = W.point_source_2d(128, (64, 64))
    for dt, tol in (("fp32", TOL32), ("fp64", TOL64)):
        got, st = gpu_solve(inst, dt)
        assert_parity(got, oracle_phi(inst, dt), tol)
    # axis exactness survives in FP32 to rounding: phi(64+k, 64) = k h
    got, _ = gpu_solve(inst, "fp32")
    k = np.arange(64)
    assert np.allclose(got[64, 64:], k * inst.h, rtol=2e-6, atol=1e-7)


@pytest.mark.parametrize("tile", ["8x8x8", "4x4x4", "8x8x4", "8x4x4"])
@pytest.mark.parametrize("dtype", ["fp32", "fp64"])
def test_oscillating_3d_small(tile, dtype):
    inst = W.oscillating_3d(45)          # several tiles and a ragged tail for every tile shape
    got, st = gpu_solve(inst, dtype, tile=tile)
    assert_parity(got, oracle_phi(inst, dtype), TOL32 if dtype == "fp32" else TOL64)


@pytest.mark.parametrize("dtype", ["fp32", "fp64"])
def test_maze_small(dtype):
    inst = W.maze_3d(72, seed=3, n_slabs=4, gap=12)
    got, st = gpu_solve(inst, dtype)
    assert_parity(got, oracle_phi(inst, dtype), TOL32 if dtype == "fp32" else TOL64)


@pytest.mark.parametrize("schedule", ["persistent", "hostloop", "async"])
def test_schedules_agree(schedule):
    inst = W.maze_3d(48, seed=7, n_slabs=3, gap=10, n_src=3)
    got, st = gpu_solve(inst, "fp64", schedule=schedule)
    assert_parity(got, oracle_phi(inst, "fp64"), TOL64)


@pytest.mark.parametrize("seed", range(24))
def test_random_small_grids(seed):
    inst = W.random_small(seed, max_edge=21, p_barrier=0.08 if seed % 2 else 0.0)
    for dt, tol in (("fp64", TOL64), ("fp32", TOL32)):
        got, _ = gpu_solve(inst, dt)
        assert_parity(got, oracle_phi(inst, dt), tol)


@pytest.mark.parametrize("ex", [1, 2, 3, 5])
def test_paper_examples_2d(ex):
    inst = W.paper_example_2d(ex, n=150)
    for dt, tol in (("fp32", TOL32), ("fp64", TOL64)):
        got, _ = gpu_solve(inst, dt)
        assert_parity(got, oracle_phi(inst, dt), tol)


def test_lognormal_single_instance():
    inst = W.lognormal_batch(B=2, seed=4, lo=40, hi=70)[1]
    got, _ = gpu_solve(inst, "fp32")
    assert_parity(got, oracle_phi(inst, "fp32"), TOL32)


# ------------------------------------------------------------------ edge cases
@pytest.mark.parametrize("dims", [(1, 1, 1), (1, 1, 9), (17, 1, 1), (1, 13, 1), (9, 9, 1), (3, 5, 7),
                                  (8, 8, 8), (9, 8, 8), (16, 16, 17)])
def test_odd_shapes_and_lines(dims):
    inst = W.random_small(31, dims=dims, three_d=dims[2] > 1)
    got, _ = gpu_solve(inst, "fp64")
    assert_parity(got, oracle_phi(inst, "fp64"), TOL64)


def test_no_sources_gives_all_inf():
    inst = W.random_small(5, dims=(10, 9, 8), three_d=True)
    inst.src_idx = np.zeros(0, dtype=np.int64)
    inst.src_val = np.zeros(0)
    got, _ = gpu_solve(inst, "fp32")
    assert np.all(np.isinf(got))


def test_barrier_wall_and_hole():
    F = np.ones((1, 20, 20))
    F[0, :, 9] = 0.0
    inst = W.Instance("wall", F, 0.1, np.array([0], np.int64), np.zeros(1))
    got, _ = gpu_solve(inst, "fp32")
    assert np.all(np.isinf(got[0, :, 9:]))
    F[0, 19, 9] = 1.0
    got, _ = gpu_solve(inst, "fp64")
    assert_parity(got, oracle_phi(inst, "fp64"), TOL64)


def test_duplicate_sources_and_source_on_barrier():
    F = np.ones((6, 7, 8))
    F[2, 3, 4] = 0.0
    idx = np.array([(2 * 7 + 3) * 8 + 4, 5, 5], dtype=np.int64)
    val = np.array([0.0, 0.3, 0.1])
    inst = W.Instance("dup", F, 0.2, idx, val)
    got, _ = gpu_solve(inst, "fp64")
    assert got.reshape(-1)[5] == 0.1
    assert_parity(got, oracle_phi(inst, "fp64"), TOL64)


def test_source_out_of_range_is_an_error():
    torch = _torch()
    from paper_2106_15869_b300 import api, EikonalError
    F = torch.ones(4, 5, 6, device="cuda")
    with pytest.raises(EikonalError) as e:
        api.solve(F, [0, 4 * 5 * 6], 0.1, return_stats=True)
    assert e.value.code == 1


def test_iteration_cap_reports_noconverge_and_upper_bounds():
    torch = _torch()
    from paper_2106_15869_b300 import api, EikonalError
    inst = W.oscillating_3d(40)
    F = torch.as_tensor(inst.F, dtype=torch.float32).cuda()
    with pytest.raises(EikonalError) as e:
        api.solve(F, inst.src_idx, inst.h, return_stats=True, max_iters=3)
    assert e.value.code == 2
    phi = api.solve(F, inst.src_idx, inst.h, max_iters=3).cpu().double().numpy()
    ref = oracle_phi(inst, "fp32")
    assert np.all(phi >= ref - 1e-4 * ref[np.isfinite(ref)].max())     # iterates are upper bounds


def test_host_tensor_round_trip():
    torch = _torch()
    from paper_2106_15869_b300 import api
    inst = W.oscillating_3d(33)
    phi = api.solve(torch.as_tensor(inst.F, dtype=torch.float32), inst.src_idx, inst.h)
    assert phi.device.type == "cpu"
    assert_parity(phi.double().numpy(), oracle_phi(inst, "fp32"), TOL32)


def test_repeated_calls_reuse_workspace():
    inst = W.maze_3d(40, seed=11, n_slabs=3, gap=8)
    a, _ = gpu_solve(inst, "fp32")
    b, _ = gpu_solve(inst, "fp32")
    ref = oracle_phi(inst, "fp32")
    assert_parity(a, ref, TOL32)
    assert_parity(b, ref, TOL32)


# ------------------------------------------------------------------ remedy ablation
def test_skip_remedy_breaks_parity_where_remedy_is_needed():
    """Sec. 4.2: after Step 2 alone some values are wrong on multi-source /
    variable-speed inputs; Step 3 finds and fixes them."""
    inst = W.maze_3d(64, seed=3, n_slabs=5, gap=10, n_src=4)
    ref = oracle_phi(inst, "fp64")
    full, st = gpu_solve(inst, "fp64")
    assert_parity(full, ref, TOL64)
    assert st["tiles_flagged"] > 0
    upd, st0 = gpu_solve(inst, "fp64", skip_remedy=True)
    fin = np.isfinite(ref)
    err = np.max(np.abs(upd[fin] - ref[fin])) / ref[fin].max()
    assert err > 1e-3, err
    assert np.all(upd[fin] >= ref[fin] - 1e-12)       # Step-2 values are upper bounds


# ------------------------------------------------------------------ batched
def test_batched_uneven_instances():
    from paper_2106_15869_b300 import api
    torch = _torch()
    insts = W.lognormal_batch(B=5, seed=21, lo=20, hi=48) + [W.random_small(3, dims=(13, 7, 5), three_d=True)]
    probs = [(torch.as_tensor(i.F, dtype=torch.float32).cuda(), i.src_idx, i.h, i.src_val) for i in insts]
    outs, st = api.solve_batched(probs, return_stats=True)
    assert st["status"] == 0
    for i, o in zip(insts, outs):
        assert_parity(o.cpu().double().numpy(), oracle_phi(i, "fp32"), TOL32)


def test_batched_shared_speed_many_sources():
    from paper_2106_15869_b300 import api
    torch = _torch()
    t = W.tomography_3d(40, rec_count=4, src_lattice=(5, 20, 35))
    F = 1.0 / t["s_true"]
    Ft = torch.as_tensor(F, dtype=torch.float64).cuda()
    probs = [(Ft, [s], t["h"]) for s in t["sources"]]
    outs = api.solve_batched(probs, shared_F=True)
    for s, o in zip(t["sources"], outs):
        ref = oracle.fmm(F, t["h"], [s])
        assert_parity(o.cpu().numpy(), ref, TOL64)


def test_batched_many_small_instances():
    """1500 small 3D instances (8..20 nodes per edge, one to four sources each) in one
    launch: lists far longer than the thread groups (two-phase iterations over many
    instances); every instance matches the oracle."""
    from paper_2106_15869_b300 import api
    torch = _torch()
    rng = np.random.default_rng(31)
    insts = []
    for q in range(1500):
        d = tuple(int(v) for v in rng.integers(8, 21, size=3))
        insts.append(W.random_small(1000 + q, dims=d, three_d=True))
    probs = [(torch.as_tensor(i.F, dtype=torch.float32).cuda(), i.src_idx, i.h, i.src_val) for i in insts]
    outs, st = api.solve_batched(probs, return_stats=True)
    assert st["status"] == 0, st
    for i, o in zip(insts, outs):
        assert_parity(o.cpu().double().numpy(), oracle_phi(i, "fp32"), TOL32)


# ------------------------------------------------------------------ full-size workloads
def test_full_point_source_2d_128_config():
    inst = W.point_source_2d(128, (64, 64))
    got, _ = gpu_solve(inst, "fp32")
    assert_parity(got, oracle_phi(inst, "fp32"), TOL32)


def test_full_oscillating_256_fp32():
    """The 256^3 oscillating-speed workload at full size, all nodes vs the oracle."""
    inst = W.oscillating_3d(256)
    got, st = gpu_solve(inst, "fp32")
    err = assert_parity(got, oracle_phi(inst, "fp32"), TOL32)
    print("oscillating_3d_256 max rel err", err, st)


def test_many_fronts_two_phase_iterations():
    """A 160^3 oscillating speed with 24 sources: iterations with more visits than
    thread groups (the two-phase classify-then-visit iterations) occur, and the
    result matches the oracle node for node."""
    torch = _torch()
    from paper_2106_15869_b300 import api
    base = W.oscillating_3d(160)
    rng = np.random.default_rng(7)
    idx = np.unique(rng.integers(0, base.F.size, size=24)).astype(np.int64)
    inst = W.Instance("osc160_multi", base.F, base.h, idx, np.zeros(idx.size))
    F = torch.as_tensor(inst.F, dtype=torch.float32).cuda()
    with api.Trace() as tr:
        phi, st = api.solve(F, inst.src_idx, inst.h, return_stats=True)
    assert st["status"] == 0, st
    visits = tr.records[1:, 3]
    groups = 3 * torch.cuda.get_device_properties(0).multi_processor_count   # 256-thread groups launched
    big = visits > groups
    assert np.any(big[:-1] & big[1:]), visits.max()    # an iteration after one with more visits than groups
    assert_parity(phi.cpu().double().numpy(), oracle_phi(inst, "fp32"), TOL32)


# ------------------------------------------------------------------ asynchronous schedule
@pytest.mark.parametrize("seed", range(12))
def test_async_random_small_grids(seed):
    inst = W.random_small(100 + seed, max_edge=25, p_barrier=0.08 if seed % 2 else 0.0)
    got, st = gpu_solve(inst, "fp64", schedule="async")
    assert_parity(got, oracle_phi(inst, "fp64"), TOL64)


@pytest.mark.parametrize("tile", ["4x4x4", "8x4x4", "8x8x4", "8x8x8"])
def test_async_oscillating_and_maze(tile):
    inst = W.oscillating_3d(50)
    got, st = gpu_solve(inst, "fp32", schedule="async", tile=tile)
    assert_parity(got, oracle_phi(inst, "fp32"), TOL32)
    inst = W.maze_3d(56, seed=9, n_slabs=4, gap=9, n_src=3)
    got, st = gpu_solve(inst, "fp32", schedule="async", tile=tile)
    assert_parity(got, oracle_phi(inst, "fp32"), TOL32)


def test_async_batched_and_2d():
    from paper_2106_15869_b300 import api
    torch = _torch()
    insts = W.lognormal_batch(B=4, seed=8, lo=24, hi=40)
    probs = [(torch.as_tensor(i.F, dtype=torch.float32).cuda(), i.src_idx, i.h) for i in insts]
    outs = api.solve_batched(probs, schedule="async")
    for i, o in zip(insts, outs):
        assert_parity(o.cpu().double().numpy(), oracle_phi(i, "fp32"), TOL32)
    inst = W.paper_example_2d(5, n=180)
    got, _ = gpu_solve(inst, "fp32", schedule="async")
    assert_parity(got, oracle_phi(inst, "fp32"), TOL32)


def test_async_skip_remedy_and_cap():
    torch = _torch()
    from paper_2106_15869_b300 import api, EikonalError
    inst = W.maze_3d(48, seed=3, n_slabs=4, gap=8, n_src=3)
    ref = oracle_phi(inst, "fp64")
    upd, st = gpu_solve(inst, "fp64", schedule="async", skip_remedy=True)
    fin = np.isfinite(ref)
    assert np.all(upd[fin] >= ref[fin] - 1e-12)
    F = torch.as_tensor(inst.F, dtype=torch.float32).cuda()
    with pytest.raises(EikonalError) as e:
        api.solve(F, inst.src_idx, inst.h, schedule="async", max_iters=1, return_stats=True)
    assert e.value.code == 2


@pytest.mark.parametrize("schedule", ["persistent", "async"])
@pytest.mark.parametrize("order", [-1.0, 4.0])
def test_converge_sweep_rule(schedule, order):
    """Step-2 convergence taken at sweep granularity reaches the same solution."""
    inst = W.maze_3d(60, seed=5, n_slabs=4, gap=9, n_src=3)
    got, st = gpu_solve(inst, "fp64", schedule=schedule, order=order, converge="sweep")
    assert_parity(got, oracle_phi(inst, "fp64"), TOL64)
    inst = W.oscillating_3d(44)
    got, st = gpu_solve(inst, "fp32", schedule=schedule, order=order, converge="sweep", tile="8x4x4")
    assert_parity(got, oracle_phi(inst, "fp32"), TOL32)


@pytest.mark.parametrize("remedy_order", [2.0, 0.5, -1.0])
@pytest.mark.parametrize("converge", ["auto", "sweep"])
def test_remedy_order_widths(remedy_order, converge):
    """The Step-3 list order alone (bucket widths and unordered), with either Step-2 test,
    reaches the oracle's solution; on 2D grids (Step-2 lists bucketed) it is ignored."""
    inst = W.maze_3d(64, seed=8, n_slabs=4, gap=10, n_src=3)
    got, st = gpu_solve(inst, "fp32", remedy_order=remedy_order, converge=converge)
    assert_parity(got, oracle_phi(inst, "fp32"), TOL32)
    assert st["tiles_flagged"] > 0
    if remedy_order < 0:
        assert st["tiles_deferred"] == 0                     # nothing waits in unordered lists
    inst = W.paper_example_2d(5, 150)
    got, _ = gpu_solve(inst, "fp32", remedy_order=remedy_order, converge=converge)
    assert_parity(got, oracle_phi(inst, "fp32"), TOL32)


def test_trace_records_iterations():
    torch = _torch()
    from paper_2106_15869_b300 import api
    inst = W.oscillating_3d(40)
    F = torch.as_tensor(inst.F, dtype=torch.float32).cuda()
    with api.Trace() as tr:
        phi, st = api.solve(F, inst.src_idx, inst.h, schedule="persistent", return_stats=True)
    s = tr.summary()
    assert s["update"]["iterations"] == st["iters_update"]
    assert s.get("remedy", {}).get("iterations", 0) == st["iters_remedy"]
    assert s["update"]["visited"] == st["tiles_update"]
    assert np.all(np.diff(tr.records[:, 0]) >= 0)


def test_batched_graph_replay_matches_and_updates():
    """The batched solve captured in a CUDA graph: replays match the oracle, and
    a replay after set_speeds solves the new speeds."""
    torch = _torch()
    from paper_2106_15869_b300 import api
    insts = W.lognormal_batch(B=6, seed=31, lo=20, hi=44)
    probs = [(torch.as_tensor(i.F, dtype=torch.float32).cuda(), i.src_idx, i.h) for i in insts]
    bs = api.BatchedSolver(probs, graph=True)
    assert bs.graph is not None
    for _ in range(2):
        outs = bs.solve()
        for i, o in zip(insts, outs):
            assert_parity(o.cpu().double().numpy(), oracle_phi(i, "fp32"), TOL32)
    new = insts[2].F * 2.0
    bs.set_speeds(2, torch.as_tensor(new, dtype=torch.float32).cuda())
    outs = bs.solve()
    ref = oracle.fmm(new.astype(np.float32).astype(np.float64), insts[2].h, insts[2].src_idx)
    assert_parity(outs[2].cpu().double().numpy(), ref, TOL32)
    assert_parity(outs[1].cpu().double().numpy(), oracle_phi(insts[1], "fp32"), TOL32)


# ------------------------------------------------------------------ FIM mode (Sec. 2.3)
@pytest.mark.parametrize("schedule", ["persistent", "hostloop", "async"])
@pytest.mark.parametrize("tile", ["8x8x8", "4x4x4", "8x8x4"])
def test_fim_mode_matches_oracle(schedule, tile):
    """The tile-level FIM (neighbour tiles re-listed when a visit lowers their
    facing boundary, no remedy) reaches the same discrete solution."""
    inst = W.maze_3d(45, seed=11, n_slabs=3, gap=10, n_src=2)
    ref = oracle_phi(inst, "fp64")
    got, st = gpu_solve(inst, "fp64", schedule=schedule, tile=tile, method="fim")
    assert_parity(got, ref, TOL64)
    assert st["iters_update"] == 0 and st["tiles_update"] == 0 and st["tiles_flagged"] == 0
    assert st["tiles_remedy"] > 0


@pytest.mark.parametrize("seed", range(8))
def test_fim_mode_random_small(seed):
    inst = W.random_small(100 + seed, max_edge=21, p_barrier=0.08 if seed % 2 else 0.0)
    for dt, tol in (("fp64", TOL64), ("fp32", TOL32)):
        got, _ = gpu_solve(inst, dt, method="fim")
        assert_parity(got, oracle_phi(inst, dt), tol)


@pytest.mark.parametrize("order", [0.0, -1.0])
def test_fim_mode_2d_and_orders(order):
    inst = W.paper_example_2d(2, n=150)
    for dt, tol in (("fp32", TOL32), ("fp64", TOL64)):
        got, _ = gpu_solve(inst, dt, method="fim", order=order)
        assert_parity(got, oracle_phi(inst, dt), tol)


def test_fim_mode_oracle_point_fim_agrees():
    """The point-wise FIM of the oracle and the tile-level FIM of the library
    end at the same values (both are the discrete solution)."""
    inst = W.oscillating_3d(33)
    fim, _ = oracle.fim(inst.F, inst.h, inst.src_idx, inst.src_val)
    got, _ = gpu_solve(inst, "fp64", method="fim")
    assert_parity(got, fim, TOL64)


def test_fim_mode_batched():
    torch = _torch()
    from paper_2106_15869_b300 import api
    insts = W.lognormal_batch(B=3, seed=9, lo=20, hi=40)
    probs = [(torch.as_tensor(i.F, dtype=torch.float64).cuda(), i.src_idx, i.h) for i in insts]
    phis, st = api.solve_batched(probs, method="fim", return_stats=True)
    assert st["status"] == 0
    for inst, phi in zip(insts, phis):
        assert_parity(phi.cpu().numpy(), oracle_phi(inst, "fp64"), TOL64)


# ------------------------------------------------------------------ unequal spacings (Alg 1.2, eq. 5/6 with dx, dy, dz)
def _aniso_case(seed, dims, hs, three_d=True):
    inst = W.random_small(seed, dims=dims, three_d=three_d, f_lo=0.2, f_hi=5.0, max_src=3)
    return inst, hs


def _gpu_solve_h(inst, h, dtype, **kw):
    torch = _torch()
    from paper_2106_15869_b300 import api
    tdt = torch.float32 if dtype == "fp32" else torch.float64
    F = torch.as_tensor(inst.F, dtype=tdt).cuda()
    phi, st = api.solve(F, inst.src_idx, h, inst.src_val, return_stats=True, **kw)
    assert st["status"] == 0, st
    return phi.cpu().double().numpy()


def _oracle_h(inst, h, dtype):
    F = inst.F.astype(np.float32).astype(np.float64) if dtype == "fp32" else inst.F
    val = inst.src_val.astype(np.float32).astype(np.float64) if dtype == "fp32" else inst.src_val
    return oracle.fmm(F, h, inst.src_idx, val)


@pytest.mark.parametrize("tile", ["8x8x8", "4x4x4", "8x8x4"])
@pytest.mark.parametrize("method", ["ifim", "fim"])
def test_unequal_spacings_3d(tile, method):
    inst, hs = _aniso_case(41, (37, 29, 23), (0.05, 0.11, 0.023))
    for dt, tol in (("fp64", TOL64), ("fp32", TOL32)):
        # the oracle gets the spacings in single precision for the FP32 run: only arithmetic differs
        h_or = tuple(float(np.float32(v)) for v in hs) if dt == "fp32" else hs
        got = _gpu_solve_h(inst, hs, dt, tile=tile, method=method)
        assert_parity(got, _oracle_h(inst, h_or, dt), tol)


@pytest.mark.parametrize("schedule", ["hostloop", "async"])
def test_unequal_spacings_schedules(schedule):
    inst, hs = _aniso_case(43, (33, 21, 19), (1.0, 0.4, 2.5))
    got = _gpu_solve_h(inst, hs, "fp64", schedule=schedule)
    assert_parity(got, _oracle_h(inst, hs, "fp64"), TOL64)


def test_unequal_spacings_2d_and_axis_exactness():
    inst, hs = _aniso_case(47, (70, 45, 1), (0.3, 0.07), three_d=False)
    for dt, tol in (("fp64", TOL64), ("fp32", TOL32)):
        h_or = tuple(float(np.float32(v)) for v in hs) if dt == "fp32" else hs
        got = _gpu_solve_h(inst, hs, dt)
        assert_parity(got, _oracle_h(inst, h_or, dt), tol)
    # F = 1, corner source: phi along the axes is k dx and k dy
    one = W.point_source_2d(64, (0, 0))
    got = _gpu_solve_h(one, (0.5, 2.0), "fp64")
    assert np.allclose(got[0, :], 0.5 * np.arange(64), rtol=1e-14, atol=0)
    assert np.allclose(got[:, 0], 2.0 * np.arange(64), rtol=1e-14, atol=0)


def test_unequal_spacings_batched_and_adjoint_rejects():
    torch = _torch()
    from paper_2106_15869_b300 import api, _lib
    a, _ = _aniso_case(51, (20, 17, 13), None)
    b, _ = _aniso_case(52, (15, 22, 9), None)
    ha, hb = (0.1, 0.3, 0.2), (0.05, 0.15, 0.1)            # same ratios
    probs = [(torch.as_tensor(a.F).cuda(), a.src_idx, ha, torch.as_tensor(a.src_val).cuda()),
             (torch.as_tensor(b.F).cuda(), b.src_idx, hb, torch.as_tensor(b.src_val).cuda())]
    phis = api.solve_batched(probs)
    assert_parity(phis[0].cpu().numpy(), oracle.fmm(a.F, ha, a.src_idx, a.src_val), TOL64)
    assert_parity(phis[1].cpu().numpy(), oracle.fmm(b.F, hb, b.src_idx, b.src_val), TOL64)
    with pytest.raises(_lib.EikonalError):
        api.solve_batched([probs[0], (probs[1][0], b.src_idx, (0.05, 0.1, 0.1))])
    r = torch.ones_like(phis[0])
    with pytest.raises(_lib.EikonalError):
        api.adjoint(probs[0][0], a.src_idx, ha, phis[0], r)
