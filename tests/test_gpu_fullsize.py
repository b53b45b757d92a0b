"""Parity at the full workload sizes, in the launch configuration bench.py times
(default options; the 64-instance batch replayed from a CUDA graph): every node
against the oracle's fast marching (FP64, fed the FP32-rounded speeds), FP32
within 1e-4 max|phi|, +inf exactly.  The oracle runs on the host cores in a
thread pool (ctypes releases the GIL).  Tomography at 192^3 with 16 shots and
256 receivers: the adjoint gradient against central finite differences of FP64
solves at 32 interior cells (eps 1e-3, aggregate relative error 1e-3) at the
configured initial slowness s = 1, and the FP32 adjoint against the FP64 one;
and, for two shots, the FP64 GPU adjoint node by node against the oracle's
adjoint on the same phi (1e-10 of max |g|)."""
import os
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_2106_15869_b300 import workloads as W

pytestmark = pytest.mark.gpu
TOL32 = 1e-4


def _pool():
    return ThreadPoolExecutor(max_workers=max(1, min(32, os.cpu_count() or 1)))


def _oracle32(inst):
    F = inst.F.astype(np.float32).astype(np.float64)
    val = np.asarray(inst.src_val, dtype=np.float32).astype(np.float64)
    return oracle.fmm(F, inst.h, inst.src_idx, val)


def _parity(got, ref, tol):
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(got)), "reachability differs"
    scale = float(np.max(np.abs(ref[fin])))
    err = float(np.max(np.abs(got[fin] - ref[fin])))
    assert err <= tol * scale, (err, scale)
    return err / scale


def test_full_maze_512_fp32():
    import torch
    from paper_2106_15869_b300 import api
    inst = W.maze_3d(512)
    F = torch.as_tensor(inst.F, dtype=torch.float32).cuda()
    phi, st = api.solve(F, inst.src_idx, inst.h, torch.as_tensor(inst.src_val, dtype=torch.float32).cuda(),
                        return_stats=True)
    assert st["status"] == 0, st
    got = phi.cpu().numpy().astype(np.float64)
    del phi, F
    t0 = time.perf_counter()
    ref = _oracle32(inst)
    err = _parity(got, ref, TOL32)
    print(f"maze 512^3: max rel err {err:.2e}, oracle {time.perf_counter() - t0:.0f} s, {st}")


def test_full_lognormal_batch64_graph_replay():
    import torch
    from paper_2106_15869_b300 import api
    insts = W.lognormal_batch(64)
    probs = [(torch.as_tensor(i.F, dtype=torch.float32).cuda(), i.src_idx, i.h) for i in insts]
    bs = api.BatchedSolver(probs, graph=True)
    bs.solve()
    phis = [p.cpu().numpy().astype(np.float64) for p in bs.solve()]        # a replay, as timed
    with _pool() as ex:
        refs = list(ex.map(_oracle32, insts))
    worst = max(_parity(g, r, TOL32) for g, r in zip(phis, refs))
    print(f"lognormal batch of 64: max rel err {worst:.2e}")


def test_full_tomography_192_gradient():
    import torch
    from paper_2106_15869_b300 import api
    t = W.tomography_3d(192)
    h, rec = t["h"], t["receivers"]
    shots = [np.array([s]) for s in t["sources"]]
    s_true = t["s_true"]
    s0 = np.asarray(t["s_init"], dtype=np.float64)       # the configured initial model, s = 1
    assert np.all(s0 == 1.0)
    with _pool() as ex:
        obs = list(ex.map(lambda sh: oracle.fmm(1.0 / s_true, h, sh).reshape(-1)[rec], shots))
    rec_d = torch.as_tensor(rec).cuda()
    obs_d = [torch.as_tensor(o).cuda() for o in obs]

    def loss_and_phis(s, dtype=torch.float64):
        F = torch.as_tensor(1.0 / s, dtype=dtype).cuda()
        phis = api.solve_batched([(F, sh, h) for sh in shots], shared_F=True)
        L = sum(0.5 * float(torch.sum((ph.reshape(-1)[rec_d].double() - obs_d[q]) ** 2)) for q, ph in enumerate(phis))
        return L, phis, F

    def gradient(s, dtype):
        _, phis, F = loss_and_phis(s, dtype)
        rs = []
        for q, ph in enumerate(phis):
            r = torch.zeros_like(ph).reshape(-1)
            r[rec_d] = (ph.reshape(-1)[rec_d].double() - obs_d[q]).to(dtype)
            rs.append(r.view(ph.shape))
        g = api.adjoint_batched([(F, sh, h) for sh in shots], phis, rs, shared_F=True, sum_instances=True)
        return g.double().cpu().numpy().reshape(-1)

    g64 = gradient(s0, torch.float64)
    g32 = gradient(s0, torch.float32)
    assert np.linalg.norm(g32 - g64) <= 1e-3 * np.linalg.norm(g64)
    n = 192
    rng = np.random.default_rng(55)
    cells = rng.integers(8, n - 8, size=(32, 3))
    eps = 1e-3
    fd, adj = [], []
    for (i, j, k) in cells:
        c = (k * n + j) * n + i
        sp = s0.copy().reshape(-1); sp[c] += eps
        sm = s0.copy().reshape(-1); sm[c] -= eps
        fd.append((loss_and_phis(sp.reshape(s0.shape))[0] - loss_and_phis(sm.reshape(s0.shape))[0]) / (2 * eps))
        adj.append(g64[c])
    fd, adj = np.array(fd), np.array(adj)
    rel = np.linalg.norm(adj - fd) / max(np.linalg.norm(fd), 1e-300)
    print(f"tomography 192^3: |adj - fd| / |fd| = {rel:.2e} over 32 cells; fp32 vs fp64 "
          f"{np.linalg.norm(g32 - g64) / np.linalg.norm(g64):.2e}")
    assert rel <= 1e-3, (adj, fd)


def test_full_tomography_192_fp64_adjoint_vs_oracle():
    """The 192^3 FP64 GPU adjoint of two shots (receivers on the bottom face, r = 1 there)
    against the oracle's back substitution on the same GPU phi, node by node."""
    import torch
    from paper_2106_15869_b300 import api
    t = W.tomography_3d(192)
    h, rec = t["h"], t["receivers"]
    F = 1.0 / np.asarray(t["s_init"], dtype=np.float64)
    Fd = torch.as_tensor(F).cuda()
    for s in (t["sources"][0], t["sources"][5]):
        phi = api.solve(Fd, [int(s)], h)
        r = torch.zeros_like(phi).reshape(-1)
        r[torch.as_tensor(rec).cuda()] = 1.0
        r = r.view(phi.shape)
        got = api.adjoint(Fd, [int(s)], h, phi, r).cpu().numpy()
        want = oracle.adjoint(F, h, [int(s)], phi.cpu().numpy(), r.cpu().numpy())
        scale = float(np.max(np.abs(want)))
        err = float(np.max(np.abs(got - want)))
        assert err <= 1e-10 * scale, (s, err, scale)
        print(f"tomography 192^3 shot {s}: fp64 adjoint vs oracle max rel err {err / scale:.2e}")
