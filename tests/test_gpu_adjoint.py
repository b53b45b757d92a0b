"""GPU adjoint (dL/d slowness) against the FP64 CPU oracle's adjoint, finite
differences of FP64 GPU solves, and exact identities (1D, homogeneity).

The GPU adjoint is fed the oracle's phi where the comparison should isolate
the adjoint; FP64 mode must match the oracle to 1e-10 (relative to max |g|),
FP32 to 1e-3 (relative L2), finite differences to 1e-3 (aggregate over the
checked cells, excluding cells whose upwind branch selection flips between
the +-eps solves).
"""
import numpy as np
import pytest

import oracle
from paper_2106_15869_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def gpu_adjoint(F, h, src, phi, r, dtype="fp64", **kw):
    torch = _torch()
    from paper_2106_15869_b300 import api
    t = torch.float64 if dtype == "fp64" else torch.float32
    g = api.adjoint(torch.as_tensor(F, dtype=t).cuda(), src, h, torch.as_tensor(phi, dtype=t).cuda(),
                    torch.as_tensor(r, dtype=t).cuda(), **kw)
    return g.cpu().double().numpy()


@pytest.mark.parametrize("seed", range(10))
def test_adjoint_fp64_matches_oracle(seed):
    inst = W.random_small(700 + seed, max_edge=18, three_d=seed % 3 != 0, f_lo=0.3, f_hi=3.0,
                          p_barrier=0.05 if seed % 2 else 0.0)
    inst.src_val[:] = 0.0
    phi = oracle.fmm(inst.F, inst.h, inst.src_idx)
    rng = np.random.default_rng(seed)
    r = np.where(np.isfinite(phi) & (rng.random(phi.shape) < 0.3), rng.standard_normal(phi.shape), 0.0)
    want = oracle.adjoint(inst.F, inst.h, inst.src_idx, phi, r)
    for tile, order in (("8x8x4", 0.0), ("4x4x4", 0.0), ("8x8x8", 0.0), ("8x8x4", -1.0), ("4x4x4", 1.0)):
        got = gpu_adjoint(inst.F, inst.h, inst.src_idx, phi, r, "fp64", tile=tile, order=order)
        scale = max(np.max(np.abs(want)), 1e-300)
        assert np.max(np.abs(got - want)) <= 1e-10 * scale, tile


def test_adjoint_2d_tiles():
    inst = W.paper_example_2d(5, n=90)
    phi = oracle.fmm(inst.F, inst.h, inst.src_idx, inst.src_val)
    r = np.zeros_like(phi)
    r[-1, :] = 1.0
    r[np.isinf(phi)] = 0.0
    want = oracle.adjoint(inst.F, inst.h, inst.src_idx, phi, r)
    got = gpu_adjoint(inst.F, inst.h, inst.src_idx, phi, r, "fp64")
    assert np.max(np.abs(got - want)) <= 1e-10 * np.max(np.abs(want))


def test_adjoint_1d_exact():
    n = 40
    F = np.linspace(0.5, 2.0, n).reshape(1, 1, n)
    h = 0.2
    phi = oracle.fmm(F, h, [0])
    r = np.zeros_like(phi)
    r[0, 0, n - 1] = 1.0
    g = gpu_adjoint(F, h, [0], phi, r, "fp64")
    assert g[0, 0, 0] == 0.0
    assert np.allclose(g[0, 0, 1:], h, rtol=1e-12, atol=0)


def test_adjoint_homogeneity_identity_fp32():
    t = W.tomography_3d(48, src_lattice=(6, 18, 30, 42), rec_count=8, rec_start=3, rec_step=6)
    F = 1.0 / t["s_true"]
    src = t["sources"][:1]
    phi = oracle.fmm(F.astype(np.float32).astype(np.float64), t["h"], src)
    r = np.zeros_like(phi)
    r.reshape(-1)[t["receivers"]] = np.linspace(-1, 1, t["receivers"].size)
    g = gpu_adjoint(F, t["h"], src, phi, r, "fp32")
    lhs = float(np.sum(t["s_true"] * g))
    rhs = float(np.sum(r * phi))
    assert lhs == pytest.approx(rhs, rel=2e-4)


def test_adjoint_fp32_vs_fp64_oracle():
    t = W.tomography_3d(64, src_lattice=(8, 24, 40, 56), rec_count=8, rec_start=4, rec_step=8)
    F = 1.0 / t["s_true"]
    src = t["sources"][5:6]
    phi = oracle.fmm(F, t["h"], src)
    r = np.zeros_like(phi)
    r.reshape(-1)[t["receivers"]] = 1.0
    want = oracle.adjoint(F, t["h"], src, phi, r)
    got = gpu_adjoint(F, t["h"], src, phi, r, "fp32")
    assert np.linalg.norm(got - want) <= 1e-3 * np.linalg.norm(want)


def test_adjoint_matches_central_differences_fp64():
    """Tomography loss 0.5 sum (phi_rec - phi_obs)^2 over shots; gradient vs
    central differences (FP64 GPU solves, eps 1e-3 on slowness) at random cells."""
    torch = _torch()
    from paper_2106_15869_b300 import api
    t = W.tomography_3d(40, src_lattice=(8, 20, 32), rec_count=6, rec_start=5, rec_step=6)
    s_true, h = t["s_true"], t["h"]
    shots = [np.array([s]) for s in t["sources"][:4]]
    rec = t["receivers"]
    s0 = 1.0 + 0.5 * (s_true - 1.0)             # a model between the start and the truth
    obs = [oracle.fmm(1.0 / s_true, h, sh).reshape(-1)[rec] for sh in shots]

    def loss_and_phis(s):
        F = torch.as_tensor(1.0 / s, dtype=torch.float64).cuda()
        phis = api.solve_batched([(F, sh, h) for sh in shots], shared_F=True)
        L = 0.0
        for q, ph in enumerate(phis):
            L += 0.5 * float(torch.sum((ph.reshape(-1)[torch.as_tensor(rec).cuda()] - torch.as_tensor(obs[q]).cuda()) ** 2))
        return L, phis

    L0, phis = loss_and_phis(s0)
    rs = []
    for q, ph in enumerate(phis):
        r = torch.zeros_like(ph).reshape(-1)
        r[torch.as_tensor(rec).cuda()] = ph.reshape(-1)[torch.as_tensor(rec).cuda()] - torch.as_tensor(obs[q]).cuda()
        rs.append(r.view(ph.shape))
    F0 = torch.as_tensor(1.0 / s0, dtype=torch.float64).cuda()
    g = api.adjoint_batched([(F0, sh, h) for sh in shots], phis, rs, shared_F=True, sum_instances=True)
    g = g.cpu().numpy().reshape(-1)
    rng = np.random.default_rng(55)
    interior = [((k * 40 + j) * 40 + i) for k in range(4, 36) for j in range(4, 36) for i in range(4, 36)]
    cells = rng.choice(interior, size=32, replace=False)
    eps = 1e-3
    fd = []
    for c in cells:
        sp = s0.copy().reshape(-1); sp[c] += eps
        sm = s0.copy().reshape(-1); sm[c] -= eps
        fd.append((loss_and_phis(sp.reshape(s0.shape))[0] - loss_and_phis(sm.reshape(s0.shape))[0]) / (2 * eps))
    fd = np.array(fd)
    adj = g[cells]
    assert np.linalg.norm(adj - fd) <= 1e-3 * max(np.linalg.norm(fd), 1e-12), (adj, fd)


def test_eikonal_fn_backward_sums_shots():
    torch = _torch()
    from paper_2106_15869_b300 import api
    t = W.tomography_3d(32, src_lattice=(6, 16, 26), rec_count=4, rec_start=4, rec_step=8)
    s = torch.as_tensor(t["s_true"], dtype=torch.float64).cuda().requires_grad_(True)
    shots = [[int(x)] for x in t["sources"][:3]]
    phi = api.EikonalFn.apply(s, shots, t["h"])
    rec = torch.as_tensor(t["receivers"]).cuda()
    loss = 0.5 * (phi.reshape(len(shots), -1)[:, rec] ** 2).sum()
    loss.backward()
    # the same gradient from one oracle adjoint per shot, summed
    want = np.zeros(s.shape)
    for q, sh in enumerate(shots):
        ph = phi[q].detach().cpu().numpy()
        r = np.zeros_like(ph)
        r.reshape(-1)[t["receivers"]] = ph.reshape(-1)[t["receivers"]]
        want += oracle.adjoint(1.0 / t["s_true"], t["h"], sh, ph, r)
    got = s.grad.cpu().numpy()
    assert np.max(np.abs(got - want)) <= 1e-10 * np.max(np.abs(want))


@pytest.mark.parametrize("dtype", ["fp32", "fp64"])
def test_shared_gradient_block_is_deterministic(dtype):
    """Instances summing into one gradient block add in instance order without
    atomics: repeated calls are bit-identical, and the sum matches the
    per-instance gradients added on the host."""
    torch = _torch()
    from paper_2106_15869_b300 import api
    t = torch.float64 if dtype == "fp64" else torch.float32
    w = W.tomography_3d(40, src_lattice=(5, 20, 35), rec_count=6, rec_start=3, rec_step=6)
    F = torch.as_tensor(1.0 / w["s_true"], dtype=t).cuda()
    probs = [(F, [int(s)], w["h"]) for s in w["sources"][:9]]
    phis = api.solve_batched(probs, shared_F=True)
    rec = torch.as_tensor(w["receivers"]).cuda()
    rs = []
    for ph in phis:
        r = torch.zeros_like(ph).reshape(-1)
        r[rec] = 1.0
        rs.append(r.view(ph.shape))
    runs = [api.adjoint_batched(probs, phis, rs, shared_F=True, sum_instances=True) for _ in range(3)]
    assert all(torch.equal(runs[0], g) for g in runs[1:])
    sep = api.adjoint_batched(probs, phis, rs, shared_F=True)
    want = torch.stack(sep).double().sum(0)
    tol = 1e-12 if dtype == "fp64" else 1e-5
    assert float((runs[0].double() - want).abs().max()) <= tol * float(want.abs().max())
    assert float(want.abs().max()) > 0


def test_interleaved_gradient_blocks_through_the_c_abi():
    """Four instances writing two gradient blocks in the order A, B, A, B (offsets
    0, N, 0, N): each block holds the sum of its two instances' gradients, and a
    repeated call gives the same bits."""
    import ctypes
    torch = _torch()
    from paper_2106_15869_b300 import _lib, api
    w = W.tomography_3d(32, src_lattice=(6, 16, 26), rec_count=4, rec_start=4, rec_step=8)
    F = torch.as_tensor(1.0 / w["s_true"], dtype=torch.float64).cuda()
    shots = [[int(s)] for s in w["sources"][:4]]
    probs = [(F, sh, w["h"]) for sh in shots]
    phis = api.solve_batched(probs, shared_F=True)
    rec = torch.as_tensor(w["receivers"]).cuda()
    rs = []
    for ph in phis:
        r = torch.zeros_like(ph).reshape(-1)
        r[rec] = ph.reshape(-1)[rec]
        rs.append(r.view(ph.shape))
    sep = api.adjoint_batched(probs, phis, rs, shared_F=True)
    want = [(sep[0] + sep[2]).reshape(-1), (sep[1] + sep[3]).reshape(-1)]
    N = F.numel()
    lib = _lib.load()
    dims = [(32, 32, 32, w["h"])] * 4
    grids = _lib.grids_array(dims)
    opt = _lib.make_options(precision="fp64")
    nbytes = lib.eik_adjoint_workspace_size_batched(4, grids, ctypes.byref(opt))
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    base = (ws.data_ptr() + 255) // 256 * 256
    phi_packed = torch.cat([p.reshape(-1) for p in phis])
    r_packed = torch.cat([r.reshape(-1) for r in rs])
    src = torch.as_tensor([s[0] for s in shots], dtype=torch.int64).cuda()
    off = _lib.i64_array([0, N, 2 * N, 3 * N])
    outs = []
    for _ in range(2):
        g = torch.zeros(2 * N, dtype=torch.float64, device="cuda")
        rc = lib.eik_adjoint_batched(4, grids, F.data_ptr(), _lib.i64_array([0, 0, 0, 0]), phi_packed.data_ptr(), off,
                                     src.data_ptr(), _lib.i64_array([0, 1, 2, 3, 4]), r_packed.data_ptr(),
                                     g.data_ptr(), _lib.i64_array([0, N, 0, N]), base, nbytes, None,
                                     ctypes.byref(opt), None)
        _lib.check(rc)
        torch.cuda.synchronize()
        outs.append(g)
    assert torch.equal(outs[0], outs[1])
    for k in range(2):
        got = outs[0][k * N:(k + 1) * N]
        assert float((got - want[k]).abs().max()) <= 1e-12 * float(want[k].abs().max())
    assert float(want[0].abs().max()) > 0 and float(want[1].abs().max()) > 0
