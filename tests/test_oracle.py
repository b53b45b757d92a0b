"""Pins for the FP64 CPU oracle, against what the paper and the mathematics fix.

None of these re-types the oracle's own cascade: they check closed forms,
invariants, an independent algorithm (Gauss-Seidel sweeping, Sec. 2.2),
the paper's own algorithm run point by point (Algorithm 2), residuals of
eq. (6) written in its "^+" form, refinement toward the Euclidean distance,
and finite differences.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2106_15869_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append([float(v) for v in line.split()])
    return rows


# ---------------------------------------------------------------- local solve
def test_local_solve_golden_closed_forms():
    """Alg 1.1 / 1.3 roots of eq. (4)/(6) on a unit grid (tests/golden/local_solve.txt)."""
    rows = _golden_rows("local_solve.txt")
    assert len(rows) >= 10
    for ax, ay, az, tau, want in rows:
        got = oracle.local_solve(ax, ay, az, tau)
        if math.isinf(want):
            assert math.isinf(got) and got > 0
        else:
            assert got == pytest.approx(want, rel=4e-16, abs=0), (ax, ay, az, tau)


def _plus_residual(u, a, tau):
    return sum(max(u - v, 0.0) ** 2 for v in a if math.isfinite(v)) - tau * tau


def test_local_solve_satisfies_eq6_and_is_upwind():
    """The root solves sum ((u - a_d)^+)^2 = tau^2 and lies in [a1 + tau/sqrt(3), a1 + tau]."""
    rng = np.random.default_rng(0)
    for _ in range(20000):
        a = list(rng.uniform(0, 3, size=3))
        k = rng.integers(0, 4)
        for q in range(k):
            a[q] = math.inf
        tau = float(rng.uniform(0.01, 2.0))
        u = oracle.local_solve(*a, tau)
        fin = [v for v in a if math.isfinite(v)]
        if not fin:
            assert math.isinf(u)
            continue
        a1 = min(fin)
        assert a1 + tau / math.sqrt(3) - 1e-12 <= u <= a1 + tau + 1e-12
        assert abs(_plus_residual(u, a, tau)) <= 1e-12 * max(1.0, tau * tau)


def test_local_solve_symmetry_shift_and_scale():
    rng = np.random.default_rng(1)
    for _ in range(2000):
        a = rng.uniform(0, 1, size=3)
        tau = float(rng.uniform(0.05, 1.0))
        u = oracle.local_solve(*a, tau)
        for perm in ([1, 0, 2], [2, 1, 0], [1, 2, 0]):
            assert oracle.local_solve(*a[perm], tau) == pytest.approx(u, rel=1e-14)
        assert oracle.local_solve(*(a + 5.0), tau) == pytest.approx(u + 5.0, rel=1e-13)
        assert oracle.local_solve(*(3.0 * a), 3.0 * tau) == pytest.approx(3.0 * u, rel=1e-13)


def test_local_solve_monotone_in_neighbours():
    """Godunov scheme monotonicity: raising a neighbour minimum never lowers u."""
    rng = np.random.default_rng(2)
    for _ in range(5000):
        a = rng.uniform(0, 1, size=3)
        tau = float(rng.uniform(0.05, 1.0))
        u = oracle.local_solve(*a, tau)
        b = a.copy()
        b[rng.integers(0, 3)] += float(rng.uniform(0, 0.5))
        assert oracle.local_solve(*b, tau) >= u - 1e-15


# ---------------------------------------------------------------- FMM vs GS vs Alg 2
@pytest.mark.parametrize("seed", range(40))
def test_fmm_equals_gauss_seidel_and_algorithm2(seed):
    """P5/P7: fast marching, alternating-sweep Gauss-Seidel (Sec. 2.2),
    Algorithm 2 and the fast iterative method of Sec. 2.3 reach the same
    discrete solution (Sec. 4.1 reports identical output from every method)."""
    inst = W.random_small(seed, max_edge=12, p_barrier=0.1 if seed % 3 == 0 else 0.0)
    phi = oracle.fmm(inst.F, inst.h, inst.src_idx, inst.src_val)
    gs, rounds = oracle.gs(inst.F, inst.h, inst.src_idx, inst.src_val)
    ifim, st = oracle.ifim(inst.F, inst.h, inst.src_idx, inst.src_val)
    fim, _ = oracle.fim(inst.F, inst.h, inst.src_idx, inst.src_val)
    fin = np.isfinite(phi)
    assert np.array_equal(fin, np.isfinite(gs)) and np.array_equal(fin, np.isfinite(ifim))
    assert np.array_equal(fin, np.isfinite(fim))
    scale = max(1.0, float(np.max(np.abs(phi[fin]))) if fin.any() else 1.0)
    assert np.max(np.abs(phi[fin] - gs[fin]), initial=0) <= 1e-13 * scale
    assert np.max(np.abs(phi[fin] - ifim[fin]), initial=0) <= 1e-13 * scale
    assert np.max(np.abs(phi[fin] - fim[fin]), initial=0) <= 1e-13 * scale


def test_fmm_equals_gs_on_odd_shapes():
    for dims in [(1, 1, 1), (7, 1, 1), (1, 9, 1), (1, 1, 6), (13, 7, 5), (5, 13, 7), (3, 3, 17)]:
        inst = W.random_small(123, dims=dims, three_d=True)
        phi = oracle.fmm(inst.F, inst.h, inst.src_idx, inst.src_val)
        gs, _ = oracle.gs(inst.F, inst.h, inst.src_idx, inst.src_val)
        assert np.allclose(phi, gs, rtol=1e-13, atol=0), dims


# ---------------------------------------------------------------- residual, causality
@pytest.mark.parametrize("seed", range(10))
def test_residual_zero_and_causality(seed):
    """P3/P4: eq. (6) holds at every reachable non-source node; every such node
    has an upwind neighbour lower by between tau/sqrt(d) and tau."""
    inst = W.random_small(1000 + seed, max_edge=20, p_barrier=0.05)
    phi = oracle.fmm(inst.F, inst.h, inst.src_idx, inst.src_val)
    assert oracle.residual(inst.F, inst.h, inst.src_idx, phi) <= 1e-12
    nx, ny, nz = inst.dims
    P = phi.reshape(nz, ny, nx)
    F = inst.F.reshape(nz, ny, nx)
    pad = np.pad(P, 1, constant_values=np.inf)
    nbmin = np.minimum.reduce([pad[:-2, 1:-1, 1:-1], pad[2:, 1:-1, 1:-1], pad[1:-1, :-2, 1:-1],
                               pad[1:-1, 2:, 1:-1], pad[1:-1, 1:-1, :-2], pad[1:-1, 1:-1, 2:]])
    src = np.zeros(P.size, bool)
    src[inst.src_idx] = True
    src = src.reshape(P.shape)
    m = np.isfinite(P) & ~src
    tau = inst.h / F[m]
    d = 3 if nz > 1 else 2
    gap = P[m] - nbmin[m]
    assert np.all(gap <= tau * (1 + 1e-12))
    assert np.all(gap >= tau / math.sqrt(d) * (1 - 1e-12))
    assert np.all(P[np.isfinite(P)] >= inst.src_val.min() - 1e-15)


def test_fmm_acceptance_order_is_monotone():
    inst = W.random_small(77, dims=(11, 9, 8), three_d=True)
    inst.src_val[:] = 0.0
    phi, order = oracle.fmm(inst.F, inst.h, inst.src_idx, inst.src_val, return_order=True)
    vals = phi.reshape(-1)[order]
    assert np.all(np.diff(vals) >= 0)
    assert order.size == np.isfinite(phi).sum()


# ---------------------------------------------------------------- exactness along axes
def test_axis_exactness_point_source_128():
    """P2: F = 1, point source: phi along the grid lines through the source is k h."""
    inst = W.point_source_2d(128, (64, 64))
    phi = oracle.fmm(inst.F, inst.h, inst.src_idx)
    k = np.arange(64)
    assert np.allclose(phi[64, 64:128], k * inst.h, rtol=1e-14, atol=0)
    assert np.allclose(phi[64, 64::-1], np.arange(65) * inst.h, rtol=1e-14, atol=0)
    assert np.allclose(phi[64:128, 64], k * inst.h, rtol=1e-14, atol=0)
    # symmetry of the constant-speed point-source solution
    assert np.array_equal(phi[64 - 10:64 + 11, 64 - 10:64 + 11], phi[64 - 10:64 + 11, 64 - 10:64 + 11].T)


def test_one_dimensional_sum_of_travel_times():
    """A 1D grid is always one-sided: phi_k = sum_{j<=k} h / F_j exactly."""
    rng = np.random.default_rng(5)
    F = rng.uniform(0.2, 3.0, size=50)
    phi = oracle.fmm(F.reshape(1, 50), 0.1, [0])
    want = np.concatenate([[0.0], np.cumsum(0.1 / F[1:])])
    assert np.allclose(phi[0], want, rtol=1e-14, atol=0)
    # the same line embedded in 3D, with a slab of different speed
    F3 = np.ones((5, 5, 40))
    F3[:, :, 10:20] = 0.25
    phi3 = oracle.fmm(F3, 0.5, [(2 * 5 + 2) * 40 + 0])
    line = phi3[2, 2]
    want3 = np.concatenate([[0.0], np.cumsum(0.5 / F3[2, 2, 1:])])
    assert np.allclose(line, want3, rtol=1e-14, atol=0)


def test_barriers_and_unreachable():
    F = np.ones((9, 9))
    F[:, 4] = 0.0                      # full wall
    phi = oracle.fmm(F, 1.0, [0])
    assert np.all(np.isinf(phi[:, 4:]))
    assert np.all(np.isfinite(phi[:, :4]))
    F[0, 4] = 1.0                      # a hole at the top
    phi = oracle.fmm(F, 1.0, [0])
    assert np.all(np.isinf(phi[1:, 4])) and np.isfinite(phi[0, 4])
    assert np.all(np.isfinite(phi[:, 5:]))


def test_duplicate_sources_keep_smaller_value_and_arg_errors():
    F = np.ones((5, 5))
    phi = oracle.fmm(F, 1.0, [12, 12], [0.7, 0.2])
    assert phi[2, 2] == 0.2
    with pytest.raises(ValueError):
        oracle.fmm(np.full((3, 3), np.nan), 1.0, [0])
    with pytest.raises(ValueError):
        oracle.fmm(-np.ones((3, 3)), 1.0, [0])
    with pytest.raises(ValueError):
        oracle.fmm(F, 0.0, [0])
    with pytest.raises(ValueError):
        oracle.fmm(F, 1.0, [25])


# ---------------------------------------------------------------- refinement
def test_first_order_refinement_toward_euclidean_distance():
    """P6: with F = 1 and a disc source initialised exactly, the max error
    against |x| - R falls about 2x per halving of h (first-order scheme)."""
    errs = []
    R = 0.3
    for n in (41, 81, 161, 321):
        xs = np.linspace(-1, 1, n)
        X, Y = np.meshgrid(xs, xs)
        d = np.hypot(X, Y)
        h = xs[1] - xs[0]
        sel = d <= R + h
        idx = np.flatnonzero(sel.reshape(-1))
        val = np.maximum(d.reshape(-1)[idx] - R, 0.0)
        phi = oracle.fmm(np.ones((n, n)), h, idx, val)
        errs.append(np.max(np.abs(phi - np.maximum(d - R, 0.0))))
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(1.6 < r < 2.6 for r in ratios), (errs, ratios)


def test_point_source_refinement_rate():
    """Point source: the error is O(h log 1/h) (the point singularity costs the
    log factor), so err / (h ln(1/h)) stays within a narrow band while h halves
    three times and the log-log slope is near 1 - 1/ln(1/h)."""
    errs, hs = [], []
    for n in (33, 65, 129, 257):
        c = n // 2
        inst = W.point_source_2d(n, (c, c))
        phi = oracle.fmm(inst.F, inst.h, inst.src_idx)
        xs = (np.arange(n) - c) * inst.h
        X, Y = np.meshgrid(xs, xs)
        errs.append(np.max(np.abs(phi - np.hypot(X, Y))))
        hs.append(inst.h)
    hs, errs = np.array(hs), np.array(errs)
    c = errs / (hs * np.log(1.0 / hs))
    assert np.all(np.diff(errs) < 0)
    assert c.max() / c.min() < 1.25, (errs, c)
    slope = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert 0.65 <= slope <= 1.05, (errs, slope)


# ---------------------------------------------------------------- Algorithm 2 behaviour
def test_remedy_needed_only_where_the_paper_says():
    """Sec. 4.2: Example 1 needs no remedy (Fig. 13); Examples 2 and 5 do
    (Figs. 14-15).  Without Step 3 their Step-2 result differs from the
    solution; with it, Algorithm 2 reaches the fast-marching solution."""
    for ex, needs in ((1, False), (2, True), (5, True)):
        inst = W.paper_example_2d(ex, n=101)
        ref = oracle.fmm(inst.F, inst.h, inst.src_idx, inst.src_val)
        upd, st0 = oracle.ifim(inst.F, inst.h, inst.src_idx, inst.src_val, skip_remedy=True)
        full, st = oracle.ifim(inst.F, inst.h, inst.src_idx, inst.src_val)
        scale = np.max(ref[np.isfinite(ref)])
        assert np.max(np.abs(full - ref)) <= 1e-12 * scale
        err_upd = np.max(np.abs(upd - ref))
        if needs:
            assert st["remedy_seed"] > 0 and err_upd > 1e-6 * scale, (ex, st, err_upd)
        else:
            assert st["remedy_seed"] == 0 and err_upd == 0.0, (ex, st, err_upd)
        # Step-2 values are upper bounds of the solution (phi only decreases)
        assert np.all(upd >= ref - 1e-12 * scale)


# ---------------------------------------------------------------- adjoint
def test_adjoint_1d_exact():
    """P8: on a 1D line, d phi_n / d s_k = h for every k in 1..n."""
    n = 30
    F = np.linspace(0.5, 2.0, n).reshape(1, n)
    h = 0.2
    phi = oracle.fmm(F, h, [0])
    r = np.zeros_like(phi)
    r[0, n - 1] = 1.0
    g = oracle.adjoint(F, h, [0], phi, r)
    assert g[0, 0] == 0.0
    assert np.allclose(g[0, 1:], h, rtol=1e-13, atol=0)


@pytest.mark.parametrize("seed", range(6))
def test_adjoint_homogeneity_identity(seed):
    """phi(c s) = c phi(s) with zero-valued sources, so sum_i s_i dL/ds_i = sum_rec r phi_rec."""
    inst = W.random_small(500 + seed, max_edge=14, three_d=True)
    inst.src_val[:] = 0.0
    phi = oracle.fmm(inst.F, inst.h, inst.src_idx, inst.src_val)
    rng = np.random.default_rng(seed)
    r = np.where(np.isfinite(phi), rng.standard_normal(phi.shape), 0.0)
    g = oracle.adjoint(inst.F, inst.h, inst.src_idx, phi, r)
    s = 1.0 / inst.F
    lhs = float(np.sum(s * g))
    rhs = float(np.sum(np.where(np.isfinite(phi), r * phi, 0.0)))
    assert lhs == pytest.approx(rhs, rel=1e-10, abs=1e-12)


@pytest.mark.parametrize("seed", range(4))
def test_adjoint_matches_central_finite_differences(seed):
    """Adjoint vs central differences of the fast-marching solve, in FP64."""
    inst = W.random_small(900 + seed, dims=(9, 8, 7), three_d=True, f_lo=0.5, f_hi=2.0)
    inst.src_val[:] = 0.0
    rng = np.random.default_rng(seed)
    phi = oracle.fmm(inst.F, inst.h, inst.src_idx)
    rec = rng.choice(phi.size, size=6, replace=False)
    target = phi.reshape(-1)[rec] * (1 + 0.1 * rng.standard_normal(6))

    def loss(F):
        p = oracle.fmm(F, inst.h, inst.src_idx).reshape(-1)
        return 0.5 * np.sum((p[rec] - target) ** 2)

    r = np.zeros(phi.size)
    r[rec] = phi.reshape(-1)[rec] - target
    g = oracle.adjoint(inst.F, inst.h, inst.src_idx, phi, r.reshape(phi.shape)).reshape(-1)
    s = (1.0 / inst.F).reshape(-1)
    cells = rng.choice(phi.size, size=12, replace=False)
    eps = 1e-6
    fd = []
    for c in cells:
        sp = s.copy(); sp[c] += eps
        sm = s.copy(); sm[c] -= eps
        fd.append((loss((1 / sp).reshape(phi.shape)) - loss((1 / sm).reshape(phi.shape))) / (2 * eps))
    fd = np.array(fd)
    assert np.linalg.norm(g[cells] - fd) <= 1e-5 * max(np.linalg.norm(fd), 1e-12)


# ---------------------------------------------------------------- unequal spacings (Alg 1.2, eq. 5/6 with dx, dy, dz)
def test_aniso_local_solve_closed_forms():
    inf = np.inf
    # two-sided, a_x = a_y = 0, dx = 1, dy = 2, F = 1: u^2 + (u/2)^2 = 1
    assert abs(oracle.local_solve_aniso(0, 0, inf, 1, 2, 1, 1) - 2 / np.sqrt(5)) < 1e-15
    # three-sided, all minima 0, spacings 1, 2, 3: u^2 (1 + 1/4 + 1/9) = 1, u = 6/7
    assert abs(oracle.local_solve_aniso(0, 0, 0, 1, 2, 3, 1) - 6 / 7) < 1e-15
    # one-sided along x, valid: u = a_x + dx / F
    assert oracle.local_solve_aniso(0, 5, inf, 1, 1, 1, 2) == 0.5
    # the printed switch of Alg 1.2 (|a_x - a_y| > sqrt(dx^2 + dy^2) / F) would take the
    # two-sided root here, which lies below a_x; the valid root is one-sided along y
    assert oracle.local_solve_aniso(1.5, 0, inf, 2, 1, 1, 1) == 1.0
    assert oracle.local_solve_aniso(1.2, 0, inf, 1, 1, 1, 1) == 1.0
    # the smallest minimum with a large spacing does not win alone
    u = oracle.local_solve_aniso(0, 2.5, inf, 3, 0.1, 1, 1)
    assert 2.5 < u < 3.0
    assert abs((u / 3) ** 2 + ((u - 2.5) / 0.1) ** 2 - 1) < 1e-12


def test_aniso_local_solve_satisfies_eq6_and_bounds():
    rng = np.random.default_rng(17)
    for _ in range(3000):
        a = rng.uniform(0, 2, 3)
        if rng.random() < 0.3:
            a[rng.integers(0, 3)] = np.inf
        h = rng.uniform(0.05, 3.0, 3)
        F = rng.uniform(0.1, 10.0)
        u = oracle.local_solve_aniso(*a, *h, F)
        t = np.maximum(u - a, 0.0) / h
        assert abs(np.sum(t * t) * F * F - 1.0) < 1e-11
        # upper bound: the best one-sided root; lower bound: the smallest minimum
        assert u <= np.min(a + h / F) * (1 + 1e-14) and u > np.min(a)


def test_aniso_local_solve_reduces_to_isotropic_and_scales():
    rng = np.random.default_rng(23)
    for _ in range(2000):
        a = rng.uniform(0, 2, 3)
        h = rng.uniform(0.05, 2.0)
        F = rng.uniform(0.1, 10.0)
        iso = oracle.local_solve(*a, h / F)
        assert abs(oracle.local_solve_aniso(*a, h, h, h, F) - iso) <= 1e-14 * max(1.0, iso)
        hs = rng.uniform(0.05, 2.0, 3)
        c = rng.uniform(0.1, 10.0)
        u = oracle.local_solve_aniso(*a, *hs, F)
        assert abs(oracle.local_solve_aniso(*(c * a), *(c * hs), F) - c * u) <= 1e-13 * max(1.0, c * u)


@pytest.mark.parametrize("seed", range(24))
def test_aniso_fmm_equals_gauss_seidel(seed):
    inst = W.random_small(500 + seed, max_edge=11, p_barrier=0.08 if seed % 3 == 0 else 0.0)
    rng = np.random.default_rng(seed)
    hs = tuple(rng.uniform(0.05, 2.0, 3))
    phi = oracle.fmm(inst.F, hs, inst.src_idx, inst.src_val)
    gs, _ = oracle.gs(inst.F, hs, inst.src_idx, inst.src_val)
    fin = np.isfinite(phi)
    assert np.array_equal(fin, np.isfinite(gs))
    scale = max(1.0, float(np.max(np.abs(phi[fin]))) if fin.any() else 1.0)
    assert np.max(np.abs(phi[fin] - gs[fin]), initial=0) <= 1e-13 * scale
    assert oracle.residual(inst.F, hs, inst.src_idx, phi) <= 1e-11


def test_aniso_axis_exactness_and_isotropic_case():
    F = np.ones((9, 11, 13))
    hs = (0.3, 0.7, 1.9)
    phi = oracle.fmm(F, hs, [0])
    k = np.arange(13)
    assert np.allclose(phi[0, 0, :], k * hs[0], rtol=1e-15, atol=0)
    assert np.allclose(phi[0, :, 0], np.arange(11) * hs[1], rtol=1e-15, atol=0)
    assert np.allclose(phi[:, 0, 0], np.arange(9) * hs[2], rtol=1e-15, atol=0)
    inst = W.random_small(77, dims=(7, 6, 5), three_d=True)
    assert np.array_equal(oracle.fmm(inst.F, (inst.h,) * 3, inst.src_idx, inst.src_val),
                          oracle.fmm(inst.F, inst.h, inst.src_idx, inst.src_val))


def test_aniso_refinement_toward_euclidean_distance():
    """A disc source of radius 0.25 on [0, 1] x [0, 2] with dy = 2 dx: the error
    against the distance to the circle falls by about 2 per halving."""
    errs = []
    for n in (33, 65, 129):
        hx, hy = 1.0 / (n - 1), 2.0 / (n - 1)
        x = np.arange(n) * hx
        y = np.arange(n) * hy
        X, Y = np.meshgrid(x, y)
        d = np.hypot(X - 0.5, Y - 1.0) - 0.25
        near = d <= max(hx, hy)
        idx = np.flatnonzero(near.reshape(-1))
        val = np.maximum(d.reshape(-1)[idx], 0.0)
        phi = oracle.fmm(np.ones((n, n)), (hx, hy), idx, val)
        errs.append(float(np.max(np.abs(phi - np.maximum(d, 0.0)))))
    assert 1.6 < errs[0] / errs[1] < 2.6 and 1.6 < errs[1] / errs[2] < 2.6, errs


# ---------------------------------------------------------------- shortest-path back-trace (Example 4)
def test_backtrace_axis_and_diagonal_paths():
    """F = 1, source at the corner: descent from an axis node runs along the
    axis, from a diagonal node along the diagonal (the steepest discrete slope)."""
    phi2 = oracle.fmm(np.ones((24, 24)), 1.0, [0])
    for k in range(1, 24):
        assert list(oracle.backtrace(phi2, 1.0, [k])[0]) == list(range(k, -1, -1))
        assert list(oracle.backtrace(phi2, 1.0, [k * 24])[0]) == [m * 24 for m in range(k, -1, -1)]
        assert list(oracle.backtrace(phi2, 1.0, [k * 25])[0]) == [m * 25 for m in range(k, -1, -1)]
    phi3 = oracle.fmm(np.ones((12, 12, 12)), 0.5, [0])
    for k in range(1, 12):
        diag = k * (1 + 12 + 144)
        assert list(oracle.backtrace(phi3, 0.5, [diag])[0]) == [m * 157 for m in range(k, -1, -1)]


@pytest.mark.parametrize("seed", range(12))
def test_backtrace_paths_descend_to_a_source(seed):
    inst = W.random_small(700 + seed, max_edge=14, p_barrier=0.1 if seed % 2 else 0.0)
    phi = oracle.fmm(inst.F, inst.h, inst.src_idx, inst.src_val)
    nx, ny, nz = inst.dims
    rng = np.random.default_rng(seed)
    starts = rng.integers(0, phi.size, size=20)
    flat = phi.reshape(-1)
    src = set(int(s) for s in inst.src_idx)
    for st, path in zip(starts, oracle.backtrace(phi, inst.h, starts)):
        if not np.isfinite(flat[st]):
            assert path.size == 0
            continue
        assert path[0] == st and int(path[-1]) in src
        assert np.all(np.diff(flat[path]) < 0)                          # strictly descending
        i, j, k = path % nx, (path // nx) % ny, path // (nx * ny)
        steps = np.stack([np.diff(i), np.diff(j), np.diff(k)])
        assert np.all(np.abs(steps) <= 1) and np.all(np.abs(steps).sum(0) >= 1)   # 26-neighbours


def test_backtrace_length_close_to_the_straight_segment():
    """F = 1: the path is at least as long as the straight segment to the source
    and, made of 26-neighbour steps, at most 20 % longer."""
    n = 40
    phi = oracle.fmm(np.ones((n, n, n)), 1.0, [0])
    rng = np.random.default_rng(3)
    starts = rng.integers(0, n ** 3, size=40)
    for st, path in zip(starts, oracle.backtrace(phi, 1.0, starts)):
        p = np.stack([path % n, (path // n) % n, path // (n * n)], 1).astype(float)
        L = np.sum(np.linalg.norm(np.diff(p, axis=0), axis=1))
        assert np.linalg.norm(p[0]) - 1e-12 <= L <= 1.2 * np.linalg.norm(p[0]) + 1e-12


# ---------------------------------------------------------------- residual checker (eq. 6), hand-worked values
def _residual_case(case):
    """phi map, speeds, spacing and sources of a case of tests/golden/residual.txt."""
    if case == "R1":
        phi = np.array([0.0, 1.0, 2.25, 3.0, 4.0]).reshape(1, 1, 5)
        return phi, np.ones_like(phi), 1.0, [0]
    if case == "R2":
        phi = np.array([[0.0, 1.0, 2.0], [1.0, 1.5, 5.0]])
        F = np.ones_like(phi)
        F[1, 1] = 2.0
        return phi, F, 1.0, [0]
    if case == "R3":
        phi = np.full((3, 3, 3), 10.0)
        phi[1, 1, 1] = 2.0
        phi[1, 1, 0], phi[1, 1, 2], phi[1, 0, 1], phi[0, 1, 1] = 1.0, 3.0, 1.25, 1.5
        return phi, np.ones_like(phi), 0.5, [0]
    raise KeyError(case)


def _golden_text_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


def test_residual_golden_hand_worked_values():
    """eko_residual reports the eq.-(6) residual worked out by hand at every listed node
    (tests/golden/residual.txt): a raised node on an exact 1D solution and its downstream
    neighbour, a 2D map where the (.)^+ clamp drops upwind terms, a 3D node with three
    upwind neighbours.  A residual that always returned 0, dropped the clamp, read a
    transposed neighbour or ignored F fails one of them."""
    rows = _golden_text_rows("residual.txt")
    assert len(rows) >= 11
    seen = set()
    for case, nx, ny, nz, h, i, j, k, want in rows:
        phi, F, hh, src = _residual_case(case)
        assert phi.size == int(nx) * int(ny) * int(nz) and hh == float(h)
        worst, res = oracle.residual(F, hh, src, phi, per_node=True)
        flat = (int(k) * int(ny) + int(j)) * int(nx) + int(i)
        assert res.reshape(-1)[flat] == float(want), (case, i, j, k, res.reshape(-1)[flat])
        assert worst >= float(want)
        seen.add(case)
    assert seen == {"R1", "R2", "R3"}
    # the maximum over the 1D line is the raised node
    phi, F, hh, src = _residual_case("R1")
    assert oracle.residual(F, hh, src, phi) == 0.5625


def test_residual_single_defect_on_a_solution():
    """On an FMM solution the residual is zero to rounding; raising one interior node by
    delta makes exactly that node and the neighbours it feeds report nonzero residuals."""
    inst = W.oscillating_3d(20)
    phi = oracle.fmm(inst.F, inst.h, inst.src_idx, inst.src_val)
    base, res0 = oracle.residual(inst.F, inst.h, inst.src_idx, phi, per_node=True)
    assert base < 1e-12
    p = (10 * 20 + 9) * 20 + 11
    bad = phi.copy().reshape(-1)
    bad[p] += 0.25 * inst.h
    worst, res = oracle.residual(inst.F, inst.h, inst.src_idx, bad.reshape(phi.shape), per_node=True)
    res = res.reshape(-1)
    changed = set(np.flatnonzero(res > 1e-9).tolist())
    nbrs = {p - 1, p + 1, p - 20, p + 20, p - 400, p + 400}
    assert p in changed and changed <= nbrs | {p}
    # at p itself: sum_d ((u + d - a_d)^+)^2 with the same minima, divided by tau^2
    tau = inst.h / inst.F.reshape(-1)[p]
    u = bad[p]
    a = []
    for lo, hi in ((p - 1, p + 1), (p - 20, p + 20), (p - 400, p + 400)):
        a.append(min(bad[lo], bad[hi]))
    want = abs(sum(max(u - v, 0.0) ** 2 for v in a) - tau * tau) / (tau * tau)
    assert res[p] == pytest.approx(want, rel=1e-12)
    assert worst == pytest.approx(max(res), rel=0)


def test_residual_impassable_sources_and_unreachable():
    """A finite value on an impassable node (F = 0) is an infinite residual; sources and
    +inf (unreachable) nodes are not checked."""
    phi = np.array([0.0, 1.0, 2.0, np.inf]).reshape(1, 1, 4)
    F = np.array([1.0, 1.0, 0.0, 0.0]).reshape(1, 1, 4)
    worst, res = oracle.residual(F, 1.0, [0], phi, per_node=True)
    assert math.isinf(res.reshape(-1)[2]) and math.isinf(worst)
    assert res.reshape(-1)[3] == 0.0 and res.reshape(-1)[1] == 0.0
    # a source holding any value is exempt
    phi2 = np.array([5.0, 1.0]).reshape(1, 1, 2)
    assert oracle.residual(np.ones((1, 1, 2)), 1.0, [0, 1], phi2) == 0.0


def test_backtrace_ties_go_to_the_lower_flat_index():
    """Equal slopes to two lower neighbours: the oracle's path takes the lower flat index
    (tests/golden/backtrace_ties.txt; the rule of Example 4's descent as read here)."""
    rows = _golden_text_rows("backtrace_ties.txt")
    assert len(rows) == 3
    for row in rows:
        case, start = row[0], int(row[1])
        rest = row[2:]
        path = [int(v) for v in rest if ":" not in v]
        phi = np.full(9, 10.0)
        for pair in (v for v in rest if ":" in v):
            n, val = pair.split(":")
            phi[int(n)] = float(val)
        got = oracle.backtrace(phi.reshape(3, 3), 1.0, [start])[0]
        assert got.tolist() == path, (case, got)
