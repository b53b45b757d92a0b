"""The fact behind the exact Step-3 listing test of the GPU path, checked on the
oracle's local solver (eq. 6, CPU, no GPU).

A visit lists the neighbour tile across a face only if a node p that dropped
to u lies below the node q across it.  The reason: let q hold phi(q) at or
below its root r(a_x, a_y, a_z) (a tile at its fixed point).  If p's new
value u is not below phi(q), then the minimum on p's axis stays at or above
min(a_old, phi(q)), and q's root stays at or above phi(q).  A lower u can take
the root below phi(q), so the test is not vacuous.
"""
import numpy as np
import pytest

import oracle


def _root(a, tau):
    return oracle.local_solve(a[0], a[1], a[2], tau)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_neighbour_not_below_cannot_lower_the_root(axis):
    rng = np.random.default_rng(100 + axis)
    below_lowered = 0
    for _ in range(4000):
        tau = rng.uniform(0.05, 2.0)
        a = rng.uniform(0.0, 3.0, size=3)
        if rng.random() < 0.2:
            a[rng.integers(3)] = np.inf          # a missing neighbour on one axis
        r0 = _root(a, tau)
        if not np.isfinite(r0):
            continue
        phi_q = r0 - rng.uniform(0.0, 1.0) * tau * (rng.random() < 0.5)   # at or below its root
        # the neighbour p on `axis` drops to u >= phi(q): the axis minimum becomes min(a, u)
        u = phi_q + rng.uniform(0.0, 2.0) * tau
        b = a.copy()
        b[axis] = min(a[axis], u)
        assert _root(b, tau) >= phi_q - 1e-12 * max(1.0, abs(phi_q))
        # the same neighbour dropping below phi(q) can lower the root under phi(q)
        c = a.copy()
        c[axis] = min(a[axis], phi_q - rng.uniform(0.01, 2.0) * tau)
        if _root(c, tau) < phi_q - 1e-12:
            below_lowered += 1
    assert below_lowered > 1000


def test_equal_spacing_fixed_point_of_a_grid_is_kept():
    """On a fast-marching solution (every reachable non-source node at its root),
    lowering one node p to any value not below a face neighbour q leaves q's
    root at or above phi(q); lowering it below can move q."""
    rng = np.random.default_rng(7)
    n = 12
    F = rng.uniform(0.5, 2.0, size=(n, n, n))
    h = 1.0 / (n - 1)
    phi = oracle.fmm(F, h, [0])
    P = np.pad(phi, 1, constant_values=np.inf)

    def root_at(P, k, j, i):
        ax = min(P[k + 1, j + 1, i], P[k + 1, j + 1, i + 2])
        ay = min(P[k + 1, j, i + 1], P[k + 1, j + 2, i + 1])
        az = min(P[k, j + 1, i + 1], P[k + 2, j + 1, i + 1])
        return oracle.local_solve(ax, ay, az, h / F[k, j, i])

    moved = 0
    for _ in range(400):
        k, j, i = rng.integers(1, n - 1, size=3)
        d = rng.integers(6)
        dk, dj, di = [(0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)][d]
        kp, jp, ip = k + dk, j + dj, i + di            # p, the face neighbour of q = (k, j, i)
        if (kp, jp, ip) == (0, 0, 0) or (k, j, i) == (0, 0, 0):
            continue
        Q = P.copy()
        Q[kp + 1, jp + 1, ip + 1] = min(phi[kp, jp, ip], phi[k, j, i] + rng.uniform(0.0, 1.0) * h)
        assert root_at(Q, k, j, i) >= phi[k, j, i] * (1 - 1e-12)
        Q[kp + 1, jp + 1, ip + 1] = phi[k, j, i] - rng.uniform(0.5, 2.0) * h
        if root_at(Q, k, j, i) < phi[k, j, i] * (1 - 1e-12):
            moved += 1
    assert moved > 100
