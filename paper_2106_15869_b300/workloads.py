"""Seeded synthetic inputs shaped like the workloads of the improved FIM.

This module holds input generation only -- speed maps, source sets and
receiver sets -- and none of the solver's arithmetic.  It imports nothing
from the CUDA path or from the oracle, and both of them (and the tests and
the benchmark) take their inputs from here.  Every generator is seeded with
``numpy.random.Generator(PCG64(seed))`` and returns float64 arrays; callers
cast to the dtype they solve in.

Workloads (grids are (nz, ny, nx), x fastest; 2D grids are (ny, nx)):
  point_source_2d   uniform 2D grid, F = 1, one point source (the constant
                    speed case of Example 1, Sec. 4.1, with a point source)
  oscillating_3d    3D grid, F = 1 + 0.5 sin(8 pi x) sin(8 pi y) sin(8 pi z),
                    corner source (smooth variable speed, like Example 5)
  maze_3d           3D maze of slow axis-aligned slabs with square gaps
                    (a synthetic stand-in for the barrier map of Example 4)
  lognormal_batch   many 3D instances of uneven size, F = exp(0.3 g) with g a
                    smoothed Gaussian random field, one source each
  tomography_3d     3D slowness with Gaussian blobs, sources on the top face
                    and receivers on the bottom face (adjoint workload)
  random_small      tiny random grids for exhaustive cross-checks
  paper_example_2d  the 2D Examples 1, 2, 3 and 5 of Sec. 4.1 on [-10, 10]^2
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class Instance:
    """One Eikonal problem: speed F, spacing h, Dirichlet sources (flat index, value)."""
    name: str
    F: np.ndarray                 # (ny, nx) or (nz, ny, nx), float64, F >= 0
    h: float
    src_idx: np.ndarray           # int64 flat indices
    src_val: np.ndarray           # float64 fixed values
    receivers: np.ndarray | None = None   # int64 flat indices (tomography)
    extra: dict = field(default_factory=dict)

    @property
    def dims(self):
        """(nx, ny, nz)."""
        if self.F.ndim == 2:
            return self.F.shape[1], self.F.shape[0], 1
        return self.F.shape[2], self.F.shape[1], self.F.shape[0]

    @property
    def n_nodes(self) -> int:
        return int(self.F.size)


def flat_index(dims, i, j, k=0):
    nx, ny, _ = dims
    return (np.asarray(k, dtype=np.int64) * ny + j) * nx + i


def point_source_2d(n: int = 128, src=(64, 64)) -> Instance:
    """n x n grid, h = 1/(n-1), F = 1, source phi = 0 at node (i, j) = src."""
    F = np.ones((n, n), dtype=np.float64)
    idx = np.array([src[1] * n + src[0]], dtype=np.int64)
    return Instance(f"point_source_2d_{n}", F, 1.0 / (n - 1), idx, np.zeros(1))


def oscillating_3d(n: int = 256, src=(0, 0, 0)) -> Instance:
    """n^3 grid, h = 1/(n-1), x = i h, F = 1 + 0.5 sin(8 pi x) sin(8 pi y) sin(8 pi z)."""
    h = 1.0 / (n - 1)
    s = np.sin(8.0 * np.pi * h * np.arange(n))
    F = 1.0 + 0.5 * s[:, None, None] * s[None, :, None] * s[None, None, :]
    i, j, k = src
    idx = np.array([(k * n + j) * n + i], dtype=np.int64)
    return Instance(f"oscillating_3d_{n}", np.ascontiguousarray(F), h, idx, np.zeros(1))


def maze_3d(n: int = 512, seed: int = 3, n_slabs: int = 16, thick: int = 4, gap: int = 32,
            n_src: int = 4, f_wall: float = 1e-3) -> Instance:
    """n^3 maze: per axis, n_slabs slabs `thick` cells thick at seeded positions,
    each holed by one seeded gap x gap square; F = f_wall in walls, 1 elsewhere;
    n_src sources uniform over free cells.  h = 1/(n-1).
    """
    rng = _rng(seed)
    gap = min(gap, n)
    wall = np.zeros((n, n, n), dtype=bool)
    for axis in range(3):          # grid axis 0 = x, 1 = y, 2 = z; array axis = 2 - axis
        starts = rng.integers(0, n - thick + 1, size=n_slabs)
        other = [a for a in range(3) if a != axis]
        for s0 in starts:
            g = rng.integers(0, n - gap + 1, size=2)
            m = np.zeros((n, n, n), dtype=bool)
            sl = [slice(None)] * 3
            sl[2 - axis] = slice(int(s0), int(s0) + thick)
            m[tuple(sl)] = True
            # one square gap in the slab plane (spanned by the two other axes)
            gs = list(sl)
            gs[2 - other[0]] = slice(int(g[0]), int(g[0]) + gap)
            gs[2 - other[1]] = slice(int(g[1]), int(g[1]) + gap)
            m[tuple(gs)] = False
            wall |= m     # where slabs cross, any slab's wall wins (a gap may be blocked)
    F = np.where(wall, f_wall, 1.0)
    free = np.flatnonzero(~wall.reshape(-1))
    idx = np.sort(rng.choice(free, size=n_src, replace=False)).astype(np.int64)
    return Instance(f"maze_3d_{n}", F, 1.0 / (n - 1), idx, np.zeros(n_src))


def _smooth_field(shape, sigma: float, rng: np.random.Generator) -> np.ndarray:
    from scipy.ndimage import gaussian_filter
    g = rng.standard_normal(shape)
    g = gaussian_filter(g, sigma=sigma, mode="reflect", truncate=3.0)
    g -= g.mean()
    sd = g.std()
    return g / sd if sd > 0 else g


def lognormal_batch(B: int = 64, seed: int = 4, lo: int = 64, hi: int = 192,
                    sigma: float = 8.0, amp: float = 0.3, h: float = 1.0 / 127) -> list[Instance]:
    """B 3D instances, each edge uniform in [lo, hi]; F = exp(amp * g), g a
    Gaussian random field smoothed with a Gaussian kernel of std `sigma` cells
    and scaled to unit std; one source uniform over the grid.
    """
    rng = _rng(seed)
    dims = rng.integers(lo, hi + 1, size=(B, 3))
    subseeds = rng.integers(0, 2**62, size=B)
    out = []
    for b in range(B):
        nx, ny, nz = (int(v) for v in dims[b])
        r = _rng(int(subseeds[b]))
        g = _smooth_field((nz, ny, nx), sigma, r)
        F = np.exp(amp * g)
        idx = np.array([r.integers(0, nx * ny * nz)], dtype=np.int64)
        out.append(Instance(f"lognormal_{b}_{nx}x{ny}x{nz}", F, h, idx, np.zeros(1)))
    return out


def tomography_3d(n: int = 192, seed: int = 5, n_blobs: int = 8, amp: float = 0.2,
                  radius: float = 12.0, src_lattice=(24, 72, 120, 168),
                  rec_count: int = 16, rec_start: int = 6, rec_step: int = 12) -> dict:
    """Travel-time tomography set-up on an n^3 grid, h = 1/(n-1).

    True slowness s = 1 + amp * sum_b exp(-|x - c_b|^2 / (2 radius^2)) (cell
    units, blob centres uniform in [n/8, 7n/8]^3); initial slowness 1.
    Sources on the top face z = 0 on a lattice, receivers on the bottom face
    z = n-1 on a rec_count x rec_count lattice.  Returns a dict with
    s_true, s_init, h, sources (flat), receivers (flat).
    """
    rng = _rng(seed)
    c = rng.uniform(n / 8.0, 7.0 * n / 8.0, size=(n_blobs, 3))
    ax = np.arange(n, dtype=np.float64)
    s = np.ones((n, n, n), dtype=np.float64)
    for b in range(n_blobs):
        gx = np.exp(-(ax - c[b, 0]) ** 2 / (2 * radius**2))
        gy = np.exp(-(ax - c[b, 1]) ** 2 / (2 * radius**2))
        gz = np.exp(-(ax - c[b, 2]) ** 2 / (2 * radius**2))
        s += amp * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    lat = [v for v in src_lattice if v < n]
    sources = np.array([(0 * n + j) * n + i for j in lat for i in lat], dtype=np.int64)
    rl = [rec_start + rec_step * m for m in range(rec_count) if rec_start + rec_step * m < n]
    receivers = np.array([((n - 1) * n + j) * n + i for j in rl for i in rl], dtype=np.int64)
    return dict(s_true=s, s_init=np.ones_like(s), h=1.0 / (n - 1), sources=sources,
                receivers=receivers, n=n)


def random_small(seed: int, dims=None, max_edge: int = 16, three_d: bool | None = None,
                 f_lo: float = 0.1, f_hi: float = 10.0, max_src: int = 4,
                 p_barrier: float = 0.0) -> Instance:
    """Tiny random grid: random dims (<= max_edge), F uniform in [f_lo, f_hi],
    1..max_src sources with value 0 or a small random value, optional barrier
    cells (F = 0) with probability p_barrier.
    """
    rng = _rng(seed)
    if three_d is None:
        three_d = bool(rng.integers(0, 2))
    if dims is None:
        nx = int(rng.integers(1, max_edge + 1))
        ny = int(rng.integers(1, max_edge + 1))
        nz = int(rng.integers(1, max_edge + 1)) if three_d else 1
    else:
        nx, ny, nz = dims
    shape = (nz, ny, nx) if nz > 1 or three_d else (ny, nx)
    F = rng.uniform(f_lo, f_hi, size=shape)
    if p_barrier > 0:
        F[rng.random(shape) < p_barrier] = 0.0
    N = F.size
    ns = int(rng.integers(1, max_src + 1))
    idx = np.unique(rng.integers(0, N, size=ns)).astype(np.int64)
    val = np.where(rng.random(idx.size) < 0.5, 0.0, rng.uniform(0.0, 0.3, size=idx.size))
    return Instance(f"random_{seed}", F, float(rng.uniform(0.05, 2.0)), idx, val)


def _circle_sources(xs, ys, centers_radii, F):
    """Nodes within one cell of a circle boundary or inside it take the exact
    travel time from the circle: (|x - c| - R)^+ / F, the smallest over circles.
    """
    h = xs[1] - xs[0]
    X, Y = np.meshgrid(xs, ys)          # (ny, nx)
    best = np.full(X.shape, np.inf)
    for (cx, cy, R) in centers_radii:
        d = np.hypot(X - cx, Y - cy)
        near = d <= R + h
        t = np.where(near, np.maximum(d - R, 0.0), np.inf)
        best = np.minimum(best, t)
    sel = np.isfinite(best)
    with np.errstate(divide="ignore"):
        val = best[sel] / F[sel]
    idx = np.flatnonzero(sel.reshape(-1)).astype(np.int64)
    return idx, val.astype(np.float64)


def paper_example_2d(example: int, n: int = 200, lo: float = -10.0, hi: float = 10.0) -> Instance:
    """The 2D Examples of Sec. 4.1 on an n x n grid over [lo, hi]^2.

    1: circle R = 3 at the origin, F = 1
    2: circles R = 3 at (2, -5) and R = 1.5 at (-2, 5), F = 1
    3: circles R = 0.5 at (-5, 5) and (5, -5); F = 1 on [3, 7]^2, 0.01 elsewhere (eq. 7)
    5: circle R = 0.5 at the origin; F = sin^2 x + sin^2 y + 0.3 (eq. 9)
    Nodes inside or within one cell of a circle are sources carrying their
    exact distance to the circle divided by F.
    """
    xs = np.linspace(lo, hi, n)
    X, Y = np.meshgrid(xs, xs)
    if example == 1:
        F = np.ones((n, n)); circ = [(0.0, 0.0, 3.0)]
    elif example == 2:
        F = np.ones((n, n)); circ = [(2.0, -5.0, 3.0), (-2.0, 5.0, 1.5)]
    elif example == 3:
        F = np.where((X >= 3) & (X <= 7) & (Y >= 3) & (Y <= 7), 1.0, 0.01)
        circ = [(-5.0, 5.0, 0.5), (5.0, -5.0, 0.5)]
    elif example == 5:
        F = np.sin(X) ** 2 + np.sin(Y) ** 2 + 0.3
        circ = [(0.0, 0.0, 0.5)]
    else:
        raise ValueError("examples 1, 2, 3 and 5 are defined (Example 4's map is not available)")
    idx, val = _circle_sources(xs, xs, circ, F)
    return Instance(f"paper_ex{example}_{n}", np.ascontiguousarray(F), float(xs[1] - xs[0]), idx, val)
