"""FP64 CPU oracle for the first-order Godunov upwind Eikonal discretisation.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this package.  It
shares no code with the CUDA path (``paper_2106_15869_b300``): the two are
independent implementations that meet only in the test-suite.

The arithmetic lives in ``eik_oracle.c`` (plain C, FP64); this module only
compiles it (``gcc``), loads it with ``ctypes`` and marshals numpy arrays.
ctypes releases the GIL during a call, so several solves can run in parallel
from a thread pool.

Functions (each cites the passage it follows in its docstring):
  local_solve  exact root of eq. (6) from per-axis upwind minima
  local_solve_aniso  the same with unequal spacings (Alg 1.2, corrected thresholds)
  fmm          fast marching (Sec. 2.1): the discrete solution
  gs           Gauss-Seidel sweeping (Sec. 2.2) to an exact fixed point
  ifim         Algorithm 2 (Steps 1-3) point by point
  fim          the fast iterative method of Sec. 2.3 point by point
  residual     relative residual of eq. (6)
  backtrace    shortest-path back-trace by steepest descent on phi (Example 4)
  adjoint      d(loss)/d(slowness) by back substitution on the upwind
               linearisation of eq. (6) (adjoint-state method; not in the paper)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "eik_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libeik_oracle.so")
_lib = None

_d = ctypes.c_double
_i64 = ctypes.c_int64
_pd = ctypes.POINTER(ctypes.c_double)
_pi64 = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile eik_oracle.c into _build/libeik_oracle.so (gcc -O2, FP64, no fast-math)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
             "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.eko_local_solve.restype = _d
        lib.eko_local_solve.argtypes = [_d, _d, _d, _d]
        lib.eko_fmm.restype = _i64
        lib.eko_fmm.argtypes = [_i64, _i64, _i64, _d, _pd, _i64, _pi64, _pd, _pd, _pi64]
        lib.eko_gs.restype = _i64
        lib.eko_gs.argtypes = [_i64, _i64, _i64, _d, _pd, _i64, _pi64, _pd, _pd, _i64]
        lib.eko_ifim.restype = ctypes.c_int
        lib.eko_ifim.argtypes = [_i64, _i64, _i64, _d, _pd, _i64, _pi64, _pd, _pd,
                                 ctypes.c_int, _i64, _pi64]
        lib.eko_fim.restype = ctypes.c_int
        lib.eko_fim.argtypes = [_i64, _i64, _i64, _d, _pd, _i64, _pi64, _pd, _pd, _i64, _pi64]
        lib.eko_residual.restype = _d
        lib.eko_residual.argtypes = [_i64, _i64, _i64, _d, _pd, _i64, _pi64, _pd, _pd]
        lib.eko_local_solve_aniso.restype = _d
        lib.eko_local_solve_aniso.argtypes = [_d, _d, _d, _d, _d, _d, _d]
        lib.eko_fmm_aniso.restype = _i64
        lib.eko_fmm_aniso.argtypes = [_i64, _i64, _i64, _d, _d, _d, _pd, _i64, _pi64, _pd, _pd, _pi64]
        lib.eko_gs_aniso.restype = _i64
        lib.eko_gs_aniso.argtypes = [_i64, _i64, _i64, _d, _d, _d, _pd, _i64, _pi64, _pd, _pd, _i64]
        lib.eko_residual_aniso.restype = _d
        lib.eko_residual_aniso.argtypes = [_i64, _i64, _i64, _d, _d, _d, _pd, _i64, _pi64, _pd, _pd]
        lib.eko_backtrace.restype = ctypes.c_int
        lib.eko_backtrace.argtypes = [_i64, _i64, _i64, _d, _d, _d, _pd, _i64, _pi64, _i64, _pi64, _pi64]
        lib.eko_adjoint.restype = ctypes.c_int
        lib.eko_adjoint.argtypes = [_i64, _i64, _i64, _d, _pd, _i64, _pi64, _pd, _pd, _pd, _pd]
        _lib = lib
    return _lib


def _dims(F: np.ndarray):
    if F.ndim == 2:
        return F.shape[1], F.shape[0], 1
    if F.ndim == 3:
        return F.shape[2], F.shape[1], F.shape[0]
    raise ValueError("F must be 2D (ny, nx) or 3D (nz, ny, nx)")


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _src(src_idx, src_val):
    idx = np.ascontiguousarray(np.asarray(src_idx, dtype=np.int64).reshape(-1))
    if src_val is None:
        val = np.zeros(idx.shape, dtype=np.float64)
    else:
        val = _f64(np.asarray(src_val, dtype=np.float64).reshape(-1))
    if val.shape != idx.shape:
        raise ValueError("src_val must match src_idx")
    return idx, val


def _spacing(h):
    """h as a number (isotropic) or per axis (hx, hy[, hz]); returns (hx, hy, hz) or None."""
    if np.ndim(h) == 0:
        return None
    hs = [float(v) for v in h]
    if len(hs) == 2:
        hs.append(hs[0])           # 2D: no z neighbours, hz unused
    if len(hs) != 3:
        raise ValueError("h must be a number or (hx, hy[, hz])")
    return tuple(hs)


def _p(a, t=_pd):
    return a.ctypes.data_as(t)


def local_solve(ax: float, ay: float, az: float, tau: float) -> float:
    """Exact root of eq. (6) (Alg 1.1 / Alg 1.3 with the validity thresholds)."""
    return _load().eko_local_solve(float(ax), float(ay), float(az), float(tau))


def local_solve_aniso(ax: float, ay: float, az: float, hx: float, hy: float, hz: float, F: float) -> float:
    """Exact root of eq. (6) with spacings hx, hy, hz (Alg 1.2 with the validity thresholds)."""
    return _load().eko_local_solve_aniso(float(ax), float(ay), float(az), float(hx), float(hy), float(hz), float(F))


def fmm(F, h: float, src_idx, src_val=None, return_order: bool = False):
    """Fast marching (Sec. 2.1): the solution of eq. (4)/(6) with Dirichlet sources.

    h: the spacing, or (hx, hy[, hz]) for unequal spacings (eq. 5/6 with dx, dy, dz).

    F: (ny, nx) or (nz, ny, nx) speeds (F == 0 impassable); src_idx: flat
    indices; src_val: values (default 0).  Returns phi (+inf where
    unreachable) and, optionally, the acceptance order.
    """
    F = _f64(F)
    nx, ny, nz = _dims(F)
    idx, val = _src(src_idx, src_val)
    phi = np.empty(F.shape, dtype=np.float64)
    order = np.empty(F.size, dtype=np.int64) if return_order else None
    hs = _spacing(h)
    if hs is None:
        n = _load().eko_fmm(nx, ny, nz, float(h), _p(F), idx.size, _p(idx, _pi64), _p(val),
                            _p(phi), _p(order, _pi64) if order is not None else None)
    else:
        n = _load().eko_fmm_aniso(nx, ny, nz, *hs, _p(F), idx.size, _p(idx, _pi64), _p(val),
                                  _p(phi), _p(order, _pi64) if order is not None else None)
    if n < 0:
        raise ValueError("oracle fmm: invalid arguments")
    if return_order:
        return phi, order[:n]
    return phi


def gs(F, h: float, src_idx, src_val=None, max_rounds: int = 100000):
    """Gauss-Seidel with 2^d alternating sweep orders (Sec. 2.2) to an exact fixed point.

    Returns (phi, rounds).  Meant for tiny grids only.
    """
    F = _f64(F)
    nx, ny, nz = _dims(F)
    idx, val = _src(src_idx, src_val)
    phi = np.empty(F.shape, dtype=np.float64)
    hs = _spacing(h)
    if hs is None:
        r = _load().eko_gs(nx, ny, nz, float(h), _p(F), idx.size, _p(idx, _pi64), _p(val),
                           _p(phi), int(max_rounds))
    else:
        r = _load().eko_gs_aniso(nx, ny, nz, *hs, _p(F), idx.size, _p(idx, _pi64), _p(val),
                                 _p(phi), int(max_rounds))
    if r == -1:
        raise ValueError("oracle gs: invalid arguments")
    if r == -2:
        raise RuntimeError("oracle gs: max_rounds reached")
    return phi, int(r)


def ifim(F, h: float, src_idx, src_val=None, skip_remedy: bool = False,
         max_iters: int = 10**9):
    """Algorithm 2 (Steps 1-3), point by point, two-phase parallel semantics (Sec. 3.2).

    Returns (phi, stats) with stats = dict(update_iters, remedy_iters,
    remedy_seed, remedy_updates).
    """
    F = _f64(F)
    nx, ny, nz = _dims(F)
    idx, val = _src(src_idx, src_val)
    phi = np.empty(F.shape, dtype=np.float64)
    st = np.zeros(4, dtype=np.int64)
    rc = _load().eko_ifim(nx, ny, nz, float(h), _p(F), idx.size, _p(idx, _pi64), _p(val),
                          _p(phi), int(bool(skip_remedy)), int(max_iters), _p(st, _pi64))
    if rc == -1:
        raise ValueError("oracle ifim: invalid arguments")
    if rc == -2:
        raise RuntimeError("oracle ifim: max_iters reached")
    return phi, dict(update_iters=int(st[0]), remedy_iters=int(st[1]),
                     remedy_seed=int(st[2]), remedy_updates=int(st[3]))


def fim(F, h: float, src_idx, src_val=None, max_iters: int = 10**9):
    """The fast iterative method of Sec. 2.3 (neighbour convergence check), point by point.

    Returns (phi, stats) with stats = dict(iters, listed_by_check).
    """
    F = _f64(F)
    nx, ny, nz = _dims(F)
    idx, val = _src(src_idx, src_val)
    phi = np.empty(F.shape, dtype=np.float64)
    st = np.zeros(2, dtype=np.int64)
    rc = _load().eko_fim(nx, ny, nz, float(h), _p(F), idx.size, _p(idx, _pi64), _p(val),
                         _p(phi), int(max_iters), _p(st, _pi64))
    if rc == -1:
        raise ValueError("oracle fim: invalid arguments")
    if rc == -2:
        raise RuntimeError("oracle fim: max_iters reached")
    return phi, dict(iters=int(st[0]), listed_by_check=int(st[1]))


def residual(F, h: float, src_idx, phi, per_node: bool = False):
    """max_p |sum_d ((phi_p - a_d)^+)^2 - tau_p^2| / tau_p^2 over non-source finite nodes (eq. 6).

    With h = (hx, hy[, hz]): |sum_d ((phi_p - a_d)^+ / h_d)^2 - 1/F_p^2| * F_p^2.
    """
    F = _f64(F)
    nx, ny, nz = _dims(F)
    idx = np.ascontiguousarray(np.asarray(src_idx, dtype=np.int64).reshape(-1))
    phi = _f64(phi)
    res = np.empty(F.shape, dtype=np.float64) if per_node else None
    hs = _spacing(h)
    if hs is None:
        m = _load().eko_residual(nx, ny, nz, float(h), _p(F), idx.size, _p(idx, _pi64), _p(phi),
                                 _p(res) if res is not None else None)
    else:
        m = _load().eko_residual_aniso(nx, ny, nz, *hs, _p(F), idx.size, _p(idx, _pi64), _p(phi),
                                       _p(res) if res is not None else None)
    return (m, res) if per_node else m


def backtrace(phi, h, start_idx, max_len: int = 100000):
    """Shortest paths by steepest descent on the phi map (Example 4, Sec. 4.1).

    phi: (ny, nx) or (nz, ny, nx) arrival times (any float dtype; compared in
    float64); h: spacing or (hx, hy[, hz]); start_idx: flat start nodes.
    Returns a list of int64 arrays of flat node ids, start first.
    """
    phi = _f64(phi)
    nx, ny, nz = _dims(phi)
    hs = _spacing(h) or (float(h),) * 3
    st = np.ascontiguousarray(np.asarray(start_idx, dtype=np.int64).reshape(-1))
    out = np.empty((st.size, int(max_len)), dtype=np.int64)
    ln = np.empty(st.size, dtype=np.int64)
    rc = _load().eko_backtrace(nx, ny, nz, *hs, _p(phi), st.size, _p(st, _pi64), int(max_len),
                               _p(out, _pi64), _p(ln, _pi64))
    if rc != 0:
        raise ValueError("oracle backtrace: invalid arguments")
    return [out[q, :ln[q]].copy() for q in range(st.size)]


def adjoint(F, h: float, src_idx, phi, r, return_lambda: bool = False):
    """dL/ds for slowness s = 1/F, given phi and r = dL/dphi (adjoint of eq. 6).

    Back substitution of J^T lambda = r in decreasing-phi order, then
    dL/ds_i = 2 h^2 s_i lambda_i (0 at sources, impassable and unreachable nodes).
    """
    F = _f64(F)
    nx, ny, nz = _dims(F)
    idx = np.ascontiguousarray(np.asarray(src_idx, dtype=np.int64).reshape(-1))
    phi = _f64(phi)
    r = _f64(r)
    if phi.shape != F.shape or r.shape != F.shape:
        raise ValueError("phi and r must match F")
    g = np.empty(F.shape, dtype=np.float64)
    lam = np.empty(F.shape, dtype=np.float64) if return_lambda else None
    rc = _load().eko_adjoint(nx, ny, nz, float(h), _p(F), idx.size, _p(idx, _pi64), _p(phi),
                             _p(r), _p(g), _p(lam) if lam is not None else None)
    if rc != 0:
        raise ValueError("oracle adjoint: invalid arguments")
    return (g, lam) if return_lambda else g
