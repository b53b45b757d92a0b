"""B300-native (sm_103a) Eikonal solver: the improved fast iterative method.

``||grad phi|| = 1/F`` on uniform 2D/3D grids by Algorithm 2 of the paper
(a tile active-list update without neighbour convergence checks, then a
remedy pass), in hand-written CUDA kernels behind the C ABI of
``libeikonal.so`` (include/eikonal.h).

Public API (loaded lazily, so that ``workloads`` imports without CUDA):
  solve, solve_batched, adjoint, adjoint_batched, EikonalFn, Workspace, EikonalError
"""
from __future__ import annotations

__all__ = ["solve", "solve_batched", "adjoint", "adjoint_batched", "EikonalFn", "Workspace", "EikonalError"]


def __getattr__(name):
    if name in ("solve", "solve_batched", "adjoint", "adjoint_batched", "EikonalFn", "Workspace"):
        from . import api
        return getattr(api, name)
    if name == "EikonalError":
        from ._lib import EikonalError
        return EikonalError
    raise AttributeError(name)
