"""Python API over the C ABI: torch tensors in, torch tensors out.

torch supplies device memory (the caching allocator) and the current CUDA
stream; every step of the solve runs in libeikonal.so.  A CPU tensor given to
``solve`` is copied to the current CUDA device and the result copied back
(the end-to-end path); there is no CPU solver.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib

_DT = {torch.float32: "fp32", torch.float64: "fp64"}


def _stream_ptr(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _dims(F: torch.Tensor):
    if F.dim() == 2:
        return int(F.shape[1]), int(F.shape[0]), 1
    if F.dim() == 3:
        return int(F.shape[2]), int(F.shape[1]), int(F.shape[0])
    raise ValueError("F must be (ny, nx) or (nz, ny, nx)")


def _as_index(src_idx, device) -> torch.Tensor:
    t = torch.as_tensor(np.asarray(src_idx, dtype=np.int64).reshape(-1)) if not torch.is_tensor(src_idx) \
        else src_idx.reshape(-1).to(torch.int64)
    return t.to(device, non_blocking=True).contiguous()


def _as_values(src_val, n, dtype, device) -> torch.Tensor:
    if src_val is None:
        return torch.zeros(n, dtype=dtype, device=device)
    t = src_val if torch.is_tensor(src_val) else torch.as_tensor(np.asarray(src_val, dtype=np.float64))
    t = t.reshape(-1).to(device=device, dtype=dtype)
    if t.numel() != n:
        raise ValueError("src_val must have one value per source index")
    return t.contiguous()


class Workspace:
    """A reusable, growable device workspace (one per stream is the usual pattern)."""

    def __init__(self, device=None):
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.buf = None

    def get(self, nbytes: int) -> torch.Tensor:
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        return self.buf


_default_ws: dict = {}


def _workspace(device, nbytes, ws: Workspace | None):
    if ws is None:
        key = (device.index, torch.cuda.current_stream(device).cuda_stream)
        ws = _default_ws.get(key)
        if ws is None:
            ws = _default_ws[key] = Workspace(device)
    buf = ws.get(nbytes)
    if buf.data_ptr() % 256:
        raise RuntimeError("workspace is not 256-byte aligned")
    return buf


def solve(F: torch.Tensor, src_idx, h: float, src_val=None, *, tile="auto", schedule="auto",
          skip_remedy=False, max_iters=0, order=0.0, converge="auto", method="ifim", return_stats=False,
          workspace: Workspace | None = None, out: torch.Tensor | None = None, wait_limit_us: int = 0,
          remedy_order: float = 0.0):
    """Arrival times phi of ||grad phi|| = 1/F with fixed values at the sources.

    F: (ny, nx) or (nz, ny, nx) float32 (or float64 = FP64 validation mode)
    speeds, F == 0 impassable; src_idx: flat indices; src_val: values
    (default 0); h: grid spacing, or (hx, hy[, hz]) for unequal spacings
    (eq. 5/6 with dx, dy, dz).  Returns phi with F's shape, dtype and device
    (+inf where unreachable); with return_stats also a dict of run statistics
    (this synchronises the stream).  order: 0 = default (the Step-3 lists
    bucketed; the Step-2 lists bucketed on 2D grids, unordered on 3D grids),
    > 0 = both loops bucketed with this width in tile-crossing times, < 0 =
    unordered lists (every
    listed tile visited in every iteration, as Algorithm 2 is printed).
    remedy_order: the Step-3 list order alone where the Step-2 lists are
    unordered (0 = as `order` sets it, > 0 = this bucket width, < 0 =
    unordered); every order gives the same solution.
    wait_limit_us: bound on every device-side wait (0 = 2 s); a wait that runs
    out ends the launch with EIK_ERR_DEVICE and phi holding upper bounds.
    method: "ifim" (Algorithm 2: Step 2 without neighbour checks, then the
    remedy) or "fim" (the fast iterative method of Sec. 2.3 at tile
    granularity: neighbour tiles are re-listed when a visit lowers their
    facing boundary; no remedy).  Both give the same discrete solution.
    """
    if F.dtype not in _DT:
        raise TypeError("F must be float32 or float64")
    host = not F.is_cuda
    dev = torch.device("cuda", torch.cuda.current_device()) if host else F.device
    Fd = F.to(dev, non_blocking=True).contiguous() if host else F.contiguous()
    nx, ny, nz = _dims(Fd)
    idx = _as_index(src_idx, dev)
    val = _as_values(src_val, idx.numel(), Fd.dtype, dev)
    lib = _lib.load()
    g = _lib.grids_array([(nx, ny, nz, h)])
    opt = _lib.make_options(tile, schedule, _DT[Fd.dtype], skip_remedy, max_iters, order, converge, method,
                            wait_limit_us, remedy_order)
    nbytes = lib.eik_workspace_size(g, ctypes.byref(opt))
    if nbytes == 0:
        raise _lib.EikonalError(_lib.EIK_ERR_ARG, "invalid grid or options")
    with torch.cuda.device(dev):
        buf = _workspace(dev, nbytes, workspace)
        phi = out if out is not None else torch.empty_like(Fd)
        st = _lib.eik_stats()
        rc = lib.eik_solve(g, Fd.data_ptr(), idx.data_ptr() if idx.numel() else None,
                           val.data_ptr() if idx.numel() else None, idx.numel(), phi.data_ptr(),
                           buf.data_ptr(), buf.numel(), _stream_ptr(), ctypes.byref(opt),
                           ctypes.byref(st) if return_stats else None)
        _lib.check(rc)
    if host:
        phi = phi.to("cpu")
    return (phi, st.as_dict()) if return_stats else phi


def solve_batched(problems, *, tile="auto", schedule="auto", skip_remedy=False, max_iters=0, order=0.0,
                  converge="auto", method="ifim", return_stats=False, workspace: Workspace | None = None,
                  shared_F: bool = False, wait_limit_us: int = 0, remedy_order: float = 0.0):
    """Solve many independent grids in one set of launches.

    problems: list of (F, src_idx, h) or (F, src_idx, h, src_val); all F on the
    same CUDA device with the same dtype.  With shared_F=True every problem
    uses the first problem's F (one copy, read by all instances; e.g. many
    sources on one speed map).  Options as for solve().  Returns a list of phi
    tensors.
    """
    if not problems:
        return ([], {}) if return_stats else []
    F0 = problems[0][0]
    dev, dtype = F0.device, F0.dtype
    if dtype not in _DT or not F0.is_cuda:
        raise TypeError("F must be a float32/float64 CUDA tensor")
    dims, Fs, idxs, vals = [], [], [], []
    for p in problems:
        F, si, h = p[0], p[1], p[2]
        sv = p[3] if len(p) > 3 else None
        if shared_F:
            F = F0
        if F.device != dev or F.dtype != dtype:
            raise ValueError("all F must share device and dtype")
        nx, ny, nz = _dims(F)
        dims.append((nx, ny, nz, h))
        Fs.append(F)
        i = _as_index(si, dev)
        idxs.append(i)
        vals.append(_as_values(sv, i.numel(), dtype, dev))
    sizes = [d[0] * d[1] * d[2] for d in dims]
    phi_off = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    if shared_F:
        F_packed = F0.contiguous().reshape(-1)
        F_off = np.zeros(len(problems), dtype=np.int64)
    else:
        F_packed = torch.cat([F.contiguous().reshape(-1) for F in Fs])
        F_off = phi_off
    nsrc = [i.numel() for i in idxs]
    src_off = np.concatenate([[0], np.cumsum(nsrc)]).astype(np.int64)
    src_idx = torch.cat(idxs) if sum(nsrc) else torch.zeros(0, dtype=torch.int64, device=dev)
    src_val = torch.cat(vals) if sum(nsrc) else torch.zeros(0, dtype=dtype, device=dev)
    lib = _lib.load()
    g = _lib.grids_array(dims)
    opt = _lib.make_options(tile, schedule, _DT[dtype], skip_remedy, max_iters, order, converge, method,
                            wait_limit_us, remedy_order)
    B = len(problems)
    nbytes = lib.eik_workspace_size_batched(B, g, ctypes.byref(opt))
    if nbytes == 0:
        raise _lib.EikonalError(_lib.EIK_ERR_ARG, "invalid grids or options")
    with torch.cuda.device(dev):
        buf = _workspace(dev, nbytes, workspace)
        phi_packed = torch.empty(int(sum(sizes)), dtype=dtype, device=dev)
        st = _lib.eik_stats()
        rc = lib.eik_solve_batched(B, g, F_packed.data_ptr(), _lib.i64_array(F_off),
                                   src_idx.data_ptr() if src_idx.numel() else None,
                                   src_val.data_ptr() if src_idx.numel() else None,
                                   _lib.i64_array(src_off), phi_packed.data_ptr(), _lib.i64_array(phi_off),
                                   buf.data_ptr(), buf.numel(), _stream_ptr(), ctypes.byref(opt),
                                   ctypes.byref(st) if return_stats else None)
        _lib.check(rc)
    outs = []
    for q, F in enumerate(Fs):
        outs.append(phi_packed[phi_off[q]:phi_off[q] + sizes[q]].view(F.shape))
    return (outs, st.as_dict()) if return_stats else outs


def adjoint_batched(problems, phis, rs, *, shared_F: bool = False, sum_instances: bool = False, tile="auto",
                    max_iters=0, order=0.0, return_stats=False, workspace: Workspace | None = None,
                    wait_limit_us: int = 0):
    """Gradients dL/ds (s = 1/F) of a loss L(phi) by the adjoint of the discrete solve.

    problems: list of (F, src_idx, h) as for solve_batched (all on one CUDA
    device, one dtype); phis: the forward solutions (checkpoints); rs: dL/dphi
    per instance (same shapes).  With shared_F every instance uses the first
    F; with sum_instances the gradients of all instances are accumulated into
    one tensor shaped like the first F (e.g. many shots on one slowness model),
    summed in instance order, so that repeated calls are bit-identical.
    Returns a list of gradients, or one tensor with sum_instances.
    """
    if not problems:
        raise ValueError("no problems")
    F0 = problems[0][0]
    dev, dtype = F0.device, F0.dtype
    if dtype not in _DT or not F0.is_cuda:
        raise TypeError("F must be a float32/float64 CUDA tensor")
    if len(phis) != len(problems) or len(rs) != len(problems):
        raise ValueError("one phi and one r per problem")
    dims, Fs, idxs = [], [], []
    for pr in problems:
        F = F0 if shared_F else pr[0]
        if F.device != dev or F.dtype != dtype:
            raise ValueError("all F must share device and dtype")
        nx, ny, nz = _dims(F)
        dims.append((nx, ny, nz, pr[2]))
        Fs.append(F)
        idxs.append(_as_index(pr[1], dev))
    if sum_instances and any(d[:3] != dims[0][:3] for d in dims):
        raise ValueError("sum_instances needs equal grid shapes")
    sizes = [d[0] * d[1] * d[2] for d in dims]
    off = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    for q, (ph, r) in enumerate(zip(phis, rs)):
        if ph.numel() != sizes[q] or r.numel() != sizes[q]:
            raise ValueError("phi and r must match their grid")
    if shared_F:
        F_packed, F_off = F0.contiguous().reshape(-1), np.zeros(len(problems), dtype=np.int64)
    else:
        F_packed, F_off = torch.cat([F.contiguous().reshape(-1) for F in Fs]), off
    phi_packed = torch.cat([ph.to(dev, dtype).contiguous().reshape(-1) for ph in phis])
    r_packed = torch.cat([r.to(dev, dtype).contiguous().reshape(-1) for r in rs])
    if sum_instances:
        g_packed = torch.zeros(sizes[0], dtype=dtype, device=dev)
        g_off = np.zeros(len(problems), dtype=np.int64)
    else:
        g_packed = torch.zeros(int(sum(sizes)), dtype=dtype, device=dev)
        g_off = off
    nsrc = [i.numel() for i in idxs]
    src_off = np.concatenate([[0], np.cumsum(nsrc)]).astype(np.int64)
    src_idx = torch.cat(idxs) if sum(nsrc) else torch.zeros(0, dtype=torch.int64, device=dev)
    lib = _lib.load()
    g = _lib.grids_array(dims)
    opt = _lib.make_options(tile, "auto", _DT[dtype], False, max_iters, order, wait_limit_us=wait_limit_us)
    B = len(problems)
    nbytes = lib.eik_adjoint_workspace_size_batched(B, g, ctypes.byref(opt))
    if nbytes == 0:
        raise _lib.EikonalError(_lib.EIK_ERR_ARG, "invalid grids or options")
    with torch.cuda.device(dev):
        buf = _workspace(dev, nbytes, workspace)
        st = _lib.eik_stats()
        rc = lib.eik_adjoint_batched(B, g, F_packed.data_ptr(), _lib.i64_array(F_off), phi_packed.data_ptr(),
                                     _lib.i64_array(off), src_idx.data_ptr() if src_idx.numel() else None,
                                     _lib.i64_array(src_off), r_packed.data_ptr(), g_packed.data_ptr(),
                                     _lib.i64_array(g_off), buf.data_ptr(), buf.numel(), _stream_ptr(),
                                     ctypes.byref(opt), ctypes.byref(st) if return_stats else None)
        _lib.check(rc)
    if sum_instances:
        out = g_packed.view(F0.shape)
    else:
        out = [g_packed[off[q]:off[q] + sizes[q]].view(Fs[q].shape) for q in range(B)]
    return (out, st.as_dict()) if return_stats else out


def adjoint(F, src_idx, h, phi, r, **kw):
    """dL/ds for one grid (see adjoint_batched)."""
    return adjoint_batched([(F, src_idx, h)], [phi], [r], **kw)[0]


def backtrace(phi: torch.Tensor, start_idx, h, max_len: int = 65536):
    """Shortest paths from start nodes back to the source by steepest descent on
    the arrival-time map phi (Example 4, Sec. 4.1; the rule is in eik_backtrace's
    header comment).

    phi: (ny, nx) or (nz, ny, nx) CUDA tensor, float32 or float64 (e.g. solve's
    output); start_idx: flat start nodes; h: spacing or (hx, hy[, hz]).
    Returns (path, length): path int64 (n_paths, max_len) of flat node ids,
    start first, -1 past the end; length int64 (n_paths,) (0: unreachable start).
    """
    if phi.dtype not in _DT or not phi.is_cuda:
        raise TypeError("phi must be a float32/float64 CUDA tensor")
    phi = phi.contiguous()
    nx, ny, nz = _dims(phi)
    dev = phi.device
    st = _as_index(start_idx, dev)
    n = st.numel()
    path = torch.empty((n, int(max_len)), dtype=torch.int64, device=dev)
    length = torch.empty(n, dtype=torch.int64, device=dev)
    g = _lib.grids_array([(nx, ny, nz, h)])
    with torch.cuda.device(dev):
        rc = _lib.load().eik_backtrace(g, _lib.PRECISIONS[_DT[phi.dtype]], phi.data_ptr(),
                                       st.data_ptr() if n else None, n, int(max_len),
                                       path.data_ptr() if n else None, length.data_ptr() if n else None,
                                       _stream_ptr())
        _lib.check(rc)
    return path, length


class EikonalFn(torch.autograd.Function):
    """phi = EikonalFn.apply(s, sources, h): arrival times for slowness s = 1/F.

    s: (ny, nx) or (nz, ny, nx) CUDA tensor (float32, or float64 for the
    validation mode); sources: list of source-index arrays, one per shot;
    h: spacing.  Returns phi stacked over shots, shape (n_shots, *s.shape).
    The forward runs all shots as one batched solve on a shared speed map and
    checkpoints phi; backward runs the batched adjoint and sums the shots'
    gradients into dL/ds.
    """

    @staticmethod
    def forward(ctx, s, sources, h, tile="auto"):
        F = (1.0 / s).contiguous()
        phis = solve_batched([(F, src, h) for src in sources], shared_F=True, tile=tile)
        phi = torch.stack(phis)
        ctx.save_for_backward(F, phi)
        ctx.sources, ctx.h, ctx.tile = sources, h, tile
        return phi

    @staticmethod
    def backward(ctx, grad_phi):
        F, phi = ctx.saved_tensors
        rs = [grad_phi[q].contiguous() for q in range(grad_phi.shape[0])]
        g = adjoint_batched([(F, src, ctx.h) for src in ctx.sources], list(phi.unbind(0)), rs, shared_F=True,
                            sum_instances=True, tile=ctx.tile)
        return g, None, None, None


class Trace:
    """Context manager: per-iteration trace of the solves run inside it.

        with api.Trace() as tr:
            api.solve(...)
        tr.records   # numpy (n, 4): time ns, phase (+256: throughput mode), list size, tiles visited
    """

    def __init__(self, capacity: int = 1 << 16, device=None):
        self.capacity = int(capacity)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.buf = None
        self.records = None

    def __enter__(self):
        self.buf = torch.zeros(4 * self.capacity + 1, dtype=torch.int64, device=self.device)
        with torch.cuda.device(self.device):
            torch.cuda.synchronize()
            _lib.check(_lib.load().eik_set_trace(self.buf.data_ptr(), self.capacity))
        return self

    def __exit__(self, *exc):
        with torch.cuda.device(self.device):
            torch.cuda.synchronize()
            _lib.check(_lib.load().eik_set_trace(None, 0))
        b = self.buf.cpu().numpy()
        n = int(b[0])
        self.records = b[1:1 + 4 * n].reshape(n, 4).astype(np.int64)
        return False

    def summary(self) -> dict:
        """Time per phase and per-iteration statistics (microseconds)."""
        r = self.records
        if r is None or len(r) < 2:
            return {}
        dt = np.diff(r[:, 0]) / 1e3
        ph = r[1:, 1] & 0xff
        thr = (r[1:, 1] & 256) != 0
        out = {}
        for p, name in ((1, "update"), (2, "seed"), (3, "remedy"), (4, "fim")):
            m = ph == p
            if m.any():
                out[name] = dict(iterations=int(m.sum()), total_us=float(dt[m].sum()),
                                 median_us=float(np.median(dt[m])), mean_list=float(r[1:, 2][m].mean()),
                                 visited=int(r[1:, 3][m].sum()), throughput_iterations=int((m & thr).sum()))
        return out


class BatchedSolver:
    """A fixed batch of grids and sources whose solve is captured once in a CUDA
    graph and replayed (the batched form: all instances in one persistent
    launch, the launch sequence replayed without host work).

        bs = BatchedSolver([(F0, src0, h0), (F1, src1, h1), ...])
        bs.set_speeds(b, F_new)      # optional: overwrite instance b's speeds in place
        phis = bs.solve()            # replay; views into one packed output buffer

    Inputs are copied once into static device buffers; set_speeds / set_sources
    overwrite them between replays.  Every solve re-initialises all device
    state, so replays are independent.  With graph=False the same launches are
    issued directly (for comparison).
    """

    def __init__(self, problems, *, tile="auto", order=0.0, converge="auto", method="ifim", max_iters=0,
                 graph=True, schedule="persistent", remedy_order=0.0):
        F0 = problems[0][0]
        self.device, self.dtype = F0.device, F0.dtype
        if self.dtype not in _DT or not F0.is_cuda:
            raise TypeError("F must be a float32/float64 CUDA tensor")
        self.shapes, dims, idxs, vals = [], [], [], []
        for p in problems:
            F = p[0]
            nx, ny, nz = _dims(F)
            dims.append((nx, ny, nz, p[2]))
            self.shapes.append(F.shape)
            i = _as_index(p[1], self.device)
            idxs.append(i)
            vals.append(_as_values(p[3] if len(p) > 3 else None, i.numel(), self.dtype, self.device))
        self.sizes = [d[0] * d[1] * d[2] for d in dims]
        self.off = np.concatenate([[0], np.cumsum(self.sizes)[:-1]]).astype(np.int64)
        self.F = torch.cat([p[0].contiguous().reshape(-1).to(self.dtype) for p in problems])
        self.phi = torch.empty_like(self.F)
        self.nsrc = [i.numel() for i in idxs]
        self.src_off = np.concatenate([[0], np.cumsum(self.nsrc)]).astype(np.int64)
        self.src_idx = torch.cat(idxs) if sum(self.nsrc) else torch.zeros(1, dtype=torch.int64, device=self.device)
        self.src_val = torch.cat(vals) if sum(self.nsrc) else torch.zeros(1, dtype=self.dtype, device=self.device)
        self._lib = _lib.load()
        self._grids = _lib.grids_array(dims)
        # the graph replays a fixed launch sequence: one cooperative launch (the persistent
        # kernel or the asynchronous work queue), no host reads
        if schedule not in ("persistent", "async"):
            raise ValueError("a captured batch runs the persistent or the asynchronous schedule")
        self._opt = _lib.make_options(tile, schedule, _DT[self.dtype], False, max_iters, order, converge, method,
                                      remedy_order=remedy_order)
        self._Foff, self._poff, self._soff = (_lib.i64_array(self.off), _lib.i64_array(self.off),
                                              _lib.i64_array(self.src_off))
        nbytes = self._lib.eik_workspace_size_batched(len(problems), self._grids, ctypes.byref(self._opt))
        if nbytes == 0:
            raise _lib.EikonalError(_lib.EIK_ERR_ARG, "invalid grids or options")
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.B = len(problems)
        self.graph = None
        with torch.cuda.device(self.device):
            st = _lib.eik_stats()
            _lib.check(self._launch(ctypes.byref(st)))        # first call: checks and device set-up
            if graph:
                side = torch.cuda.Stream(self.device)
                side.wait_stream(torch.cuda.current_stream())
                with torch.cuda.stream(side):
                    _lib.check(self._launch(None))            # warm the side stream
                torch.cuda.current_stream().wait_stream(side)
                self.graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(self.graph):
                    _lib.check(self._launch(None))

    def _launch(self, stats_ptr):
        return self._lib.eik_solve_batched(self.B, self._grids, self.F.data_ptr(), self._Foff,
                                           self.src_idx.data_ptr(), self.src_val.data_ptr(), self._soff,
                                           self.phi.data_ptr(), self._poff, self.ws.data_ptr(), self.ws.numel(),
                                           _stream_ptr(), ctypes.byref(self._opt), stats_ptr)

    def set_speeds(self, b: int, F: torch.Tensor):
        self.F[self.off[b]:self.off[b] + self.sizes[b]].copy_(F.reshape(-1))

    def set_sources(self, b: int, src_idx, src_val=None):
        n = self.nsrc[b]
        i = _as_index(src_idx, self.device)
        if i.numel() != n:
            raise ValueError("the number of sources of an instance is fixed by the captured graph")
        self.src_idx[self.src_off[b]:self.src_off[b] + n].copy_(i)
        self.src_val[self.src_off[b]:self.src_off[b] + n].copy_(_as_values(src_val, n, self.dtype, self.device))

    def solve(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            _lib.check(self._launch(None))
        return [self.phi[self.off[q]:self.off[q] + self.sizes[q]].view(self.shapes[q]) for q in range(self.B)]

    def stats(self) -> dict:
        """Run once outside the graph and return the run statistics (synchronises)."""
        st = _lib.eik_stats()
        _lib.check(self._launch(ctypes.byref(st)))
        return st.as_dict()
