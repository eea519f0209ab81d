"""Python handles over the C ABI: ``Stefan`` (one problem) and ``StefanBatch``.

Arrays may be numpy arrays (host memory, copied synchronously) or torch CUDA
tensors (device memory, used in place on the handle's stream).  No method
computes anything itself.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _abi
from ._abi import check

try:
    import torch
except ImportError:  # the C ABI does not need torch
    torch = None


def _is_cuda_tensor(a):
    return torch is not None and isinstance(a, torch.Tensor) and a.is_cuda


def _ptr(a, dtype=np.float64):
    """(pointer, on_device, keepalive) for a numpy array or a CUDA tensor."""
    if a is None:
        return None, 0, None
    if _is_cuda_tensor(a):
        if not a.is_contiguous():
            raise ValueError("device tensors must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), 1, a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return ctypes.c_void_p(arr.ctypes.data), 0, arr


def _stream_handle(stream):
    if stream is None and torch is not None and torch.cuda.is_available():
        stream = torch.cuda.current_stream()
    if stream is None:
        return None
    if torch is not None and isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


class Stefan:
    """One IREBM problem on the GPU (wraps lbm_stefan_*)."""

    def __init__(self, lattice, nx, ny=1, tau=1.0, delta=0.01, ste=0.1, precision=_abi.LBM_FP64,
                 walls=None, newton_tol=1e-14, newton_max_iter=60, bb_mode=_abi.LBM_BB_MIRROR, stream=None):
        self.lib = _abi.load()
        self.lattice, self.nx, self.ny, self.precision = int(lattice), int(nx), int(ny), int(precision)
        p = _abi.lbm_stefan_params(self.lattice, self.nx, self.ny, float(tau), float(delta), float(ste),
                                   self.precision, float(newton_tol), int(newton_max_iter), int(bb_mode))
        self._stream = _stream_handle(stream)
        h = ctypes.c_void_p()
        check(self.lib.lbm_stefan_create(ctypes.byref(p), self._stream, ctypes.byref(h)))
        self.h = h
        for name, (kind, th) in (walls or {}).items():
            self.set_bc(name, kind, th)
        sb, rs = ctypes.c_size_t(), ctypes.c_int()
        check(self.lib.lbm_stefan_layout(self.h, ctypes.byref(sb), ctypes.byref(rs)))
        self.state_bytes, self.row_stride = sb.value, rs.value

    @classmethod
    def from_case(cls, case, stream=None, **kw):
        kw.setdefault("bb_mode", case.bb_mode)
        return cls(case.lattice, case.nx, case.ny, case.tau, case.delta, case.ste, case.precision,
                   case.walls, stream=stream, **kw)

    # -- forward
    def set_bc(self, wall, kind, theta_wall):
        w = _abi.WALLS[wall] if isinstance(wall, str) else int(wall)
        check(self.lib.lbm_stefan_set_bc(self.h, w, int(kind), float(theta_wall)))

    def set_ste(self, ste):
        check(self.lib.lbm_stefan_set_ste(self.h, float(ste)))

    def set_method(self, method):
        """"IREBM" (Algorithm 3, default), "EEBM" (Algorithm 2) or "ILFBM"
        (Algorithm 1, D1Q3 FP64); set_ic follows."""
        m = {"IREBM": _abi.LBM_IREBM, "EEBM": _abi.LBM_EEBM, "ILFBM": _abi.LBM_ILFBM}.get(method, method)
        check(self.lib.lbm_stefan_set_method(self.h, int(m)))

    def set_ic(self, theta0):
        if not _is_cuda_tensor(theta0):
            theta0 = np.asarray(theta0, dtype=np.float64).reshape(self.ny, self.nx)
        ptr, dev, keep = _ptr(theta0)
        check(self.lib.lbm_stefan_set_ic(self.h, ptr, dev))
        self._keep = keep

    def step(self, n=1):
        check(self.lib.lbm_stefan_step(self.h, int(n)))

    def front_position(self, wall="W"):
        """Interface position from `wall` in node units: (mean first zero, mean
        integrated phase fraction, per-line first zeros, per-line integrated)."""
        w = _abi.WALLS[wall] if isinstance(wall, str) else int(wall)
        n = self.ny if w <= 1 else self.nx
        a, b = ctypes.c_double(), ctypes.c_double()
        la, lb = np.empty(n), np.empty(n)
        dp = ctypes.POINTER(ctypes.c_double)
        check(self.lib.lbm_stefan_front_position(self.h, w, ctypes.byref(a), ctypes.byref(b),
                                                 la.ctypes.data_as(dp), lb.ctypes.data_as(dp)))
        return a.value, b.value, la, lb

    def step_timed(self, nsteps, flat=False):
        """Advance nsteps D2Q9 or D2Q5 steps launch by launch; returns the mean device
        time per step (ms) of the stream/collide kernel and of the job kernel, and
        with flat=True also that of the FP32 D2Q9 flat kernel's launches."""
        out = (ctypes.c_double * 3)()
        check(self.lib.lbm_stefan_step_timed(self.h, int(nsteps), ctypes.cast(out, ctypes.POINTER(ctypes.c_double))))
        return (out[0], out[1], out[2]) if flat else (out[0], out[1])

    def set_wait_test(self, wait_limit_s=2.0, withhold_load=-1):
        """Test hook of the TMA row-pipeline kernel: bound of its waits on row
        loads, and a row load (0, 1, 2) of its first block that it skips; while a
        load is withheld this FP32 D2Q9 handle steps with that kernel (-1: off)."""
        check(self.lib.lbm_stefan_set_wait_test(self.h, float(wait_limit_s), int(withhold_load)))

    def step_record(self, n, traj):
        """traj: CUDA float64 tensor holding at least n planes of ny x row_stride."""
        if not _is_cuda_tensor(traj) or traj.dtype != torch.float64:
            raise ValueError("traj must be a CUDA float64 tensor")
        if traj.numel() < n * self.ny * self.row_stride:
            raise ValueError("traj too small")
        check(self.lib.lbm_stefan_step_record(self.h, int(n), ctypes.c_void_p(traj.data_ptr())))

    def sync(self):
        check(self.lib.lbm_stefan_sync(self.h))

    def fields(self, device=False):
        """(theta, phi, H): numpy arrays, or CUDA tensors with device=True."""
        if device:
            out = [torch.empty((self.ny, self.nx), dtype=torch.float64, device="cuda") for _ in range(3)]
            check(self.lib.lbm_stefan_get_fields(self.h, *[ctypes.c_void_p(t.data_ptr()) for t in out], 1))
            return tuple(out)
        out = [np.empty((self.ny, self.nx)) for _ in range(3)]
        check(self.lib.lbm_stefan_get_fields(self.h, *[ctypes.c_void_p(a.ctypes.data) for a in out], 0))
        return tuple(out)

    def theta(self):
        th = np.empty((self.ny, self.nx))
        check(self.lib.lbm_stefan_get_fields(self.h, ctypes.c_void_p(th.ctypes.data), None, None, 0))
        return th

    def stats(self):
        s = _abi.lbm_stefan_stats()
        check(self.lib.lbm_stefan_get_stats(self.h, ctypes.byref(s)))
        return s.as_dict()

    # -- state
    def new_state_buffer(self):
        return torch.zeros(self.state_bytes, dtype=torch.uint8, device="cuda")

    def get_state(self, buf):
        ptr, dev, _ = _ptr(buf, dtype=np.uint8)
        check(self.lib.lbm_stefan_get_state(self.h, ptr, dev))

    def set_state(self, buf):
        ptr, dev, _ = _ptr(buf, dtype=np.uint8)
        check(self.lib.lbm_stefan_set_state(self.h, ptr, dev))

    def new_theta_planes(self, n):
        return torch.empty((n, self.ny, self.row_stride), dtype=torch.float64, device="cuda")

    def theta_plane(self, plane):
        check(self.lib.lbm_stefan_theta_plane(self.h, ctypes.c_void_p(plane.data_ptr())))

    # -- adjoint
    def adjoint_seed(self, theta_T, phi_target, adj, want_loss=True):
        loss = ctypes.c_double()
        check(self.lib.lbm_stefan_adjoint_seed(self.h, ctypes.c_void_p(theta_T.data_ptr()),
                                               ctypes.c_void_p(phi_target.data_ptr()),
                                               ctypes.c_void_p(adj.data_ptr()),
                                               ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def adjoint_step(self, theta_t, theta_t1, adj_in, adj_out):
        check(self.lib.lbm_stefan_adjoint_step(self.h, ctypes.c_void_p(theta_t.data_ptr()),
                                               ctypes.c_void_p(theta_t1.data_ptr()),
                                               ctypes.c_void_p(adj_in.data_ptr()),
                                               ctypes.c_void_p(adj_out.data_ptr())))

    def adjoint_run(self, traj, adj, adj_other):
        """len(traj)-1 reverse steps over the recorded planes traj (theta(t0) ..
        theta(t0+n), one contiguous tensor); returns (result, spare) buffers."""
        idx = ctypes.c_int()
        check(self.lib.lbm_stefan_adjoint_run(self.h, int(traj.shape[0]) - 1, ctypes.c_void_p(traj.data_ptr()),
                                              ctypes.c_void_p(adj.data_ptr()), ctypes.c_void_p(adj_other.data_ptr()),
                                              ctypes.byref(idx)))
        return (adj, adj_other) if idx.value == 0 else (adj_other, adj)

    def adjoint_segment(self, checkpoint, n, traj, adj, adj_other):
        """Reload `checkpoint`, recompute n steps recording theta into traj[:n+1],
        run n reverse steps; returns (result, spare) buffers."""
        idx = ctypes.c_int()
        check(self.lib.lbm_stefan_adjoint_segment(self.h, ctypes.c_void_p(checkpoint.data_ptr()), int(n),
                                                  ctypes.c_void_p(traj.data_ptr()), ctypes.c_void_p(adj.data_ptr()),
                                                  ctypes.c_void_p(adj_other.data_ptr()), ctypes.byref(idx)))
        return (adj, adj_other) if idx.value == 0 else (adj_other, adj)

    def adjoint_finish(self, adj0, g_theta0):
        gw = (ctypes.c_double * 4)()
        gs = ctypes.c_double()
        ptr, dev, _ = _ptr(g_theta0)
        check(self.lib.lbm_stefan_adjoint_finish(self.h, ctypes.c_void_p(adj0.data_ptr()), ptr, dev,
                                                 ctypes.cast(gw, ctypes.POINTER(ctypes.c_double)),
                                                 ctypes.byref(gs)))
        return list(gw), gs.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.lbm_stefan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class StefanBatch:
    """Many independent D2Q9 problems advanced by one persistent launch per step."""

    def __init__(self, cases, precision=_abi.LBM_FP32, newton_tol=1e-14, newton_max_iter=60, stream=None):
        self.lib = _abi.load()
        arr = (_abi.lbm_stefan_problem * len(cases))()
        for k, c in enumerate(cases):
            arr[k].nx, arr[k].ny = int(c.nx), int(c.ny)
            arr[k].tau, arr[k].delta, arr[k].ste = float(c.tau), float(c.delta), float(c.ste)
            for name, w in _abi.WALLS.items():
                kind, th = c.walls.get(name, (0, 0.0))
                arr[k].wall_kind[w] = int(kind)
                arr[k].wall_theta[w] = float(th)
        self.cases = list(cases)
        self._stream = _stream_handle(stream)
        h = ctypes.c_void_p()
        check(self.lib.lbm_stefan_batch_create(len(cases), arr, int(precision), float(newton_tol),
                                               int(newton_max_iter), self._stream, ctypes.byref(h)))
        self.h = h

    def set_ic(self, k, theta0):
        c = self.cases[k]
        if not _is_cuda_tensor(theta0):
            theta0 = np.asarray(theta0, dtype=np.float64).reshape(c.ny, c.nx)
        ptr, dev, keep = _ptr(theta0)
        check(self.lib.lbm_stefan_batch_set_ic(self.h, int(k), ptr, dev))

    def step(self, n=1):
        check(self.lib.lbm_stefan_batch_step(self.h, int(n)))

    def theta(self, k):
        c = self.cases[k]
        th = np.empty((c.ny, c.nx))
        check(self.lib.lbm_stefan_batch_get_fields(self.h, int(k), ctypes.c_void_p(th.ctypes.data), 0))
        return th

    def stats(self, k):
        s = _abi.lbm_stefan_stats()
        check(self.lib.lbm_stefan_batch_get_stats(self.h, int(k), ctypes.byref(s)))
        return s.as_dict()

    def autotune(self, trial_steps=20):
        th = ctypes.c_int()
        check(self.lib.lbm_stefan_batch_autotune(self.h, int(trial_steps), ctypes.byref(th)))
        return th.value

    def set_schedule(self, tile_h, schedule=1):
        check(self.lib.lbm_stefan_batch_set_schedule(self.h, int(tile_h), int(schedule)))

    def close(self):
        if getattr(self, "h", None):
            self.lib.lbm_stefan_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
