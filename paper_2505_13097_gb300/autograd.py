"""torch.autograd.Function over the IREBM forward run and its discrete adjoint.

    L(theta0, theta_wall, Ste) = 1/2 sum_x (phi(theta_T(x)) - phi_target(x))^2

after ``steps`` steps from theta0.  The forward pass keeps a copy of the
state every ``checkpoint_every`` steps (default ceil(sqrt(steps))).  The
backward pass walks the segments from last to first: it reloads the
segment's checkpoint, recomputes the segment forward while recording
theta(t) (one FP64 plane per step), then runs the adjoint step kernel
backwards through the segment (on D2Q9 one lbm_stefan_adjoint_segment call
per segment, replayed as a CUDA graph).  Memory: sqrt(T) states plus
sqrt(T) theta planes instead of T states.

A run's handle and buffers (the library handle, checkpoints, theta planes,
adjoint buffers and a CUDA stream of its own) are kept in a small pool and
reused by the next call with the same lattice, size, parameters, wall kinds
and step count; Ste and the wall temperatures are set on the kept handle.

All arithmetic runs in the CUDA library (lbm_stefan_step, _step_record,
lbm_stefan_adjoint_*); this module only orders the calls and owns the
buffers (torch tensors).
"""
from __future__ import annotations

import collections
import math
import threading

import torch

from . import _abi
from .solver import Stefan

_POOL_SIZE = 2
_pool: "collections.OrderedDict" = collections.OrderedDict()
_pool_lock = threading.Lock()


def _wall_names(case):
    return ("W", "E") if case.lattice == _abi.LBM_D1Q3 else ("W", "E", "S", "N")


class _Run:
    """Handle, stream and buffers of one checkpointed forward/backward pair."""

    def __init__(self, case, steps, every, bb_mode, ste):
        self.stream = torch.cuda.Stream()
        names = _wall_names(case)
        self.kinds = {n: case.walls.get(n, (_abi.LBM_ADIABATIC, 0.0))[0] for n in names}
        walls = {n: (self.kinds[n], case.walls.get(n, (0, 0.0))[1]) for n in names}
        self.S = Stefan(case.lattice, case.nx, case.ny, case.tau, case.delta, float(ste), case.precision, walls,
                        bb_mode=bb_mode, stream=self.stream)
        self.ste = float(ste)
        self.wall_theta = {n: walls[n][1] for n in names}
        self.starts = list(range(0, steps, every))
        self.ends = self.starts[1:] + [steps]
        with torch.cuda.stream(self.stream):
            self.checkpoints = [self.S.new_state_buffer() for _ in self.starts]
            self.planes = self.S.new_theta_planes(max(e - s for s, e in zip(self.starts, self.ends)) + 1)
            self.adj = self.S.new_state_buffer()
            self.other = self.S.new_state_buffer()

    def set_params(self, theta_wall, ste):
        S = self.S
        if float(ste) != self.ste:
            S.set_ste(float(ste))
            self.ste = float(ste)
        for k, name in enumerate(self.kinds):
            th = float(theta_wall[k])
            if th != self.wall_theta[name]:
                S.set_bc(name, self.kinds[name], th)
                self.wall_theta[name] = th

    def forward(self, theta0, theta_wall, ste, phi_target):
        S = self.S
        self.stream.wait_stream(torch.cuda.current_stream())
        self.set_params(theta_wall, ste)
        S.set_ic(theta0)
        for buf, start, end in zip(self.checkpoints, self.starts, self.ends):
            S.get_state(buf)
            S.step(end - start)
        S.theta_plane(self.planes[0])
        return S.adjoint_seed(self.planes[0], phi_target, self.adj)

    def backward(self):
        S = self.S
        adj, other = self.adj, self.other
        for buf, start, end in reversed(list(zip(self.checkpoints, self.starts, self.ends))):
            n = end - start
            traj = self.planes[:n + 1]
            if S.lattice == _abi.LBM_D2Q9:
                adj, other = S.adjoint_segment(buf, n, self.planes, adj, other)
            else:
                S.set_state(buf)
                S.theta_plane(traj[0])
                S.step_record(n, traj[1:])
                adj, other = S.adjoint_run(traj, adj, other)
        g0 = torch.empty((S.ny, S.nx), dtype=torch.float64, device="cuda")   # on the caller's stream
        self.stream.wait_stream(torch.cuda.current_stream())
        gw, gs = S.adjoint_finish(adj, g0)   # synchronizes the run's stream
        return g0, gw, gs

    def close(self):
        self.S.close()


def _key(case, steps, every, bb_mode):
    kinds = tuple(case.walls.get(n, (0, 0.0))[0] for n in _wall_names(case))
    return (case.lattice, case.nx, case.ny, case.tau, case.delta, case.precision, kinds, steps, every, bb_mode,
            torch.cuda.current_device())


def _take(key, make):
    with _pool_lock:
        run = _pool.pop(key, None)
    return run if run is not None else make()


def _give(key, run):
    drop = []
    with _pool_lock:
        old = _pool.pop(key, None)
        if old is not None:
            drop.append(old)
        _pool[key] = run
        while len(_pool) > _POOL_SIZE:
            drop.append(_pool.popitem(last=False)[1])
    for r in drop:
        r.close()


def clear_pool():
    """Release every kept handle and buffer."""
    with _pool_lock:
        runs = list(_pool.values())
        _pool.clear()
    for r in runs:
        r.close()


class StefanMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta0, theta_wall, ste, case, steps, phi_target, checkpoint_every=None, bb_mode=0):
        """theta0: (ny, nx) float64 CUDA tensor; theta_wall: (4,) float64 tensor
        (W, E, S, N values; used on the case's Dirichlet walls); ste: 0-d tensor."""
        every = int(checkpoint_every or max(1, math.ceil(math.sqrt(steps))))
        key = _key(case, steps, every, bb_mode)
        run = _take(key, lambda: _Run(case, steps, every, bb_mode, float(ste)))
        tw = [float(v) for v in theta_wall.detach().cpu()]
        loss = run.forward(theta0.detach().contiguous(), tw, float(ste), phi_target.detach().contiguous())
        if any(ctx.needs_input_grad[:3]):
            ctx.run, ctx.key = run, key
        else:
            ctx.run = None
            _give(key, run)   # no backward will follow
        return torch.tensor(loss, dtype=torch.float64, device=theta0.device)

    @staticmethod
    def backward(ctx, grad):
        run, ctx.run = ctx.run, None
        g0, gw, gs = run.backward()
        _give(ctx.key, run)
        g = grad.to(torch.float64)
        return (g0 * g, torch.tensor(gw, dtype=torch.float64, device=g0.device) * g,
                torch.tensor(gs, dtype=torch.float64, device=g0.device) * g, None, None, None, None, None)


def misfit(theta0, theta_wall, ste, case, steps, phi_target, checkpoint_every=None, bb_mode=0):
    """Differentiable liquid-fraction misfit after ``steps`` IREBM steps."""
    return StefanMisfit.apply(theta0, theta_wall, ste, case, steps, phi_target, checkpoint_every, bb_mode)
