"""torch.autograd.Function over the IREBM forward run and its discrete adjoint.

    L(theta0, theta_wall, Ste) = 1/2 sum_x (phi(theta_T(x)) - phi_target(x))^2

after ``steps`` steps from theta0.  The forward pass keeps a copy of the
state every ``checkpoint_every`` steps (default ceil(sqrt(steps))).  The
backward pass walks the segments from last to first: it reloads the
segment's checkpoint, recomputes the segment forward while recording
theta(t) (one FP64 plane per step), then runs the adjoint step kernel
backwards through the segment.  Memory: sqrt(T) states plus sqrt(T) theta
planes instead of T states.

All arithmetic runs in the CUDA library (lbm_stefan_step_record,
lbm_stefan_adjoint_*); this module only orders the calls and owns the
buffers (torch tensors).
"""
from __future__ import annotations

import math

import torch

from . import _abi
from .solver import Stefan


class StefanMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta0, theta_wall, ste, case, steps, phi_target, checkpoint_every=None, bb_mode=0):
        """theta0: (ny, nx) float64 CUDA tensor; theta_wall: (4,) float64 tensor
        (W, E, S, N values; used on the case's Dirichlet walls); ste: 0-d tensor."""
        walls = {}
        names = ("W", "E") if case.lattice == _abi.LBM_D1Q3 else ("W", "E", "S", "N")
        for k, name in enumerate(names):
            kind, _ = case.walls.get(name, (_abi.LBM_ADIABATIC, 0.0))
            walls[name] = (kind, float(theta_wall[k]))
        S = Stefan(case.lattice, case.nx, case.ny, case.tau, case.delta, float(ste), case.precision, walls,
                   bb_mode=bb_mode)
        S.set_ic(theta0.detach().contiguous())
        C = int(checkpoint_every or max(1, math.ceil(math.sqrt(steps))))
        checkpoints = []
        done = 0
        while done < steps:
            buf = S.new_state_buffer()
            S.get_state(buf)
            checkpoints.append((done, buf))
            n = min(C, steps - done)
            S.step(n)
            done += n
        plane = S.new_theta_planes(1)
        S.theta_plane(plane[0])
        adj = S.new_state_buffer()
        target = phi_target.detach().contiguous()
        loss = S.adjoint_seed(plane[0], target, adj)
        ctx.S, ctx.checkpoints, ctx.adj, ctx.steps = S, checkpoints, adj, steps
        return torch.tensor(loss, dtype=torch.float64, device=theta0.device)

    @staticmethod
    def backward(ctx, grad):
        S = ctx.S
        adj = ctx.adj
        other = S.new_state_buffer()
        starts = [c[0] for c in ctx.checkpoints]
        ends = starts[1:] + [ctx.steps]
        planes = S.new_theta_planes(max(e - s for s, e in zip(starts, ends)) + 1)
        for (start, buf), end in reversed(list(zip(ctx.checkpoints, ends))):
            n = end - start
            traj = planes[:n + 1]
            S.set_state(buf)
            S.theta_plane(traj[0])
            S.step_record(n, traj[1:])
            adj, other = S.adjoint_run(traj, adj, other)
        g0 = torch.empty((S.ny, S.nx), dtype=torch.float64, device="cuda")
        gw, gs = S.adjoint_finish(adj, g0)
        S.close()
        ctx.S = None
        g = grad.to(torch.float64)
        return (g0 * g, torch.tensor(gw, dtype=torch.float64, device=g0.device) * g,
                torch.tensor(gs, dtype=torch.float64, device=g0.device) * g, None, None, None, None, None)


def misfit(theta0, theta_wall, ste, case, steps, phi_target, checkpoint_every=None, bb_mode=0):
    """Differentiable liquid-fraction misfit after ``steps`` IREBM steps."""
    return StefanMisfit.apply(theta0, theta_wall, ste, case, steps, phi_target, checkpoint_every, bb_mode)
