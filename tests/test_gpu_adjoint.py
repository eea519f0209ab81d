"""Adjoint of the GPU step (through the C ABI, driven by the autograd Function).

Checks: the oracle's FP64 discrete adjoint on a 64 x 64 problem with the
parameters and step count of the 1024^2 adjoint workload (2,000 steps), central
finite differences (h = 1e-4) of the GPU FP64 forward to 1e-4 relative, the
FP32 form against the FP64 adjoint, and independence from the checkpoint
interval.
"""
import numpy as np
import pytest

from paper_2505_13097_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def phi(x, d):
    return 0.5 * (1.0 + np.tanh(x / d))


def make_problem(orc, n=64, steps=2000, precision=0):
    base = workloads.adjoint_2d(n=n, steps=steps, precision=precision)
    tcase = workloads.adjoint_target_case(base)
    t0 = workloads.adjoint_target_theta0(base)
    P = orc.Problem(2, n, n, tau=tcase.tau, delta=tcase.delta, ste=tcase.ste, walls=tcase.walls)
    _, thT = P.run(t0, steps)
    return base, phi(thT, base.delta)


def gpu_grad(torch, case, target, steps=None, checkpoint_every=None, ste=None, wall=None, theta0=None, bb_mode=0):
    from paper_2505_13097_gb300.autograd import misfit
    steps = case.steps if steps is None else steps
    th0 = torch.tensor(case.theta0() if theta0 is None else theta0, device="cuda", requires_grad=True)
    tw = torch.tensor([case.walls.get(k, (0, 0.0))[1] for k in "WESN"], dtype=torch.float64, device="cuda")
    if wall is not None:
        tw = tw + torch.tensor(wall, dtype=torch.float64, device="cuda")
    tw.requires_grad_(True)
    st = torch.tensor(case.ste if ste is None else ste, dtype=torch.float64, device="cuda", requires_grad=True)
    tgt = torch.tensor(target, device="cuda")
    L = misfit(th0, tw, st, case, steps, tgt, checkpoint_every, bb_mode)
    L.backward()
    return float(L.detach()), th0.grad.cpu().numpy(), tw.grad.cpu().numpy(), float(st.grad)


def oracle_adjoint_floor(P, theta0, steps, target):
    """Oracle adjoint and its FP64 rounding floor: the relative change of L and of
    the gradients when theta0 moves by one ulp at random nodes (the forward run
    amplifies rounding at nodes leaving the mushy zone)."""
    ref = P.adjoint(theta0, steps, target)
    rng = np.random.Generator(np.random.PCG64(12345))
    pert = theta0 + np.spacing(theta0) * rng.choice([-1, 0, 1], size=theta0.shape)
    alt = P.adjoint(pert, steps, target)
    fl = abs(alt[0] - ref[0]) / abs(ref[0])
    fg = np.max(np.abs(alt[1] - ref[1])) / np.max(np.abs(ref[1]))
    fw = abs(alt[2][0] - ref[2][0]) / max(abs(ref[2][0]), 1e-300)
    fs = abs(alt[3] - ref[3]) / abs(ref[3])
    return ref, (fl, fg, fw, fs)


def test_fp64_adjoint_matches_oracle_adjoint(torch_mod, orc):
    case, target = make_problem(orc)
    L, g0, gw, gs = gpu_grad(torch_mod, case, target)
    P = orc.Problem(2, case.nx, case.ny, tau=case.tau, delta=case.delta, ste=case.ste, walls=case.walls)
    (Lo, g0o, gwo, gso), (fl, fg, fw, fs) = oracle_adjoint_floor(P, case.theta0(), case.steps, target)
    assert abs(L - Lo) <= max(1e-10, 10 * fl) * abs(Lo)
    assert np.max(np.abs(g0 - g0o)) <= max(1e-9, 10 * fg) * np.max(np.abs(g0o))
    assert abs(gw[0] - gwo[0]) <= max(1e-9, 10 * fw) * abs(gwo[0])
    assert abs(gs - gso) <= max(1e-9, 10 * fs) * abs(gso)


@pytest.mark.parametrize("bb_mode", [0, 1])
def test_fp64_adjoint_oracle_walls(torch_mod, orc, bb_mode):
    walls = {"W": (1, 0.9), "S": (1, -0.3), "E": (0, 0.0), "N": (0, 0.0)}
    case = workloads.Case("t", 2, 70, 45, 0.84, 0.03, 0.2, walls, 80, workloads.FP64)
    th0 = workloads.random_field((45, 70), -0.15, 0.15, seed=31)
    target = workloads.random_field((45, 70), 0.0, 1.0, seed=32)
    L, g0, gw, gs = gpu_grad(torch_mod, case, target, theta0=th0, bb_mode=bb_mode)
    P = orc.Problem(2, 70, 45, tau=0.84, delta=0.03, ste=0.2, walls=walls, bb_mode=bb_mode)
    Lo, g0o, gwo, gso = P.adjoint(th0, 80, target)
    assert abs(L - Lo) <= 1e-10 * abs(Lo)
    assert np.max(np.abs(g0 - g0o)) <= 1e-9 * np.max(np.abs(g0o))
    for k in (0, 2):
        assert abs(gw[k] - gwo[k]) <= 1e-9 * max(abs(gwo[k]), 1e-12)
    assert abs(gs - gso) <= 1e-9 * abs(gso)


def test_d1q3_adjoint_matches_oracle(torch_mod, orc):
    case = workloads.melt_1d(n=200, steps=600)
    target = phi(workloads.random_field((1, 200), -0.05, 0.05, seed=4), case.delta)
    L, g0, gw, gs = gpu_grad(torch_mod, case, target)
    P = orc.Problem(1, 200, 1, tau=case.tau, delta=case.delta, ste=case.ste, walls=case.walls)
    Lo, g0o, gwo, gso = P.adjoint(case.theta0(), case.steps, target)
    assert abs(L - Lo) <= 1e-10 * abs(Lo)
    assert np.max(np.abs(g0 - g0o)) <= 1e-9 * np.max(np.abs(g0o))
    assert abs(gs - gso) <= 1e-9 * abs(gso)


def test_fp64_adjoint_central_differences(torch_mod, orc):
    from paper_2505_13097_gb300.autograd import misfit
    torch = torch_mod
    case, target = make_problem(orc, n=64, steps=400)
    L, g0, gw, gs = gpu_grad(torch, case, target)
    h = 1e-4
    tgt = torch.tensor(target, device="cuda")

    def loss(theta0, wall_w, ste):
        tw = torch.tensor([wall_w, 0.0, 0.0, 0.0], dtype=torch.float64, device="cuda")
        with torch.no_grad():
            return float(misfit(torch.tensor(theta0, device="cuda"), tw, torch.tensor(ste, dtype=torch.float64),
                                case, case.steps, tgt))

    th0, tw0 = case.theta0(), case.walls["W"][1]
    v = workloads.random_direction(th0.shape, seed=77)

    def cdiff(f):
        # central differences with h = 1e-4 and h/2, Richardson-extrapolated
        # (removes the O(h^2) truncation term, which alone is ~1e-4 here)
        d1 = (f(h) - f(-h)) / (2 * h)
        d2 = (f(h / 2) - f(-h / 2)) / h
        return (4 * d2 - d1) / 3

    fd = cdiff(lambda e: loss(th0 + e * v, tw0, case.ste))
    assert abs(np.sum(g0 * v) - fd) <= 1e-4 * abs(fd)
    fdw = cdiff(lambda e: loss(th0, tw0 + e, case.ste))
    assert abs(gw[0] - fdw) <= 1e-4 * abs(fdw)
    # Ste = 0.1: a step of 1e-4 relative (1e-5 absolute); an absolute 1e-4 step
    # leaves a truncation error of ~5e-3 because L bends sharply in Ste
    hs = 1e-4 * case.ste
    d1 = (loss(th0, tw0, case.ste + hs) - loss(th0, tw0, case.ste - hs)) / (2 * hs)
    d2 = (loss(th0, tw0, case.ste + hs / 2) - loss(th0, tw0, case.ste - hs / 2)) / hs
    fds = (4 * d2 - d1) / 3
    assert abs(gs - fds) <= 1e-4 * abs(fds)


def test_fp32_adjoint_close_to_fp64(torch_mod, orc):
    case64, target = make_problem(orc, n=64, steps=500, precision=0)
    case32 = case64.scaled(precision=1)
    _, g64, gw64, gs64 = gpu_grad(torch_mod, case64, target)
    _, g32, gw32, gs32 = gpu_grad(torch_mod, case32, target)
    assert np.max(np.abs(g32 - g64)) <= 2e-3 * np.max(np.abs(g64))
    assert abs(gs32 - gs64) <= 2e-3 * abs(gs64)
    assert abs(gw32[0] - gw64[0]) <= 2e-3 * abs(gw64[0])


def test_checkpoint_interval_does_not_change_gradient(torch_mod, orc):
    case, target = make_problem(orc, n=64, steps=130)
    a = gpu_grad(torch_mod, case, target, checkpoint_every=130)
    b = gpu_grad(torch_mod, case, target, checkpoint_every=7)
    assert a[0] == b[0]
    assert np.max(np.abs(a[1] - b[1])) <= 1e-13 * np.max(np.abs(a[1]))
    assert abs(a[3] - b[3]) <= 1e-12 * abs(a[3])


# Shapes for the marching D2Q9 adjoint: several segments (64 columns in the
# FP32 form, 32 in the FP64 form) with a ragged last one, an east wall in the
# column right of a segment (nx = 64k + 1), several row tiles with a ragged
# last one, and rows fewer than a tile.
ADJ_SHAPES = [(193, 75), (129, 40), (97, 33), (66, 2), (33, 3)]
ADJ_WALLS = [
    {"W": (1, 0.9), "E": (1, -0.4), "S": (0, 0.0), "N": (1, 0.2)},
    {"W": (0, 0.0), "E": (1, 0.6), "S": (1, -0.3), "N": (0, 0.0)},
]


def _adj_case(nx, ny, walls, precision, steps):
    case = workloads.Case("t", 2, nx, ny, 0.8, 0.03, 0.25, walls, steps, precision)
    # mushy and saturated regions both present
    th0 = workloads.random_field((ny, nx), -0.4, 0.4, seed=nx * 1000 + ny)
    target = workloads.random_field((ny, nx), 0.0, 1.0, seed=nx + 7 * ny)
    return case, th0, target


@pytest.mark.parametrize("shape", ADJ_SHAPES)
@pytest.mark.parametrize("wi", [0, 1])
@pytest.mark.parametrize("bb_mode", [0, 1])
def test_fp64_adjoint_oracle_shapes(torch_mod, orc, shape, wi, bb_mode):
    nx, ny = shape
    case, th0, target = _adj_case(nx, ny, ADJ_WALLS[wi], workloads.FP64, 25)
    L, g0, gw, gs = gpu_grad(torch_mod, case, target, theta0=th0, bb_mode=bb_mode)
    P = orc.Problem(2, nx, ny, tau=case.tau, delta=case.delta, ste=case.ste, walls=case.walls, bb_mode=bb_mode)
    Lo, g0o, gwo, gso = P.adjoint(th0, case.steps, target)
    assert abs(L - Lo) <= 1e-10 * abs(Lo)
    assert np.max(np.abs(g0 - g0o)) <= 1e-9 * np.max(np.abs(g0o))
    for k in range(4):
        if case.walls[k_name(k)][0] == 1:
            assert abs(gw[k] - gwo[k]) <= 1e-9 * max(abs(gwo[k]), 1e-12)
        else:
            assert gw[k] == 0.0
    assert abs(gs - gso) <= 1e-9 * abs(gso)


@pytest.mark.parametrize("shape", ADJ_SHAPES)
@pytest.mark.parametrize("bb_mode", [0, 1])
def test_fp32_adjoint_oracle_shapes(torch_mod, orc, shape, bb_mode):
    """FP32 form (FP32 populations and adjoint, interior terms in FP32) against
    the FP64 oracle adjoint: within 2e-3 of the largest gradient entry."""
    nx, ny = shape
    case, th0, target = _adj_case(nx, ny, ADJ_WALLS[0], workloads.FP32, 25)
    L, g0, gw, gs = gpu_grad(torch_mod, case, target, theta0=th0, bb_mode=bb_mode)
    P = orc.Problem(2, nx, ny, tau=case.tau, delta=case.delta, ste=case.ste, walls=case.walls, bb_mode=bb_mode)
    Lo, g0o, gwo, gso = P.adjoint(th0, case.steps, target)
    assert abs(L - Lo) <= 1e-4 * abs(Lo)
    assert np.max(np.abs(g0 - g0o)) <= 2e-3 * np.max(np.abs(g0o))
    for k in range(4):
        if case.walls[k_name(k)][0] == 1:
            assert abs(gw[k] - gwo[k]) <= 2e-3 * max(abs(gwo[k]), 1e-12)
    assert abs(gs - gso) <= 2e-3 * abs(gso)


def k_name(k):
    return "WESN"[k]


def test_adjoint_run_matches_single_steps(torch_mod, orc):
    """lbm_stefan_adjoint_run over a recorded segment equals the same reverse
    steps issued one at a time (bit for bit)."""
    from paper_2505_13097_gb300 import solver
    torch = torch_mod
    case, th0, target = _adj_case(129, 40, ADJ_WALLS[1], workloads.FP32, 9)
    S = solver.Stefan.from_case(case)
    S.set_ic(th0)
    traj = S.new_theta_planes(case.steps + 1)
    S.theta_plane(traj[0])
    S.step_record(case.steps, traj[1:])
    a = S.new_state_buffer()
    S.adjoint_seed(traj[-1], torch.tensor(target, device="cuda"), a, want_loss=False)
    b = a.clone()
    x, y = S.new_state_buffer(), S.new_state_buffer()
    res, _ = S.adjoint_run(traj, a, x)
    for s in range(case.steps - 1, -1, -1):
        S.adjoint_step(traj[s], traj[s + 1], b, y)
        b, y = y, b
    torch.cuda.synchronize()
    assert torch.equal(res, b)
    S.close()
