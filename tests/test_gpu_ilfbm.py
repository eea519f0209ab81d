"""ILFBM (Algorithm 1, the implicit liquid fraction based method) on the GPU
in FP64, D1Q3 and D2Q9 (and D2Q5, whose inner loop does not converge),
against the oracle's ILFBM (``oracle.Problem.ilfbm_run``).

Parity: theta to 1e-12 relative (FP64), the liquid fraction to 1e-10
absolute (the lever rule's slope Ste maps theta's rounding into l), or ten
times the problem's own rounding floor where that is larger (random fields
with many mushy nodes: up to 1e-11 for the oracle against itself started one
ulp away, 801 nodes, 300 steps).  The smooth single-front paper case keeps
the plain 1e-12.
"""
import json
import os

import numpy as np
import pytest

from oracle import neumann
from paper_2505_13097_gb300 import _abi, workloads

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_1d_case.json")


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_13097_gb300 import solver
    return solver


def make(gpu, n, tau, ste, walls, bb_mode=0, tol=1e-12, maxit=200):
    S = gpu.Stefan(_abi.LBM_D1Q3, n, 1, tau, 0.01, ste, _abi.LBM_FP64, walls, newton_tol=tol, newton_max_iter=maxit,
                   bb_mode=bb_mode)
    S.set_method("ILFBM")
    return S


@pytest.mark.parametrize("n", [2, 5, 64, 513, 801, 2844])
@pytest.mark.parametrize("wi", [0, 1, 2])
@pytest.mark.parametrize("bb_mode", [0, 1])
def test_ilfbm_parity(gpu, orc, n, wi, bb_mode):
    walls = [{"W": (1, 1.0), "E": (1, -0.5)}, {"W": (1, 0.8), "E": (0, 0.0)}, {}][wi]
    tau, ste, steps = 0.62, 0.2857, 300
    th0 = workloads.random_field((1, n), -0.6, 0.4, seed=n + 7 * wi)
    S = make(gpu, n, tau, ste, walls, bb_mode)
    S.set_ic(th0)
    S.step(steps)
    th, l, H = S.fields()
    st = S.stats()
    S.close()
    P = orc.Problem(1, n, 1, tau=tau, delta=0.01, ste=ste, walls=walls, bb_mode=bb_mode)
    _, lo, tho, failed, mx = P.ilfbm_run(th0, steps, tol=1e-12, maxit=200)
    # the problem's own FP64 rounding floor (as for IREBM): the oracle against the
    # oracle started one ulp away at random nodes, the largest of three such
    # starts (random fields put many nodes in the mushy band, which amplifies
    # rounding; the floor varies by 6x between starts)
    fl_t = fl_l = 0.0
    for seed in (12345, 1, 2):
        rng = np.random.Generator(np.random.PCG64(seed))
        pert = th0 + np.spacing(th0) * rng.choice([-1, 0, 1], size=th0.shape)
        _, lp_, thp, _, _ = P.ilfbm_run(pert, steps, tol=1e-12, maxit=200)
        fl_t = max(fl_t, np.max(np.abs(thp - tho)))
        fl_l = max(fl_l, np.max(np.abs(lp_ - lo)))
    tol_t = max(1e-12, 10 * fl_t / np.max(np.abs(tho)))
    tol_l = max(1e-10, 10 * fl_l)
    assert failed == 0 and st["error"] == 0
    assert np.max(np.abs(th - tho)) <= tol_t * np.max(np.abs(tho))
    assert np.max(np.abs(l - lo)) <= tol_l
    assert np.max(np.abs(H - (th + l / ste))) <= 1e-12 * np.max(np.abs(H))
    assert 1 <= st["newton_max_iter"] <= mx


def test_ilfbm_closed_bar_conserves_energy(gpu):
    # link-wise bounce-back at both ends: sum theta + l/Ste is kept by every inner
    # iteration, so by every converged step to the loop's tolerance
    n, ste = 400, 0.5
    S = make(gpu, n, 0.8, ste, {}, bb_mode=1, tol=1e-13)
    S.set_ic(workloads.random_field((1, n), -0.6, 0.6, seed=3))
    e0 = S.stats()["energy"]
    S.step(500)
    st = S.stats()
    assert st["error"] == 0
    assert abs(st["energy"] - e0) <= 500 * n * 1e-13 / ste + 1e-11 * abs(e0)
    assert st["imbalance_max"] <= n * 1e-13 / ste + 1e-11 * abs(e0)


def test_ilfbm_iteration_limit_reports_error(gpu):
    # one inner iteration cannot settle a moving front: the loop stops at its
    # limit and the step reports LBM_ERR_NEWTON (the state stays usable)
    S = make(gpu, 128, 0.62, 0.2857, {"W": (1, 1.0), "E": (1, -0.5)}, maxit=1)
    S.set_ic(np.full((1, 128), -0.5))
    S.step(50)
    with pytest.raises(_abi.LBMError) as e:
        S.sync()
    assert e.value.status == _abi.LBM_ERR_NEWTON
    S.close()


def test_ilfbm_paper_1d_case(gpu, orc):
    """Sec. 6.1 bar (N = 801, Ste = 0.2857, tau = 0.62) on the GPU: the printed
    final-time maximum error of ILFBM, 4.50e-3, lies within the band that the
    error sweeps over the last cell crossing of the front (the sharp front
    jumps from node to node), and the first 20,000 steps equal the oracle's."""
    g = json.load(open(GOLDEN))
    ste, th_c, n, tau = g["ste"], g["theta0"], g["N"], g["tau"]
    lam = neumann.stefan_lambda(ste, th_c)
    t0 = (g["x_f0"] / (2 * lam)) ** 2
    dx = 1.0 / (n - 1)
    dt = (tau - 0.5) * dx * dx / 3.0
    steps = int(round((g["t_final"] - t0) / dt))
    window = int(round(dx / (lam / np.sqrt(g["t_final"])) / dt))
    x = np.arange(n) * dx
    init = neumann.profile(x, t0, ste, th_c, lam)[None, :]
    walls = {"W": (_abi.LBM_DIRICHLET, 1.0), "E": (_abi.LBM_DIRICHLET, th_c)}
    S = make(gpu, n, tau, ste, walls)
    S.set_ic(init)
    S.step(20000)
    th_20k = S.theta()
    S.step(steps - window - 20000)
    errs = []
    done = steps - window
    while done < steps:
        k = min(100, steps - done)
        S.step(k)
        done += k
        errs.append(np.max(np.abs(S.theta()[0] - neumann.profile(x, t0 + done * dt, ste, th_c, lam))))
    st = S.stats()
    S.close()
    assert st["error"] == 0
    assert min(errs) <= g["max_error_ilfbm"] <= max(errs), (min(errs), max(errs))
    P = orc.Problem(1, n, 1, tau=tau, delta=g["delta"], ste=ste, walls={"W": (1, 1.0), "E": (1, th_c)})
    _, _, tho, failed, _ = P.ilfbm_run(init, 20000, tol=1e-12, maxit=200)
    assert failed == 0
    assert np.max(np.abs(th_20k - tho)) <= 1e-12


def test_ilfbm_argument_errors(gpu):
    cases = [
        (_abi.LBM_D1Q3, 64, 1, _abi.LBM_FP32),
        (_abi.LBM_D1Q3, 2845, 1, _abi.LBM_FP64),
    ]
    for lat, nx, ny, prec in cases:
        S = gpu.Stefan(lat, nx, ny, 0.8, 0.01, 0.1, prec, {})
        with pytest.raises(_abi.LBMError) as e:
            S.set_method("ILFBM")
        assert e.value.status == _abi.LBM_ERR_ARG
        S.close()
    import torch
    S = make(gpu, 64, 0.8, 0.1, {"W": (1, 1.0)})
    S.set_ic(np.full((1, 64), -0.2))
    traj = torch.empty(2 * S.row_stride, dtype=torch.float64, device="cuda")
    with pytest.raises(_abi.LBMError) as e:
        S.step_record(2, traj)
    assert e.value.status == _abi.LBM_ERR_STATE
    planes = S.new_theta_planes(2)
    a, b = S.new_state_buffer(), S.new_state_buffer()
    with pytest.raises(_abi.LBMError) as e:
        S.adjoint_step(planes[0], planes[1], a, b)
    assert e.value.status == _abi.LBM_ERR_STATE
    S.close()


# ---------------------------------------------------------------- 2D lattices
ILF2_CASES = [
    (40, 30, {"W": (1, 1.0), "E": (0, 0.0)}, 0),
    (67, 45, {"W": (1, -1.0), "S": (1, -1.0)}, 1),
    (130, 5, {"W": (1, 0.7), "E": (1, -0.4), "S": (1, 0.2), "N": (1, -0.9)}, 0),
    (3, 3, {}, 1),
]


@pytest.mark.parametrize("case", range(len(ILF2_CASES)))
@pytest.mark.parametrize("init", ["uniform", "random"])
def test_ilfbm_d2q9_parity(gpu, orc, case, init):
    nx, ny, walls, bb_mode = ILF2_CASES[case]
    tau, ste, steps, maxit = 0.8, 0.3, 60, 400
    th0 = (np.full((ny, nx), -0.3) if init == "uniform"
           else workloads.random_field((ny, nx), -0.5, 0.3, seed=nx * 3 + ny))
    S = gpu.Stefan(_abi.LBM_D2Q9, nx, ny, tau, 0.01, ste, _abi.LBM_FP64, walls, newton_tol=1e-12,
                   newton_max_iter=maxit, bb_mode=bb_mode)
    S.set_method("ILFBM")
    S.set_ic(th0)
    S.step(steps)
    th, l, H = S.fields()
    st = S.stats()
    S.close()
    P = orc.Problem(2, nx, ny, tau=tau, delta=0.01, ste=ste, walls=walls, bb_mode=bb_mode)
    _, lo, tho, failed, mx = P.ilfbm_run(th0, steps, tol=1e-12, maxit=maxit)
    fl_t = fl_l = 0.0
    for seed in (12345, 1, 2):
        rng = np.random.Generator(np.random.PCG64(seed))
        pert = th0 + np.spacing(th0) * rng.choice([-1, 0, 1], size=th0.shape)
        _, lp_, thp, _, _ = P.ilfbm_run(pert, steps, tol=1e-12, maxit=maxit)
        fl_t = max(fl_t, np.max(np.abs(thp - tho)))
        fl_l = max(fl_l, np.max(np.abs(lp_ - lo)))
    assert failed == 0 and st["error"] == 0
    assert np.max(np.abs(th - tho)) <= max(1e-12 * np.max(np.abs(tho)), 10 * fl_t)
    assert np.max(np.abs(l - lo)) <= max(1e-10, 10 * fl_l)
    assert 1 <= st["newton_max_iter"] <= mx


def test_ilfbm_d2q9_closed_box_conserves_energy(gpu):
    nx, ny, ste = 50, 40, 0.5
    S = gpu.Stefan(_abi.LBM_D2Q9, nx, ny, 0.8, 0.01, ste, _abi.LBM_FP64, {}, newton_tol=1e-13, newton_max_iter=400,
                   bb_mode=1)
    S.set_method("ILFBM")
    S.set_ic(workloads.random_field((ny, nx), -0.6, 0.6, seed=4))
    e0 = S.stats()["energy"]
    S.step(40)
    st = S.stats()
    assert st["error"] == 0
    assert abs(st["energy"] - e0) <= 40 * nx * ny * 1e-13 / ste + 1e-11 * abs(e0)


def test_ilfbm_d2q5_inner_loop_fails_as_in_the_oracle(gpu, orc):
    # the D2Q5 cavity: the inner loop reaches its limit in the oracle (the
    # checkerboard factor of the iteration is 4/3) and the GPU reports it
    c = workloads.cavity_2d(n=32, steps=20, precision=workloads.FP64)
    P = orc.Problem(3, c.nx, c.ny, tau=c.tau, delta=c.delta, ste=c.ste, walls=c.walls)
    *_, failed, _ = P.ilfbm_run(c.theta0(), c.steps, maxit=100)
    assert failed > 0
    S = gpu.Stefan(_abi.LBM_D2Q5, c.nx, c.ny, c.tau, c.delta, c.ste, _abi.LBM_FP64, c.walls, newton_max_iter=100)
    S.set_method("ILFBM")
    S.set_ic(c.theta0())
    S.step(c.steps)
    with pytest.raises(_abi.LBMError) as e:
        S.sync()
    assert e.value.status == _abi.LBM_ERR_NEWTON
    S.close()


def test_ilfbm_2d_argument_errors(gpu):
    S = gpu.Stefan(_abi.LBM_D2Q9, 32, 32, 0.8, 0.01, 0.1, _abi.LBM_FP32, {})
    with pytest.raises(_abi.LBMError) as e:
        S.set_method("ILFBM")
    assert e.value.status == _abi.LBM_ERR_ARG
    S.close()
    S = gpu.Stefan(_abi.LBM_D2Q5, 32, 32, 0.8, 0.01, 0.1, _abi.LBM_FP64, {}, bb_mode=2)
    with pytest.raises(_abi.LBMError) as e:
        S.set_method("ILFBM")
    assert e.value.status == _abi.LBM_ERR_ARG
    S.close()
    # the state grows by the liquid-fraction plane
    S = gpu.Stefan(_abi.LBM_D2Q9, 32, 32, 0.8, 0.01, 0.1, _abi.LBM_FP64, {})
    b0 = S.state_bytes
    S.set_method("ILFBM")
    import ctypes
    sb, rs = ctypes.c_size_t(), ctypes.c_int()
    _abi.check(S.lib.lbm_stefan_layout(S.h, ctypes.byref(sb), ctypes.byref(rs)))
    assert sb.value == (b0 - 256) // 9 * 10 + 256   # nine planes and a 256-byte tail, then ten
    S.set_ic(np.full((32, 32), -0.2))
    with pytest.raises(_abi.LBMError) as e:
        S.step_timed(2)
    assert e.value.status == _abi.LBM_ERR_STATE
    S.close()
