"""D2Q5 step (Sec. 3.2 lattice, Sec. 4.2 closures) on the GPU through the C ABI
against the FP64 oracle on the same seeded inputs.

Tolerances as for D2Q9: FP64 1e-12 relative on theta (or ten times the
problem's own rounding floor where the mushy zone amplifies rounding), FP32
populations 2e-5 relative on theta and 1e-4 absolute on phi.
"""
import numpy as np
import pytest

from paper_2505_13097_gb300 import _abi, workloads

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32_T, TOL32_PHI = 2e-5, 1e-4


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_13097_gb300 import solver
    return solver


def phi(x, d):
    return 0.5 * (1.0 + np.tanh(x / d))


def rel_err(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


WALLS = [
    {"W": (1, 1.0), "E": (0, 0.0), "S": (0, 0.0), "N": (0, 0.0)},
    {"W": (1, -1.0), "S": (1, -1.0), "E": (0, 0.0), "N": (0, 0.0)},
    {"W": (1, 0.7), "E": (1, -0.4), "S": (1, 0.2), "N": (1, -0.9)},
    {"W": (0, 0.0), "E": (0, 0.0), "S": (0, 0.0), "N": (0, 0.0)},
]
# several 128-column segments and 16-row tiles with ragged tails, the smallest
# lattice, a thin strip and a tall one
SHAPES = [(64, 64), (67, 45), (130, 5), (3, 3), (3, 70), (257, 19), (300, 40)]


def run_pair(gpu, orc, nx, ny, walls, precision, steps, bb_mode, tau=0.8, ste=0.2, delta=0.05, theta0=None):
    th0 = workloads.random_field((ny, nx), -0.5, 0.5, seed=nx * 131 + ny) if theta0 is None else theta0
    S = gpu.Stefan(_abi.LBM_D2Q5, nx, ny, tau, delta, ste, precision, walls, bb_mode=bb_mode)
    S.set_ic(th0)
    S.step(steps)
    th, ph, _ = S.fields()
    st = S.stats()
    S.close()
    P = orc.Problem(3, nx, ny, tau=tau, delta=delta, ste=ste, walls=walls, bb_mode=bb_mode)
    _, tho = P.run(th0, steps)
    return th, ph, tho, st


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("wi", range(4))
@pytest.mark.parametrize("bb_mode", [0, 1, 2])
def test_d2q5_fp64_parity(gpu, orc, shape, wi, bb_mode):
    th, _, tho, st = run_pair(gpu, orc, *shape, WALLS[wi], _abi.LBM_FP64, 60, bb_mode)
    assert rel_err(th, tho) <= TOL64, rel_err(th, tho)
    assert st["error"] == 0


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("wi", [0, 1, 2])
@pytest.mark.parametrize("bb_mode", [0, 2])
def test_d2q5_fp32_parity(gpu, orc, shape, wi, bb_mode):
    th, ph, tho, st = run_pair(gpu, orc, *shape, WALLS[wi], _abi.LBM_FP32, 60, bb_mode)
    assert rel_err(th, tho) <= TOL32_T, rel_err(th, tho)
    assert np.max(np.abs(ph - phi(tho, 0.05))) <= TOL32_PHI
    assert st["error"] == 0


@pytest.mark.parametrize("precision", [_abi.LBM_FP64, _abi.LBM_FP32])
def test_d2q5_cavity_parity(gpu, orc, precision):
    # the paper's 2D case (Sec. 6.2) at 256 x 256: liquid at theta = 1 frozen from
    # two walls at -2, Eq. (17) on the symmetry lines, tau 0.84, delta 0.01
    c = workloads.cavity_2d(n=256, steps=400, precision=precision)
    S = gpu.Stefan.from_case(c)
    S.set_ic(c.theta0())
    S.step(c.steps)
    th, ph, _ = S.fields()
    st = S.stats()
    S.close()
    P = orc.Problem(3, c.nx, c.ny, tau=c.tau, delta=c.delta, ste=c.ste, walls=c.walls, bb_mode=2)
    _, tho = P.run(c.theta0(), c.steps)
    if precision == _abi.LBM_FP64:
        assert rel_err(th, tho) <= TOL64
    else:
        assert rel_err(th, tho) <= TOL32_T
        assert np.max(np.abs(ph - phi(tho, c.delta))) <= TOL32_PHI
    assert st["newton_nodes"] > 0 and st["error"] == 0
    # the symmetry lines keep theta equal to the next line inwards (Eq. 17), away
    # from the Dirichlet corners
    assert np.max(np.abs(th[-1, 1:] - th[-2, 1:])) <= 1e-5
    assert np.max(np.abs(th[1:, -1] - th[1:, -2])) <= 1e-5


@pytest.mark.parametrize("precision", [_abi.LBM_FP64, _abi.LBM_FP32])
def test_d2q5_closed_box_conserves_energy(gpu, precision):
    # link-wise bounce-back on every wall: E = sum theta + phi(theta)/Ste is invariant
    nx, ny = 200, 150
    S = gpu.Stefan(_abi.LBM_D2Q5, nx, ny, 0.8, 0.02, 0.2, precision, {}, bb_mode=1)
    S.set_ic(workloads.random_field((ny, nx), -1.0, 1.0, seed=7))
    e0 = S.stats()["energy"]
    S.step(100)
    st = S.stats()
    tol = 1e-11 if precision == _abi.LBM_FP64 else 1e-5
    assert abs(st["energy"] - e0) <= tol * abs(e0)
    assert st["newton_nodes"] > 0
    S.close()


@pytest.mark.parametrize("bb_mode", [0, 2])
def test_d2q5_energy_balance_with_walls(gpu, orc, bb_mode):
    # Dirichlet walls with mirror bounce-back or Eq. (17): the energy changes by
    # the boundary flux only, and both match the oracle's per-step diagnostics
    nx, ny, ste = 190, 77, 0.1
    th0 = workloads.random_field((ny, nx), -0.5, 0.5, seed=8)
    S = gpu.Stefan(_abi.LBM_D2Q5, nx, ny, 0.9, 0.02, ste, _abi.LBM_FP64, WALLS[1], bb_mode=bb_mode)
    S.set_ic(th0)
    P = orc.Problem(3, nx, ny, tau=0.9, delta=0.02, ste=ste, walls=WALLS[1], bb_mode=bb_mode)
    f = P.init(th0)
    for _ in range(20):
        S.step(1)
        f, d = P.step(f, detail=True)
        st = S.stats()
        assert abs(st["energy"] - d["energy_after"]) < 1e-10 * abs(d["energy_after"])
        assert abs(st["flux"] - d["flux"]) < 1e-10 * max(1.0, abs(d["flux"]))
    # each node's theta' + phi/Ste carries a few ulps of (|theta| + 1/Ste) per step
    assert st["imbalance_max"] <= 8 * nx * ny * 2.2e-16 * (1 + 1 / ste)
    S.close()


def test_d2q5_step_record_and_timed(gpu):
    import torch
    nx, ny = 150, 40
    th0 = workloads.random_field((ny, nx), -0.5, 0.5, seed=9)
    A = gpu.Stefan(_abi.LBM_D2Q5, nx, ny, 0.8, 0.05, 0.2, _abi.LBM_FP32, WALLS[0], bb_mode=2)
    B = gpu.Stefan(_abi.LBM_D2Q5, nx, ny, 0.8, 0.05, 0.2, _abi.LBM_FP32, WALLS[0], bb_mode=2)
    C = gpu.Stefan(_abi.LBM_D2Q5, nx, ny, 0.8, 0.05, 0.2, _abi.LBM_FP32, WALLS[0], bb_mode=2)
    for S in (A, B, C):
        S.set_ic(th0)
    A.step(7)
    ms = B.step_timed(7)
    traj = torch.empty(7 * ny * C.row_stride, dtype=torch.float64, device="cuda")
    C.step_record(7, traj)
    ta, tb, tc = A.theta(), B.theta(), C.theta()
    rec = traj.view(7, ny, C.row_stride)[-1, :, :nx].cpu().numpy()
    for S in (A, B, C):
        S.close()
    assert np.array_equal(ta, tb) and np.array_equal(ta, tc)
    assert np.max(np.abs(rec - ta)) <= 1e-6 * np.max(np.abs(ta))
    assert ms[0] > 0 and ms[1] > 0


def test_d2q5_deterministic(gpu):
    c = workloads.cavity_2d(n=300, steps=50)
    out = []
    for _ in range(2):
        S = gpu.Stefan.from_case(c)
        S.set_ic(c.theta0())
        S.step(c.steps)
        out.append((S.theta(), S.stats()["energy"]))
        S.close()
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]


def _crop_reference(orc, case, theta0, steps, x, y):
    """Oracle value of node (x, y) after `steps` steps, from a window of radius
    steps + 2 around it (Eq. 17 reads one node further in than the streaming)."""
    r = steps + 2
    x0, x1 = max(0, x - r), min(case.nx, x + r + 1)
    y0, y1 = max(0, y - r), min(case.ny, y + r + 1)
    walls = {}
    for name, (kind, th) in case.walls.items():
        real = {"W": x0 == 0, "E": x1 == case.nx, "S": y0 == 0, "N": y1 == case.ny}[name]
        walls[name] = (kind, th) if real else (0, 0.0)
    P = orc.Problem(3, x1 - x0, y1 - y0, tau=case.tau, delta=case.delta, ste=case.ste, walls=walls,
                    bb_mode=case.bb_mode)
    _, th = P.run(theta0[y0:y1, x0:x1], steps)
    return th[y - y0, x - x0]


def test_d2q5_full_size_cavity_sampled(gpu, orc):
    """4096 x 4096 FP32 cavity in the benchmark's launch configuration: sampled
    nodes (corners, walls, segment and tile seams, random) against the oracle
    on windows around them."""
    c = workloads.cavity_2d()
    th0 = c.theta0()
    steps = 6
    S = gpu.Stefan.from_case(c)
    S.set_ic(th0)
    S.step(steps)
    th = S.theta()
    S.close()
    n = c.nx
    rng = np.random.Generator(np.random.PCG64(5))
    pts = [(0, 0), (n - 1, 0), (0, n - 1), (n - 1, n - 1), (1, 1), (n - 2, n - 2), (0, n // 2), (n - 1, n // 3),
           (n // 2, 0), (n // 3, n - 1), (127, 15), (128, 16), (129, 17), (n - 1, 2), (2, n - 1)]
    pts += [(int(rng.integers(0, n)), int(rng.integers(0, n))) for _ in range(30)]
    pts += [(int(rng.integers(0, 12)), int(rng.integers(0, n))) for _ in range(15)]   # front band
    for (x, y) in pts:
        ref = _crop_reference(orc, c, th0, steps, x, y)
        assert abs(th[y, x] - ref) <= TOL32_T * 2.0, (x, y, th[y, x], ref)


def test_d2q5_argument_errors(gpu):
    def make(**kw):
        d = dict(lattice=_abi.LBM_D2Q5, nx=32, ny=32, tau=0.8, delta=0.01, ste=0.1,
                 precision=_abi.LBM_FP64, walls={}, bb_mode=0)
        d.update(kw)
        return gpu.Stefan(d.pop("lattice"), d.pop("nx"), d.pop("ny"), d.pop("tau"), d.pop("delta"),
                          d.pop("ste"), d.pop("precision"), d.pop("walls"), bb_mode=d.pop("bb_mode"))

    for kw in (dict(nx=2), dict(ny=2), dict(lattice=_abi.LBM_D2Q9, bb_mode=2), dict(bb_mode=3)):
        with pytest.raises(_abi.LBMError) as e:
            make(**kw)
        assert e.value.status == _abi.LBM_ERR_ARG
    S = make(precision=_abi.LBM_FP32)
    with pytest.raises(_abi.LBMError) as e:
        S.set_method("ILFBM")   # ILFBM is FP64 only
    assert e.value.status == _abi.LBM_ERR_ARG
    S.close()
    S = make()
    S.set_ic(np.zeros((32, 32)))
    planes = S.new_theta_planes(2)
    a, b = S.new_state_buffer(), S.new_state_buffer()
    with pytest.raises(_abi.LBMError) as e:
        S.adjoint_step(planes[0], planes[1], a, b)
    assert e.value.status == _abi.LBM_ERR_ARG
    S.close()
