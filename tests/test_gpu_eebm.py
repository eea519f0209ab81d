"""The explicit enthalpy based method (EEBM, Algorithm 2) on the GPU against
the oracle's EEBM (``oracle.Problem.eebm_run``): D2Q9, D1Q3 and D2Q5 (with
the Eq. 17 closure on D2Q5).

EEBM is the paper's comparison scheme: its populations carry the enthalpy,
so in the FP32 form they hold the latent part 1/Ste as well, and theta =
Theta(H) keeps only the FP32 resolution of H (about 1e-6 at Ste = 0.1); the
FP32 tolerance below is set by that, not by the IREBM form's 2e-5.
"""
import numpy as np
import pytest

from paper_2505_13097_gb300 import _abi, workloads

pytestmark = pytest.mark.gpu

SHAPES = [(97, 70), (130, 33), (64, 2), (515, 37), (400, 11)]   # the last two: interior strips
WALLS = [
    {"W": (1, 1.0), "S": (1, -0.5), "E": (0, 0.0), "N": (0, 0.0)},
    {"W": (1, 0.8), "E": (1, 0.0), "S": (0, 0.0), "N": (1, 1.5)},
]


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_13097_gb300 import solver
    return solver


def run_pair(gpu, orc, nx, ny, walls, precision, steps, bb_mode=0, tau=0.9, ste=0.1):
    th0 = workloads.random_field((ny, nx), -0.6, 0.4, seed=nx * 7 + ny)
    S = gpu.Stefan(2, nx, ny, tau, 0.01, ste, precision, walls, bb_mode=bb_mode)
    S.set_method("EEBM")
    S.set_ic(th0)
    S.step(steps)
    th, ph, H = S.fields()
    st = S.stats()
    S.close()
    P = orc.Problem(2, nx, ny, tau=tau, delta=0.01, ste=ste, walls=walls, bb_mode=bb_mode)
    f, tho = P.eebm_run(th0, steps)
    return th, H, tho, P.eebm_fields(f)[1], st


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("wi", [0, 1])
@pytest.mark.parametrize("bb_mode", [0, 1])
def test_eebm_fp64_parity(gpu, orc, shape, wi, bb_mode):
    th, H, tho, Ho, st = run_pair(gpu, orc, *shape, WALLS[wi], workloads.FP64, 150, bb_mode)
    assert np.max(np.abs(th - tho)) <= 1e-12 * np.max(np.abs(tho))
    assert np.max(np.abs(H - Ho)) <= 1e-12 * np.max(np.abs(Ho))
    assert st["error"] == 0 and st["newton_nodes"] == 0


@pytest.mark.parametrize("shape", SHAPES)
def test_eebm_fp32_parity(gpu, orc, shape):
    # FP32 populations hold H, latent part 1/Ste = 10 included: a step rounds H
    # (nine stored populations and their sum) by at most 10 half-ulps of
    # max|H|, and Theta is 1-Lipschitz, so after T steps |dtheta| <= T * 5 ulp(max H)
    steps = 150
    th, H, tho, Ho, st = run_pair(gpu, orc, *shape, WALLS[0], workloads.FP32, steps)
    bound = steps * 5 * np.spacing(np.float32(np.max(np.abs(Ho))))
    assert np.max(np.abs(th - tho)) <= bound
    assert st["error"] == 0


def test_eebm_conserves_enthalpy_gpu(gpu):
    # link-wise bounce-back on all walls: the sum of H (the energy statistic) is invariant
    nx, ny = 120, 90
    S = gpu.Stefan(2, nx, ny, 0.8, 0.01, 0.2, workloads.FP64, {}, bb_mode=1)
    S.set_method("EEBM")
    S.set_ic(workloads.random_field((ny, nx), -1.0, 1.0, seed=12))
    e0 = S.stats()["energy"]
    S.step(100)
    st = S.stats()
    assert abs(st["energy"] - e0) <= 1e-11 * abs(e0)
    assert st["imbalance_max"] <= 1e-10


def test_eebm_melting_front(gpu, orc):
    # the 2D melting workload at 300^2 with EEBM: the same front as the oracle's EEBM
    from oracle.front import front_position
    c = workloads.melt_2d(n=300, steps=400, precision=workloads.FP64)
    S = gpu.Stefan.from_case(c)
    S.set_method("EEBM")
    S.set_ic(c.theta0())
    S.step(c.steps)
    fz = S.front_position("W")[0]
    th = S.theta()
    S.close()
    P = orc.Problem(2, c.nx, c.ny, tau=c.tau, delta=c.delta, ste=c.ste, walls=c.walls)
    _, tho = P.eebm_run(c.theta0(), c.steps)
    assert np.max(np.abs(th - tho)) <= 1e-12
    assert abs(fz - front_position(tho, c.delta, 0)[0]) <= 1e-9


def test_eebm_argument_errors(gpu):
    S = gpu.Stefan(2, 64, 32, 1.0, 0.01, 0.1, workloads.FP64, {})
    with pytest.raises(_abi.LBMError) as e:
        S.set_method(7)
    assert e.value.status == _abi.LBM_ERR_ARG
    S.set_method("EEBM")
    S.set_ic(np.zeros((32, 64)))
    planes = S.new_theta_planes(2)
    a, b = S.new_state_buffer(), S.new_state_buffer()
    with pytest.raises(_abi.LBMError) as e:
        S.adjoint_step(planes[0], planes[1], a, b)
    assert e.value.status == _abi.LBM_ERR_STATE
    S.close()


# ---------------------------------------------------------------- D1Q3 and D2Q5
@pytest.mark.parametrize("n", [2, 64, 513, 5000])
@pytest.mark.parametrize("precision", [workloads.FP64, workloads.FP32])
def test_eebm_d1q3_parity(gpu, orc, n, precision):
    # 5,000 nodes: beyond one block's shared memory, the per-step kernel
    walls = {"W": (1, 1.0), "E": (1, -0.5)}
    th0 = workloads.random_field((1, n), -0.6, 0.4, seed=n)
    S = gpu.Stefan(1, n, 1, 0.62, 0.01, 0.2857, precision, walls)
    S.set_method("EEBM")
    S.set_ic(th0)
    S.step(300)
    th, _, H = S.fields()
    st = S.stats()
    S.close()
    P = orc.Problem(1, n, 1, tau=0.62, delta=0.01, ste=0.2857, walls=walls)
    f, tho = P.eebm_run(th0, 300)
    Ho = P.eebm_fields(f)[1]
    if precision == workloads.FP64:
        assert np.max(np.abs(th - tho)) <= 1e-12 * np.max(np.abs(tho))
    else:
        assert np.max(np.abs(th - tho)) <= 300 * 3 * np.spacing(np.float32(np.max(np.abs(Ho))))
    # FP32: every stored population rounds each step, a random walk far below 1e-5 of sum |H|
    rel = 1e-9 if precision == workloads.FP64 else 1e-5
    assert abs(st["energy"] - Ho.sum()) <= rel * np.abs(Ho).sum()
    assert st["error"] == 0


D5_SHAPES = [(67, 45), (130, 5), (3, 3), (257, 19)]


@pytest.mark.parametrize("shape", D5_SHAPES)
@pytest.mark.parametrize("wi", [0, 1])
@pytest.mark.parametrize("bb_mode", [0, 1, 2])
def test_eebm_d2q5_fp64_parity(gpu, orc, shape, wi, bb_mode):
    nx, ny = shape
    th0 = workloads.random_field((ny, nx), -0.6, 0.4, seed=nx * 5 + ny)
    S = gpu.Stefan(3, nx, ny, 0.9, 0.01, 0.1, workloads.FP64, WALLS[wi], bb_mode=bb_mode)
    S.set_method("EEBM")
    S.set_ic(th0)
    S.step(150)
    th, _, H = S.fields()
    S.close()
    P = orc.Problem(3, nx, ny, tau=0.9, delta=0.01, ste=0.1, walls=WALLS[wi], bb_mode=bb_mode)
    f, tho = P.eebm_run(th0, 150)
    assert np.max(np.abs(th - tho)) <= 1e-12 * np.max(np.abs(tho))
    assert np.max(np.abs(H - P.eebm_fields(f)[1])) <= 1e-12 * np.max(np.abs(P.eebm_fields(f)[1]))


@pytest.mark.parametrize("shape", D5_SHAPES)
def test_eebm_d2q5_fp32_parity(gpu, orc, shape):
    # FP32 populations carry H: the bound of the D2Q9 FP32 case with five populations
    nx, ny = shape
    steps = 150
    th0 = workloads.random_field((ny, nx), -0.6, 0.4, seed=nx * 5 + ny)
    S = gpu.Stefan(3, nx, ny, 0.9, 0.01, 0.1, workloads.FP32, WALLS[0], bb_mode=2)
    S.set_method("EEBM")
    S.set_ic(th0)
    S.step(steps)
    th = S.theta()
    S.close()
    P = orc.Problem(3, nx, ny, tau=0.9, delta=0.01, ste=0.1, walls=WALLS[0], bb_mode=2)
    f, tho = P.eebm_run(th0, steps)
    bound = steps * 5 * np.spacing(np.float32(np.max(np.abs(P.eebm_fields(f)[1]))))
    assert np.max(np.abs(th - tho)) <= bound


def test_eebm_d2q5_cavity(gpu, orc):
    # the paper's 2D case on D2Q5 with EEBM (its timing table's comparison)
    c = workloads.cavity_2d(n=200, steps=300, precision=workloads.FP64)
    S = gpu.Stefan.from_case(c)
    S.set_method("EEBM")
    S.set_ic(c.theta0())
    S.step(c.steps)
    th = S.theta()
    S.close()
    P = orc.Problem(3, c.nx, c.ny, tau=c.tau, delta=c.delta, ste=c.ste, walls=c.walls, bb_mode=2)
    _, tho = P.eebm_run(c.theta0(), c.steps)
    assert np.max(np.abs(th - tho)) <= 1e-12 * np.max(np.abs(tho))
