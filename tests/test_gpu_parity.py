"""GPU path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances: FP64 form 1e-12 relative on theta (norm-wise: max |d theta| /
max |theta_ref|), or ten times the problem's own FP64 rounding floor where
that is larger: the difference between the oracle and the oracle started from
theta0 moved by one ulp at random nodes.  A node leaving the mushy zone maps
errors in theta(t) into theta(t+1) with gain phi'(theta)/Ste (up to
1/(2 delta Ste)), so two correct FP64 programs drift apart by more than
1e-12 after some hundred steps when most nodes sit in the mushy zone.
FP32 form (FP32 populations, FP64 Newton): 2e-5 relative on theta and 1e-4
absolute on the liquid fraction phi.
"""
import numpy as np
import pytest

from paper_2505_13097_gb300 import workloads

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32_T, TOL32_PHI = 2e-5, 1e-4


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_13097_gb300 import solver
    return solver


def phi(x, d):
    return 0.5 * (1.0 + np.tanh(x / d))


def rel_err(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def fp64_tol(orc, case, theta0, steps, bb_mode=0):
    """max(1e-12, 10 x the relative rounding floor of this problem)."""
    P = orc.Problem(case.lattice, case.nx, case.ny, tau=case.tau, delta=case.delta, ste=case.ste,
                    walls=case.walls, bb_mode=bb_mode)
    rng = np.random.Generator(np.random.PCG64(12345))
    pert = theta0 + np.spacing(theta0) * rng.choice([-1, 0, 1], size=theta0.shape)
    _, a = P.run(theta0, steps)
    _, b = P.run(pert, steps)
    return max(TOL64, 10.0 * rel_err(b, a))


def run_pair(gpu, orc, case, steps, theta0=None, **kw):
    theta0 = case.theta0() if theta0 is None else theta0
    S = gpu.Stefan.from_case(case, **kw)
    S.set_ic(theta0)
    S.step(steps)
    th_g, ph_g, H_g = S.fields()
    st = S.stats()
    S.close()
    P = orc.Problem(case.lattice, case.nx, case.ny, tau=case.tau, delta=case.delta, ste=case.ste,
                    walls=case.walls, bb_mode=kw.get("bb_mode", 0))
    _, th_o = P.run(theta0, steps)
    return th_g, ph_g, H_g, th_o, st


D2_WALLS = [
    {"W": (1, 1.0), "E": (0, 0.0), "S": (0, 0.0), "N": (0, 0.0)},
    {"W": (1, -1.0), "S": (1, -1.0), "E": (0, 0.0), "N": (0, 0.0)},
    {"W": (1, 0.7), "E": (1, -0.4), "S": (1, 0.2), "N": (1, -0.9)},
    {"W": (0, 0.0), "E": (0, 0.0), "S": (0, 0.0), "N": (0, 0.0)},
]


@pytest.mark.parametrize("shape", [(64, 64), (67, 45), (130, 5), (2, 2), (3, 70), (257, 19)])
@pytest.mark.parametrize("wi", range(4))
@pytest.mark.parametrize("bb_mode", [0, 1])
def test_d2q9_fp64_parity(gpu, orc, shape, wi, bb_mode):
    nx, ny = shape
    c = workloads.Case("t", 2, nx, ny, 0.84, 0.02, 0.07, D2_WALLS[wi], 0, workloads.FP64)
    th0 = workloads.random_field((ny, nx), -0.3, 0.3, seed=100 + nx + ny + wi)
    th_g, ph_g, H_g, th_o, st = run_pair(gpu, orc, c, 40, th0, bb_mode=bb_mode)
    tol = fp64_tol(orc, c, th0, 40, bb_mode)
    err = rel_err(th_g, th_o)
    print("FP64 D2Q9 %dx%d walls %d bb %d: error %.2e, tolerance %.2e" % (nx, ny, wi, bb_mode, err, tol))
    assert err < tol
    # phi' <= 1/(2 delta): errors in theta carry into phi and H = theta + phi/Ste
    dth = tol * np.max(np.abs(th_o))
    assert np.max(np.abs(ph_g - phi(th_o, c.delta))) <= dth / (2 * c.delta) + 1e-15
    assert np.max(np.abs(H_g - (th_o + phi(th_o, c.delta) / c.ste))) <= dth * (1 + 1 / (2 * c.delta * c.ste)) + 1e-13


@pytest.mark.parametrize("tau,ste,delta", [(1.0, 0.1, 0.01), (0.62, 0.01, 0.005), (1.7, 1.0, 0.05)])
def test_d2q9_fp64_parity_params(gpu, orc, tau, ste, delta):
    c = workloads.Case("t", 2, 150, 70, tau, delta, ste, D2_WALLS[1], 0, workloads.FP64)
    th0 = workloads.random_field((70, 150), -0.1, 0.1, seed=7)
    th_g, _, _, th_o, st = run_pair(gpu, orc, c, 120, th0)
    tol, err = fp64_tol(orc, c, th0, 120), rel_err(th_g, th_o)
    print("FP64 D2Q9 tau %g Ste %g delta %g: error %.2e, tolerance %.2e" % (tau, ste, delta, err, tol))
    assert err < tol
    assert st["error"] == 0


@pytest.mark.parametrize("shape", [(64, 64), (131, 37), (5, 300), (2, 3)])
@pytest.mark.parametrize("wi", [0, 1, 2])
def test_d2q9_fp32_parity(gpu, orc, shape, wi):
    nx, ny = shape
    c = workloads.Case("t", 2, nx, ny, 1.0, 0.01, 0.1, D2_WALLS[wi], 0, workloads.FP32)
    th0 = -0.2 + workloads.random_field((ny, nx), -1e-3, 1e-3, seed=nx * 7 + ny + wi)
    th_g, ph_g, _, th_o, _ = run_pair(gpu, orc, c, 300, th0)
    assert rel_err(th_g, th_o) < TOL32_T
    assert np.max(np.abs(ph_g - phi(th_o, c.delta))) < TOL32_PHI


# The flat kernel takes rows 1 .. ny-2 of every 128-column strip, four
# columns per lane; a lane whose four columns hold column 0 or nx-1, or reach
# past nx, runs the scalar path with the closures; rows 0 and ny-1 go to the
# wall-row kernel.  Shapes with nx - 1 at every position in a four-column
# group, several strips, a ragged last strip and last 8-row band, and ny = 3
# (one flat row).  The initial field ramps through theta = 0 at mid-width, so
# the flat kernel hands nodes to the Newton job kernel.  On the legacy stream
# (steps launched one by one) and on a stream of the handle's own (steps
# replayed from a captured graph).
@pytest.mark.parametrize("shape", [(515, 37), (384, 3), (700, 9), (1029, 18), (6, 9), (129, 12), (132, 10), (262, 5)])
@pytest.mark.parametrize("wi", range(4))
@pytest.mark.parametrize("own_stream", [False, True], ids=["legacy_stream", "own_stream"])
def test_d2q9_fp32_flat_parity(gpu, orc, shape, wi, own_stream):
    import torch
    nx, ny = shape
    c = workloads.Case("t", 2, nx, ny, 1.0, 0.01, 0.1, D2_WALLS[wi], 0, workloads.FP32)
    ramp = 0.3 * (np.arange(nx) - nx / 2) / (nx / 2)
    th0 = ramp[None, :] + workloads.random_field((ny, nx), -1e-3, 1e-3, seed=nx + 3 * ny + wi)
    stream = torch.cuda.Stream() if own_stream else None
    th_g, ph_g, _, th_o, st = run_pair(gpu, orc, c, 200, th0, stream=stream)
    et, ep = rel_err(th_g, th_o), np.max(np.abs(ph_g - phi(th_o, c.delta)))
    print("flat FP32 %dx%d walls %d: max|d theta|/max|theta| %.2e, max|d phi| %.2e, Newton nodes %d"
          % (nx, ny, wi, et, ep, st["newton_nodes"]))
    assert et < TOL32_T
    assert ep < TOL32_PHI
    assert st["error"] == 0
    # the first step hands interior nodes to the Newton kernel
    S = gpu.Stefan.from_case(c, stream=stream)
    S.set_ic(th0)
    S.step(1)
    assert S.stats()["newton_nodes"] > 0
    S.close()


def test_d2q9_fp32_streams_bitwise_equal(gpu):
    """Steps replayed from a graph on a stream of the handle's own give the
    same bits as steps on the legacy stream."""
    import torch
    c = workloads.melt_2d(n=600, steps=60)
    th0 = c.theta0()
    th0[:, 250:350] += 0.2      # mushy nodes in the interior strips as well
    outs = []
    for stream in (None, torch.cuda.Stream()):
        S = gpu.Stefan.from_case(c, stream=stream)
        S.set_ic(th0)
        S.step(c.steps)
        outs.append((S.theta(), S.stats()))
        S.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    for k in ("energy", "flux", "newton_nodes", "newton_iters"):
        assert outs[0][1][k] == outs[1][1][k], k


def test_d2q9_fp32_parity_melt_256(gpu, orc):
    # the 2D melting workload at 256 x 256, 2,000 steps
    c = workloads.melt_2d(n=256, steps=2000)
    th_g, ph_g, _, th_o, st = run_pair(gpu, orc, c, c.steps)
    assert rel_err(th_g, th_o) < TOL32_T
    assert np.max(np.abs(ph_g - phi(th_o, c.delta))) < TOL32_PHI
    assert st["newton_nodes"] > 0 and st["error"] == 0


def test_d2q9_fp64_parity_corner_64(gpu, orc):
    for ste in workloads.CORNER_STE:
        c = workloads.corner_2d(n=64, ste=ste, steps=1500)
        th_g, _, _, th_o, st = run_pair(gpu, orc, c, c.steps)
        tol, err = fp64_tol(orc, c, c.theta0(), c.steps), rel_err(th_g, th_o)
        print("FP64 corner 64, Ste %g: error %.2e, tolerance %.2e" % (ste, err, tol))
        assert err < tol, ste


@pytest.mark.parametrize("n", [2, 3, 33, 512, 700])
@pytest.mark.parametrize("precision", [0, 1])
def test_d1q3_parity(gpu, orc, n, precision):
    c = workloads.melt_1d(n=n).scaled(precision=precision)
    th_g, ph_g, _, th_o, st = run_pair(gpu, orc, c, 3000)
    tol = fp64_tol(orc, c, c.theta0(), 3000) if precision == 0 else TOL32_T
    err = rel_err(th_g, th_o)
    print("D1Q3 n %d %s: error %.2e, tolerance %.2e" % (n, "FP64" if precision == 0 else "FP32", err, tol))
    assert err < tol
    assert st["steps"] == 3000


def test_d1q3_large_per_step_kernel(gpu, orc):
    # above the shared-memory size the per-step kernel runs instead of the fused one
    c = workloads.melt_1d(n=40000)
    th_g, _, _, th_o, _ = run_pair(gpu, orc, c, 200)
    assert rel_err(th_g, th_o) < TOL64


def test_energy_balance_and_stats(gpu, orc):
    c = workloads.corner_2d(n=48, ste=0.1)
    S = gpu.Stefan.from_case(c)
    S.set_ic(c.theta0())
    P = orc.Problem(2, 48, 48, tau=c.tau, delta=c.delta, ste=c.ste, walls=c.walls)
    f = P.init(c.theta0())
    for _ in range(25):
        S.step(1)
        f, d = P.step(f, detail=True)
        st = S.stats()
        assert abs(st["energy"] - d["energy_after"]) < 1e-10 * abs(d["energy_after"])
        assert abs(st["flux"] - d["flux"]) < 1e-10 * max(1.0, abs(d["flux"]))
        assert abs(st["imbalance"]) < 1e-9
    S.close()


def test_link_bounce_back_conserves_energy_gpu(gpu):
    c = workloads.Case("t", 2, 200, 120, 0.8, 0.02, 0.05, {}, 0, workloads.FP64)
    S = gpu.Stefan.from_case(c, bb_mode=1)
    S.set_ic(workloads.random_field((120, 200), -0.5, 0.5, seed=9))
    e0 = S.stats()["energy"]
    S.step(500)
    st = S.stats()
    assert abs(st["energy"] - e0) < 1e-11 * abs(e0)
    # per step, each node's theta' + phi/Ste carries a few ulps of (|theta| + 1/Ste)
    assert st["imbalance_max"] < 8 * 200 * 120 * 2.2e-16 * (1 + 1 / c.ste)
    S.close()


def test_deterministic(gpu):
    c = workloads.melt_2d(n=300, steps=50)
    outs = []
    for _ in range(2):
        S = gpu.Stefan.from_case(c)
        S.set_ic(c.theta0())
        S.step(c.steps)
        outs.append((S.theta(), S.stats()["energy"]))
        S.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1]


@pytest.mark.parametrize("precision", [workloads.FP32, workloads.FP64])
def test_step_timed_matches_step(gpu, precision):
    """lbm_stefan_step_timed (launch by launch, events between the kernels)
    advances the state exactly like lbm_stefan_step and reports positive times."""
    c = workloads.melt_2d(n=300, steps=40, precision=precision)
    outs = []
    for timed in (False, True):
        S = gpu.Stefan.from_case(c)
        S.set_ic(c.theta0())
        if timed:
            k0, k1 = S.step_timed(c.steps)
            assert k0 > 0.0 and k1 > 0.0
        else:
            S.step(c.steps)
        outs.append((S.theta(), S.stats()["energy"], S.stats()["steps"]))
        S.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1] and outs[0][2] == outs[1][2] == c.steps


def test_checkpoint_resume_is_exact(gpu):
    c = workloads.melt_2d(n=200, steps=0)
    S = gpu.Stefan.from_case(c)
    S.set_ic(c.theta0())
    S.step(37)
    buf = S.new_state_buffer()
    S.get_state(buf)
    S.step(63)
    ref = S.theta()
    S.set_state(buf)
    S.step(63)
    assert np.array_equal(S.theta(), ref)
    host = np.empty(S.state_bytes, dtype=np.uint8)
    S.set_state(buf)
    S.get_state(host)
    S.set_state(host)
    S.step(63)
    assert np.array_equal(S.theta(), ref)
    S.close()


def test_device_arrays_round_trip(gpu):
    import torch
    c = workloads.melt_2d(n=100, steps=0)
    S = gpu.Stefan.from_case(c)
    S.set_ic(torch.tensor(c.theta0(), device="cuda"))
    S.step(10)
    th_d, ph_d, H_d = S.fields(device=True)
    th_h, ph_h, H_h = S.fields()
    assert np.array_equal(th_d.cpu().numpy(), th_h)
    assert np.array_equal(H_d.cpu().numpy(), H_h)
    S.close()


def test_newton_limit_reports_error(gpu):
    from paper_2505_13097_gb300 import LBMError
    c = workloads.melt_2d(n=64, steps=0)
    S = gpu.Stefan.from_case(c, newton_max_iter=1)
    S.set_ic(c.theta0())
    S.step(20)
    with pytest.raises(LBMError) as ei:
        S.sync()
    assert ei.value.status == 3
    S.close()


def test_nonfinite_input_reports_error(gpu):
    from paper_2505_13097_gb300 import LBMError
    c = workloads.melt_2d(n=64, steps=0)
    th0 = c.theta0()
    th0[10, 20] = np.nan
    S = gpu.Stefan.from_case(c)
    S.set_ic(th0)
    S.step(3)
    with pytest.raises(LBMError):
        S.theta()
    S.close()


def _crop_reference(orc, case, theta0, steps, x, y):
    """Oracle value of node (x, y) after `steps` steps, from a window of radius
    steps + 1 around it; walls of the window that are not walls of the problem
    are artificial, and their influence cannot reach (x, y) in `steps` steps."""
    r = steps + 1
    x0, x1 = max(0, x - r), min(case.nx, x + r + 1)
    y0, y1 = max(0, y - r), min(case.ny, y + r + 1)
    walls = {}
    for name, (kind, th) in case.walls.items():
        real = {"W": x0 == 0, "E": x1 == case.nx, "S": y0 == 0, "N": y1 == case.ny}[name]
        walls[name] = (kind, th) if real else (0, 0.0)
    P = orc.Problem(2, x1 - x0, y1 - y0, tau=case.tau, delta=case.delta, ste=case.ste, walls=walls)
    _, th = P.run(theta0[y0:y1, x0:x1], steps)
    return th[y - y0, x - x0]


def _sample_nodes(nx, ny, rng, k=40):
    pts = [(0, 0), (nx - 1, 0), (0, ny - 1), (nx - 1, ny - 1), (0, ny // 2), (nx - 1, ny // 3),
           (nx // 2, 0), (nx // 3, ny - 1), (1, 1), (127, 5), (128, 6), (129, 300)]
    pts += [(int(rng.integers(0, nx)), int(rng.integers(0, ny))) for _ in range(k)]
    pts += [(int(rng.integers(0, 40)), int(rng.integers(0, ny))) for _ in range(k // 2)]   # front band
    return pts


def test_full_size_melt_2d_sampled(gpu, orc):
    """4096 x 4096 FP32 workload in the launch configuration of the benchmark:
    sampled nodes after 6 steps against the oracle on windows around them."""
    c = workloads.melt_2d()
    th0 = c.theta0()
    steps = 6
    S = gpu.Stefan.from_case(c)
    S.set_ic(th0)
    S.step(steps)
    th = S.theta()
    S.close()
    rng = np.random.Generator(np.random.PCG64(3))
    for (x, y) in _sample_nodes(c.nx, c.ny, rng):
        ref = _crop_reference(orc, c, th0, steps, x, y)
        assert abs(th[y, x] - ref) <= TOL32_T * 1.0, (x, y, th[y, x], ref)


def test_full_size_corner_fp64_sampled(gpu, orc):
    c = workloads.corner_2d(ste=0.01)
    th0 = c.theta0()
    steps = 5
    S = gpu.Stefan.from_case(c)
    S.set_ic(th0)
    S.step(steps)
    th = S.theta()
    S.close()
    rng = np.random.Generator(np.random.PCG64(4))
    for (x, y) in _sample_nodes(c.nx, c.ny, rng):
        ref = _crop_reference(orc, c, th0, steps, x, y)
        assert abs(th[y, x] - ref) <= TOL64 * 1.0, (x, y, th[y, x], ref)


def test_full_size_melt_2d_properties(gpu):
    """Full 4096^2 FP32 run of 2,000 steps: planar front (the front column
    varies only with the 1e-3 noise), Dirichlet column held, energy balance."""
    c = workloads.melt_2d()
    S = gpu.Stefan.from_case(c)
    S.set_ic(c.theta0())
    S.step(2000)
    th = S.theta()
    st = S.stats()
    S.close()
    assert st["error"] == 0
    assert np.max(np.abs(th[:, 0] - 1.0)) < 1e-6
    fronts = np.argmax(th < 0.0, axis=1)
    assert fronts.max() - fronts.min() <= 1
    assert abs(st["imbalance"]) < 1e-3 * max(1.0, abs(st["flux"])) + 1e-2


@pytest.mark.parametrize("lattice,precision,wall", [(2, workloads.FP32, "W"), (2, workloads.FP64, "W"),
                                                    (2, workloads.FP64, "S"), (1, workloads.FP64, "W")])
def test_front_position_matches_oracle_definition(gpu, lattice, precision, wall):
    """lbm_stefan_front_position against the oracle's definition applied to
    the GPU's own theta field (same field, so the check is the reduction)."""
    from oracle.front import front_position
    if lattice == 2:
        c = workloads.melt_2d(n=300, steps=300, precision=precision)
        if wall == "S":
            c = c.scaled(walls={"S": (1, 1.0), "W": (0, 0.0), "E": (0, 0.0), "N": (0, 0.0)})
    else:
        c = workloads.melt_1d(n=512, steps=2000)
    S = gpu.Stefan.from_case(c)
    S.set_ic(c.theta0())
    S.step(c.steps)
    th = S.theta()
    fz, it, lfz, lit = S.front_position(wall)
    S.close()
    w = "WESN".index(wall)
    ofz, oit, olfz, olit = front_position(th.reshape(c.ny, c.nx), c.delta, w)
    assert np.max(np.abs(lfz - olfz)) <= 1e-12 * max(1.0, np.max(np.abs(olfz)))
    assert np.max(np.abs(lit - olit)) <= 1e-10
    assert abs(fz - ofz) <= 1e-12 * max(1.0, abs(ofz)) and abs(it - oit) <= 1e-10
    assert 1.0 < ofz < 100.0   # a front has formed near the hot wall
