"""Failure detection of the bounded device waits, without a GPU fault.

The TMA row-pipeline kernel (the FP32 D2Q9 step of batches) waits for row
loads that its blocks issued themselves (TMA copies completing on
mbarriers), each wait bounded in time.  While the test hook
lbm_stefan_set_wait_test is on, a single FP32 D2Q9 handle steps with that
kernel, and its first block skips one row load, so that the waits for it run
out after a short limit (5 ms here): the block records LBM_ERR_TIMEOUT,
waits (bounded) for the copies it still has in flight and stops; the launch
ends normally and the next synchronizing call returns the status.  Nothing
faults or hangs, and a fresh handle on the same device then steps and
matches the FP64 oracle.
"""
import numpy as np
import pytest

from paper_2505_13097_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_13097_gb300 import solver
    return solver


def small_case():
    return workloads.melt_2d(n=256, steps=30).scaled(ny=96)


@pytest.mark.parametrize("load", [0, 1, 2])
def test_withheld_row_load_times_out(gpu, orc, load):
    from paper_2505_13097_gb300 import _abi
    c = small_case()
    S = gpu.Stefan.from_case(c)
    S.set_wait_test(wait_limit_s=0.005, withhold_load=load)
    S.set_ic(c.theta0())
    S.step(1)
    with pytest.raises(_abi.LBMError) as ei:
        S.sync()
    assert ei.value.status == _abi.LBM_ERR_TIMEOUT
    S.close()

    # the context is intact: a fresh handle steps and matches the oracle
    S = gpu.Stefan.from_case(c)
    S.set_ic(c.theta0())
    S.step(c.steps)
    th = S.theta()
    st = S.stats()
    S.close()
    assert st["error"] == 0
    P = orc.Problem(c.lattice, c.nx, c.ny, tau=c.tau, delta=c.delta, ste=c.ste, walls=c.walls)
    _, ref = P.run(c.theta0(), c.steps)
    assert np.max(np.abs(th - ref)) / np.max(np.abs(ref)) < 2e-5


def test_hook_off_again_steps_normally(gpu, orc):
    """The hook switched back off: the same handle's next steps are normal."""
    c = small_case()
    S = gpu.Stefan.from_case(c)
    S.set_wait_test(wait_limit_s=0.005, withhold_load=-1)
    S.set_ic(c.theta0())
    S.step(c.steps)
    th = S.theta()
    S.close()
    P = orc.Problem(c.lattice, c.nx, c.ny, tau=c.tau, delta=c.delta, ste=c.ste, walls=c.walls)
    _, ref = P.run(c.theta0(), c.steps)
    assert np.max(np.abs(th - ref)) / np.max(np.abs(ref)) < 2e-5


def test_hook_rejects_bad_values(gpu):
    from paper_2505_13097_gb300 import _abi
    S = gpu.Stefan.from_case(small_case())
    for lim, load in ((0.0, -1), (-1.0, -1), (0.01, -2), (0.01, 3), (61.0, 0)):
        with pytest.raises(_abi.LBMError) as ei:
            S.set_wait_test(lim, load)
        assert ei.value.status == _abi.LBM_ERR_ARG
    S.close()
