"""The no-allocation D2Q9 step (lbm_stefan_step_d2q9_noalloc) against the
regular step (lbm_stefan_step) and the FP64 oracle.

The no-allocation entry point serves callers that cannot call cudaMalloc when
they step (a memory budget or allocator they do not own, real-time loops that
must not block on an allocation); its scratch lives in a fixed device array in
the library.  Two calls in a row, through the C ABI, must give the populations
of one and two regular steps: within the FP32-form tolerance of the parity
tests in FP32 (the regular FP32 step runs another kernel), bit for bit in
FP64 (the same kernels).  One FP64 call must match the oracle's step, and a
Newton solve that hits its iteration limit must be reported.  This file is
collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2505_13097_gb300 import workloads

pytestmark = pytest.mark.gpu

TOL32_T = 2e-5
TOL64 = 1e-12

WALL_SETS = [
    {"W": (1, 1.0), "E": (0, 0.0), "S": (0, 0.0), "N": (0, 0.0)},
    {"W": (1, -1.0), "S": (1, -1.0), "E": (0, 0.0), "N": (0, 0.0)},
    {"W": (1, 0.7), "E": (1, -0.4), "S": (1, 0.2), "N": (1, -0.9)},
    {"W": (0, 0.0), "E": (0, 0.0), "S": (0, 0.0), "N": (0, 0.0)},
]


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_13097_gb300 import _abi, solver
    return torch, _abi, solver


def noalloc_call(_abi, c, src, dst, stream, bb_mode=0, maxit=60):
    lib = _abi.load()
    p = _abi.lbm_stefan_params(2, c.nx, c.ny, c.tau, c.delta, c.ste, c.precision, 1e-14, maxit, bb_mode)
    kinds = (ctypes.c_int * 4)(*[c.walls.get(w, (0, 0.0))[0] for w in "WESN"])
    thetas = (ctypes.c_double * 4)(*[c.walls.get(w, (0, 0.0))[1] for w in "WESN"])
    st = lib.lbm_stefan_step_d2q9_noalloc(ctypes.byref(p), kinds, thetas, ctypes.c_void_p(src.data_ptr()),
                                          ctypes.c_void_p(dst.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    return st, lib.lbm_stefan_last_error()


def planes(torch, c, buf):
    """The nine planes of a state buffer (the last 256 bytes are its tail)."""
    dt = torch.float32 if c.precision == workloads.FP32 else torch.float64
    return buf[:buf.numel() - 256].view(dt).reshape(9, c.ny + 2, -1)[:, 1:-1, :c.nx]


def regular_states(solver, c, stream, pre, bb_mode=0):
    """State after `pre` steps of a regular handle, and after one and two more."""
    S = solver.Stefan.from_case(c, stream=stream, bb_mode=bb_mode)
    S.set_ic(c.theta0())
    S.step(pre)
    out = []
    for k in range(3):
        if k:
            S.step(1)
        b = S.new_state_buffer()
        S.get_state(b)
        out.append(b)
    S.sync()
    S.close()
    return out


@pytest.mark.parametrize("wi", [0, 1])
def test_noalloc_fp32_matches_regular_step(env, wi):
    torch, _abi, solver = env
    c = workloads.melt_2d(n=300, steps=0).scaled(ny=200, walls=WALL_SETS[wi])
    stream = torch.cuda.Stream()
    s0, ref1, ref2 = regular_states(solver, c, stream, 40)   # a state with a front and Newton nodes
    out1, out2 = torch.zeros_like(s0), torch.zeros_like(s0)
    for src, dst in ((s0, out1), (out1, out2)):
        st, msg = noalloc_call(_abi, c, src, dst, stream)
        assert st == _abi.LBM_OK, msg
    for got, ref in ((out1, ref1), (out2, ref2)):
        fg, fr = planes(torch, c, got), planes(torch, c, ref)
        tg, tr = fg.double().sum(0).cpu().numpy(), fr.double().sum(0).cpu().numpy()
        assert np.max(np.abs(tg - tr)) / np.max(np.abs(tr)) < TOL32_T
        assert float((fg - fr).abs().max()) <= TOL32_T * float(fr.abs().max())


@pytest.mark.parametrize("wi", range(4))
@pytest.mark.parametrize("bb_mode", [0, 1])
def test_noalloc_fp64_matches_regular_step_bitwise(env, wi, bb_mode):
    torch, _abi, solver = env
    c = workloads.Case("t", 2, 130, 70, 0.84, 0.02, 0.07, WALL_SETS[wi], 0, workloads.FP64)
    c.theta_init, c.noise, c.seed = 0.0, 0.3, 7   # a mushy random field: most nodes run Newton
    stream = torch.cuda.Stream()
    s0, ref1, ref2 = regular_states(solver, c, stream, 5, bb_mode=bb_mode)
    out1, out2 = torch.zeros_like(s0), torch.zeros_like(s0)
    for src, dst in ((s0, out1), (out1, out2)):
        st, msg = noalloc_call(_abi, c, src, dst, stream, bb_mode=bb_mode)
        assert st == _abi.LBM_OK, msg
    for got, ref in ((out1, ref1), (out2, ref2)):
        assert torch.equal(planes(torch, c, got), planes(torch, c, ref))


def test_noalloc_fp64_one_step_matches_oracle(env, orc):
    torch, _abi, solver = env
    c = workloads.Case("t", 2, 67, 45, 0.84, 0.02, 0.07, WALL_SETS[2], 0, workloads.FP64)
    c.theta_init, c.noise, c.seed = 0.0, 0.3, 11
    stream = torch.cuda.Stream()
    s0 = regular_states(solver, c, stream, 0)[0]   # the initial state of set_ic
    out = torch.zeros_like(s0)
    st, msg = noalloc_call(_abi, c, s0, out, stream)
    assert st == _abi.LBM_OK, msg
    th = planes(torch, c, out).sum(0).cpu().numpy()
    P = orc.Problem(2, c.nx, c.ny, tau=c.tau, delta=c.delta, ste=c.ste, walls=c.walls)
    _, ref = P.run(c.theta0(), 1)
    assert np.max(np.abs(th - ref)) / np.max(np.abs(ref)) < TOL64


def test_noalloc_reports_newton_limit(env):
    """newton_max_iter = 1 on a mushy field: every Newton node needs more, and
    the call returns LBM_ERR_NEWTON; a normal call afterwards succeeds (each
    call clears the error flag)."""
    torch, _abi, solver = env
    c = workloads.Case("t", 2, 64, 64, 1.0, 0.01, 0.1, WALL_SETS[3], 0, workloads.FP64)
    c.theta_init, c.noise, c.seed = 0.0, 0.02, 3
    stream = torch.cuda.Stream()
    s0 = regular_states(solver, c, stream, 0)[0]
    out = torch.zeros_like(s0)
    st, msg = noalloc_call(_abi, c, s0, out, stream, maxit=1)
    assert st == _abi.LBM_ERR_NEWTON, msg
    st, msg = noalloc_call(_abi, c, s0, out, stream)
    assert st == _abi.LBM_OK, msg


def test_noalloc_rejects_oversize_problem(env):
    torch, _abi, solver = env
    lib = _abi.load()
    p = _abi.lbm_stefan_params(2, 1024, 1024, 1.0, 0.01, 0.1, 1, 1e-14, 60, 0)
    kinds = (ctypes.c_int * 4)(0, 0, 0, 0)
    thetas = (ctypes.c_double * 4)(0, 0, 0, 0)
    st = lib.lbm_stefan_step_d2q9_noalloc(ctypes.byref(p), kinds, thetas, ctypes.c_void_p(16), ctypes.c_void_p(32), None)
    assert st == _abi.LBM_ERR_ARG
    assert b"exceed the maximum" in lib.lbm_stefan_last_error()
