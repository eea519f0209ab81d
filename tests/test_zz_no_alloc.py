"""The no-allocation D2Q9 step (lbm_stefan_step_d2q9_noalloc) against the
regular step (lbm_stefan_step).

The no-allocation entry point serves callers that cannot call cudaMalloc when
they step (a memory budget or allocator they do not own, real-time loops that
must not block on an allocation); its scratch lives in a fixed device array in
the library.  Two calls in a row, through the C ABI, must give the populations
of one and two regular steps, within the FP32-form tolerance of the parity
tests.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2505_13097_gb300 import workloads

pytestmark = pytest.mark.gpu

TOL32_T = 2e-5


def test_noalloc_step_matches_regular_step():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_13097_gb300 import _abi, solver

    c = workloads.melt_2d(n=300, steps=0).scaled(ny=200)
    stream = torch.cuda.Stream()
    S = solver.Stefan.from_case(c, stream=stream)
    S.set_ic(c.theta0())
    S.step(40)                       # a state with a front and Newton nodes
    s0 = S.new_state_buffer()
    S.get_state(s0)
    S.step(1)
    ref1 = S.new_state_buffer()
    S.get_state(ref1)
    S.step(1)
    ref2 = S.new_state_buffer()
    S.get_state(ref2)
    S.sync()
    S.close()

    lib = _abi.load()
    p = _abi.lbm_stefan_params(2, c.nx, c.ny, c.tau, c.delta, c.ste, c.precision, 1e-14, 60, 0)
    kinds = (ctypes.c_int * 4)(*[c.walls.get(w, (0, 0.0))[0] for w in "WESN"])
    thetas = (ctypes.c_double * 4)(*[c.walls.get(w, (0, 0.0))[1] for w in "WESN"])
    out1 = torch.zeros_like(s0)
    out2 = torch.zeros_like(s0)
    h = ctypes.c_void_p(stream.cuda_stream)
    for src, dst in ((s0, out1), (out1, out2)):
        st = lib.lbm_stefan_step_d2q9_noalloc(ctypes.byref(p), kinds, thetas, ctypes.c_void_p(src.data_ptr()),
                                              ctypes.c_void_p(dst.data_ptr()), h)
        assert st == _abi.LBM_OK, lib.lbm_stefan_last_error()

    def theta(buf):
        # theta = sum over the 9 planes of the interior rows and columns
        f = buf.view(torch.float32).reshape(9, c.ny + 2, -1)[:, 1:-1, :c.nx].double()
        return f.sum(0).cpu().numpy()

    for got, ref in ((out1, ref1), (out2, ref2)):
        tg, tr = theta(got), theta(ref)
        assert np.max(np.abs(tg - tr)) / np.max(np.abs(tr)) < TOL32_T
        fg = got.view(torch.float32).reshape(9, c.ny + 2, -1)[:, 1:-1, :c.nx]
        fr = ref.view(torch.float32).reshape(9, c.ny + 2, -1)[:, 1:-1, :c.nx]
        assert float((fg - fr).abs().max()) <= TOL32_T * float(fr.abs().max())


def test_noalloc_rejects_oversize_problem():
    from paper_2505_13097_gb300 import _abi
    lib = _abi.load()
    p = _abi.lbm_stefan_params(2, 1024, 1024, 1.0, 0.01, 0.1, 1, 1e-14, 60, 0)
    kinds = (ctypes.c_int * 4)(0, 0, 0, 0)
    thetas = (ctypes.c_double * 4)(0, 0, 0, 0)
    st = lib.lbm_stefan_step_d2q9_noalloc(ctypes.byref(p), kinds, thetas, ctypes.c_void_p(16), ctypes.c_void_p(32), None)
    assert st == _abi.LBM_ERR_ARG
    assert b"exceed the maximum" in lib.lbm_stefan_last_error()
