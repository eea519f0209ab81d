"""The stored oracle results that bench.py compares its legs with
(tests/golden/bench_refs.npz) are the oracle's: a sample of them is
recomputed here and must agree to rounding (the file was written by
tests/golden/make_bench_refs.py with the same oracle and inputs)."""
import os

import numpy as np
import pytest

from paper_2505_13097_gb300 import workloads

HERE = os.path.dirname(os.path.abspath(__file__))
REFS = os.path.join(HERE, "golden", "bench_refs.npz")


@pytest.fixture(scope="module")
def mk():
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_bench_refs", os.path.join(HERE, "golden", "make_bench_refs.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def close(a, b):
    return np.max(np.abs(a - b)) <= 1e-12 * max(1.0, np.max(np.abs(b)))


@pytest.mark.parametrize("name", ["melt_2d_fp64", "eebm_fp32", "d2q5_cavity_fp32", "bar_1d_ilfbm",
                                  "cavity_d2q9_eebm", "corner_ste0.01"])
def test_stored_case_is_the_oracles(orc, mk, name):
    refs = np.load(REFS)
    c, method, kw = workloads.bench_parity_cases()[name]
    th, ph = mk.run_case(c, method, kw)
    assert close(th, refs[name + "/theta"])
    assert close(ph, refs[name + "/phi"])


def test_every_leg_has_a_stored_result():
    refs = np.load(REFS)
    for name, (c, _, _) in workloads.bench_parity_cases().items():
        assert refs[name + "/theta"].shape == (c.ny, c.nx)
        assert refs[name + "/phi"].shape == (c.ny, c.nx)
    for k, c in enumerate(workloads.bench_parity_batch()):
        assert refs["batch%d/theta" % k].shape == (c.ny, c.nx)
    a = workloads.bench_parity_adjoint()
    assert refs["adjoint/g_theta0"].shape == (a.ny, a.nx)
    assert refs["adjoint/g_wall"].shape == (4,)


def test_stored_adjoint_is_the_oracles(orc, mk):
    refs = np.load(REFS)
    got = mk.adjoint_refs()
    for k in ("adjoint/target", "adjoint/g_theta0", "adjoint/g_wall"):
        assert close(got[k], refs[k])
    assert abs(float(got["adjoint/g_ste"]) - float(refs["adjoint/g_ste"])) <= 1e-12 * abs(float(refs["adjoint/g_ste"]))
