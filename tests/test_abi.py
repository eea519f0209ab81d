"""The C-ABI library loads and exports every entry point include/*.h declares;
argument checks happen before any CUDA call (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(lbm_[A-Za-z0-9_]+)\s*\(", src, re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    import sys
    sys.path.insert(0, ROOT)
    from paper_2505_13097_gb300 import build as b
    b.build()
    from paper_2505_13097_gb300 import _abi
    return _abi.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("lbm_stefan_create", "lbm_stefan_set_ic", "lbm_stefan_set_bc", "lbm_stefan_step",
              "lbm_stefan_get_fields", "lbm_stefan_adjoint_step", "lbm_stefan_destroy"):
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2505_13097_gb300 import _abi
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    # the Python binding covers the same names
    assert names == set(_abi.SIGNATURES)


def _params(**kw):
    from paper_2505_13097_gb300 import _abi
    d = dict(lattice=2, nx=16, ny=16, tau=1.0, delta=0.01, ste=0.1, precision=1, newton_tol=1e-14,
             newton_max_iter=60, bb_mode=0)
    d.update(kw)
    return _abi.lbm_stefan_params(**d)


@pytest.mark.parametrize("bad", [dict(tau=0.5), dict(tau=float("nan")), dict(ste=0.0), dict(delta=-1.0),
                                 dict(nx=1), dict(lattice=4), dict(precision=2), dict(bb_mode=5),
                                 dict(lattice=1, ny=2), dict(lattice=2, ny=1), dict(newton_max_iter=0),
                                 dict(newton_tol=0.0), dict(lattice=3, nx=2), dict(lattice=3, ny=2),
                                 dict(lattice=2, bb_mode=2), dict(lattice=3, bb_mode=3)])
def test_create_rejects_bad_arguments(lib, bad):
    from paper_2505_13097_gb300 import _abi
    h = ctypes.c_void_p()
    p = _params(**bad)
    st = lib.lbm_stefan_create(ctypes.byref(p), None, ctypes.byref(h))
    assert st == _abi.LBM_ERR_ARG
    assert not h.value
    assert lib.lbm_stefan_last_error()


def test_null_handles_are_rejected(lib):
    from paper_2505_13097_gb300 import _abi
    assert lib.lbm_stefan_step(None, 1) == _abi.LBM_ERR_ARG
    assert lib.lbm_stefan_set_ic(None, None, 0) == _abi.LBM_ERR_ARG
    assert lib.lbm_stefan_create(None, None, None) == _abi.LBM_ERR_ARG
    assert lib.lbm_stefan_batch_create(0, None, 1, 1e-14, 60, None, None) == _abi.LBM_ERR_ARG
    assert lib.lbm_stefan_set_ste(None, 0.1) == _abi.LBM_ERR_ARG
    assert lib.lbm_stefan_set_wait_test(None, 0.01, -1) == _abi.LBM_ERR_ARG
    idx = ctypes.c_int()
    assert lib.lbm_stefan_adjoint_segment(None, None, 1, None, None, None, ctypes.byref(idx)) == _abi.LBM_ERR_ARG
    lib.lbm_stefan_destroy(None)
    lib.lbm_stefan_batch_destroy(None)


def test_binding_constants_match_the_header():
    # every enum constant of include/*.h has the same value in the Python binding
    import sys
    sys.path.insert(0, ROOT)
    from paper_2505_13097_gb300 import _abi
    consts = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for body in re.findall(r"enum\s*\{([^}]*)\}", src):
            for m in re.finditer(r"(LBM_[A-Z0-9_]+)\s*=\s*(\d+)", body):
                consts[m.group(1)] = int(m.group(2))
        for body in re.findall(r"typedef\s+enum\s*\{([^}]*)\}", src):
            for m in re.finditer(r"(LBM_[A-Z0-9_]+)\s*=\s*(\d+)", body):
                consts[m.group(1)] = int(m.group(2))
    assert {"LBM_D2Q5", "LBM_NEU_EQ17", "LBM_ILFBM", "LBM_ERR_NEWTON"} <= set(consts)
    for name, v in consts.items():
        assert getattr(_abi, name) == v, name
