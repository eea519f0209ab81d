"""Float-float helpers of the FP32 form's Newton solves, checked on the host.

The CUDA kernels refine each deferred node's root (Eq. 14) in float-float
arithmetic (csrc/ffmath.cuh): exp for non-positive arguments (Cody-Waite
reduction by ln2, Taylor series) and phi(x) = 1/(1 + exp(-2x/delta)) with
1 - phi (Sec. 4.1).  The same header compiles for the CPU with plain IEEE
float operations; tests/native/ffmath_check.cpp compares it with long double
on seeded random inputs.  The bounds are those the solve's accuracy argument
needs: theta' = m0 + (phi(theta) - phi(root))/Ste carries phi's absolute
error times 1/Ste (<= 100 here), which must stay far below the FP32 storage
rounding of theta (about 1e-9 in the band).
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def ffmath_errors(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("ffmath") / "ffmath_check")
    # -ffp-contract=off: the host build must not fuse the error-free
    # transformations' separate multiplies and adds
    subprocess.run([cxx, "-O2", "-ffp-contract=off", "-std=c++17", os.path.join(HERE, "native", "ffmath_check.cpp"),
                    "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return {k: float(v) for k, v in (line.split() for line in out.strip().splitlines())}


def test_exp_nonpos_relative_error(ffmath_errors):
    assert ffmath_errors["exp_rel"] < 1e-12


def test_phi_absolute_error(ffmath_errors):
    assert ffmath_errors["phi_abs"] < 5e-14


def test_one_minus_phi_relative_error(ffmath_errors):
    assert ffmath_errors["phic_rel"] < 2e-12


def test_quotient_and_product(ffmath_errors):
    assert ffmath_errors["quot_rel"] < 1e-13
    assert ffmath_errors["prod_rel"] < 1e-13
