"""The algorithmic operation count of a point-stage as the oracle performs
it (its C source compiled with a counting scalar in place of double, one
RK4 step of a perturbed single puncture with a Sommerfeld shell), against
the count of the stage kernel's own templates that the bench line's
roofline divides by: the kernel's count is the smaller, so the fraction the
bench reports is the conservative one."""
import ctypes
import os
import shutil
import subprocess

import pytest

import oracle as O
from paper_2406_11626_gb300 import ccz4 as C, inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def opcount_lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("opcount") / "libopcount.so")
    subprocess.run([gxx, "-O1", "-std=c++17", "-fPIC", "-shared", "-w", os.path.join(HERE, "oracle_opcount.cpp"),
                    "-o", out], check=True, capture_output=True)
    lib = ctypes.CDLL(out)
    lib.oracle_ops_per_point_stage.restype = None
    return lib


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_kernel_count_is_a_lower_bound_of_the_oracle_count(opcount_lib, precision):
    out = (ctypes.c_double * 5)()
    P = O.make_params(**I.PUNCTURE_PARAMS)
    opcount_lib.oracle_ops_per_point_stage(ctypes.c_int(6), ctypes.c_int(2), ctypes.byref(P), out)
    add, mul, div, root, total = list(out)
    # thousands of operations per point-stage: the stencils, the algebra, the update
    assert 10000 < total < 30000 and add > 1000 and mul > 1000 and div > 0 and root > 0
    k = C.flops_per_point_stage(precision)
    assert k["fp64"] + k["fp32"] < total
