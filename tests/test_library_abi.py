"""The CUDA library loads on a machine without a GPU and exports every
function that the headers in include/ declare (no compute call is made
here)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(ccz4_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_hot_path_calls():
    names = _declared()
    for n in ("ccz4_alloc_patches", "ccz4_fill_halos", "ccz4_rhs", "ccz4_rk_stage", "ccz4_constraints",
              "ccz4_alloc_mesh", "ccz4_restrict", "ccz4_id_solve"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2406_11626_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_library_is_built_for_sm_103a():
    from paper_2406_11626_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.NVCC_FLAGS)


def test_flop_count_is_available_without_a_gpu():
    """The algorithmic flop count of the stage kernel comes from the host
    instantiation of the kernel templates with counting scalars."""
    from paper_2406_11626_gb300 import build, ccz4
    build.build()
    f64 = ccz4.flops_per_point_stage("fp64")
    fmx = ccz4.flops_per_point_stage("mixed")
    # the whole right-hand side (stencils, dissipation, algebra, update): thousands of flops per point-stage
    assert f64["fp32"] == 0 and 2500 < f64["fp64"] < 4000 and f64["conversions"] == 0
    assert f64["fp64"] == 2 * f64["fp64_fma"] + f64["fp64_add_mul"] + f64["fp64_div_root"]
    assert fmx["fp32"] > 1000 and fmx["fp64"] < f64["fp64"] and fmx["conversions"] > 0
    # the mixed path's stencil differences (every field but alpha and phi) run on split FP32
    # pairs: what stays FP64 is the 1/phi terms, the differences of alpha and phi and the
    # update, under a fifth of the FP64 path's work; the differences add thousands of FP32 flops
    assert fmx["fp64"] < 0.2 * f64["fp64"] and fmx["fp32"] > 5000
    assert fmx["fp64"] == 2 * fmx["fp64_fma"] + fmx["fp64_add_mul"] + fmx["fp64_div_root"]
