"""The stage kernel's pointwise templates, evaluated on the host, against
the oracle: the FP64 right-hand side within 1e-12 and the mixed-precision
one (split-pair differences, FP32 algebra) within the single-precision
bound of the GPU tests, on flat and puncture neighbourhoods, both gauges.
No GPU is needed: tests/host_rhs.cu instantiates the same templates the
device compiles (with the host's own float/double conversions), so an
algebra or differencing regression in either path shows on the CPU."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
from gpu_common import ko_pieces, offset_state, random_state, rel_err
from paper_2406_11626_gb300 import ccz4 as C, inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
MIXED_TOL = 2e-5   # the mixed path's single-precision bound (tests/test_gpu_mixed.py)


@pytest.fixture(scope="module")
def host_lib(tmp_path_factory):
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    nvcc = nvcc if os.path.exists(nvcc) else shutil.which("nvcc")
    if not nvcc:
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("host_rhs") / "libhost_rhs.so")
    subprocess.run([nvcc, "-O2", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC", "-shared",
                    "-I" + os.path.join(ROOT, "include"), os.path.join(HERE, "host_rhs.cu"), "-o", out],
                   check=True, capture_output=True)
    lib = ctypes.CDLL(out)
    lib.host_rhs.restype = None
    return lib


def _run(lib, bc, base, gauge, p, npv, mixed):
    dx = 1.0 / (npv[0] * p) if base == "flat" else 0.45
    origin = (-0.5 * npv[0] * p * dx, -0.5 * npv[1] * p * dx - 0.013, -0.5 * npv[2] * p * dx + 0.021)
    ijk = I.patch_ijk(npv, 2)
    og = O.Grid(p, npv, ijk, origin, dx, bc)
    U, G = random_state(p, npv, origin, dx, ijk, seed=p, bc=bc, base=base)
    kw = dict(I.PUNCTURE_PARAMS, slicing=gauge[0], shift=gauge[1], ko_eps=0.3)
    tiles = np.ascontiguousarray(og.fill_tiles(U, G))
    out = np.empty(og.ushape)
    P = C.make_params(**kw)
    lib.host_rhs(tiles.ctypes.data_as(ctypes.c_void_p), ctypes.c_int(p), ctypes.c_int(og.n_patches),
                 ctypes.c_double(dx), ctypes.byref(P), ctypes.c_int(int(mixed)), out.ctypes.data_as(ctypes.c_void_p))
    ref, _ = og.rhs(O.make_params(**kw), U, G, G)
    return rel_err(out, ref)


CASES = [("periodic", "flat", ("harmonic", "zero"), 6, (3, 2, 2)),
         ("periodic", "flat", ("1+log", "gamma-driver"), 6, (3, 2, 2)),
         ("sommerfeld", "puncture", ("1+log", "gamma-driver"), 5, (2, 3, 1))]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join([c[0], c[1], c[2][0]]))
def test_fp64_templates_match_the_oracle(host_lib, case):
    e = _run(host_lib, *case, mixed=False)
    assert e.max() < 1e-12, dict(zip(I.FIELDS, e))


@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join([c[0], c[1], c[2][0]]))
def test_mixed_templates_within_the_single_precision_bound(host_lib, case):
    e = _run(host_lib, *case, mixed=True)
    assert e.max() < MIXED_TOL, dict(zip(I.FIELDS, e))
    assert e.max() > 1e-12   # the algebra really ran in single precision


def test_mixed_templates_keep_fp64_differences_on_a_large_offset(host_lib):
    """The host counterpart of the GPU test of the same name: beta and b on
    offsets of 1000 and -500 with the zero-shift option (right-hand sides
    of pure dissipation) match the oracle to within the FP32 rounding of
    the combined second differences; taking the differences without the
    low parts of the split pairs misses this bar."""
    p, npv, dx = 6, (3, 2, 2), 1.0 / 18
    origin = (-0.5 * npv[0] * p * dx, -0.5 * npv[1] * p * dx, -0.5 * npv[2] * p * dx)
    ijk = I.patch_ijk(npv, 6)
    og = O.Grid(p, npv, ijk, origin, dx, "periodic")
    U, G, offset = offset_state(p, npv, origin, dx, ijk)
    kw = dict(I.PUNCTURE_PARAMS, shift="zero", ko_eps=0.3)
    tiles = np.ascontiguousarray(og.fill_tiles(U, G))
    out = np.empty(og.ushape)
    host_lib.host_rhs(tiles.ctypes.data_as(ctypes.c_void_p), ctypes.c_int(p), ctypes.c_int(og.n_patches),
                      ctypes.c_double(dx), ctypes.byref(C.make_params(**kw)), ctypes.c_int(1),
                      out.ctypes.data_as(ctypes.c_void_p))
    ref, _ = og.rhs(O.make_params(**kw), U, G, G)
    cko = kw["ko_eps"] / (64.0 * dx)
    for name in offset:
        v = I.IDX[name]
        b1, _ = ko_pieces(tiles, v, p)
        bar = 4.0 * 2.0 ** -24 * 144.0 * cko * b1
        assert np.abs(out[v] - ref[v]).max() <= bar, name


@pytest.mark.parametrize("bc,base,gauge,p,npv", CASES)
def test_two_phase_evaluation_equals_the_one_phase_one(host_lib, bc, base, gauge, p, npv):
    """The two-phase launch shape of the mixed stage kernel (stencil values
    recorded into per-thread slots, then the algebra replayed from them)
    computes the same right-hand side bit for bit as the one-phase one."""
    dx = 1.0 / (npv[0] * p) if base == "flat" else 0.45
    origin = (-0.5 * npv[0] * p * dx, -0.5 * npv[1] * p * dx - 0.013, -0.5 * npv[2] * p * dx + 0.021)
    ijk = I.patch_ijk(npv, 2)
    og = O.Grid(p, npv, ijk, origin, dx, bc)
    U, G = random_state(p, npv, origin, dx, ijk, seed=p + 1, bc=bc, base=base)
    tiles = np.ascontiguousarray(og.fill_tiles(U, G))
    P = C.make_params(**dict(I.PUNCTURE_PARAMS, slicing=gauge[0], shift=gauge[1]))
    outs = []
    for mode in (1, 2):
        out = np.empty(og.ushape)
        host_lib.host_rhs(tiles.ctypes.data_as(ctypes.c_void_p), ctypes.c_int(p), ctypes.c_int(og.n_patches),
                          ctypes.c_double(dx), ctypes.byref(P), ctypes.c_int(mode), out.ctypes.data_as(ctypes.c_void_p))
        outs.append(out)
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("shift", ["zero", "gamma-driver"])
def test_two_phase_slots_fit(host_lib, shift):
    """The stencil values one point asks for fit the kernel's slots."""
    nf, nd, mf, md = (ctypes.c_int() for _ in range(4))
    P = C.make_params(**dict(I.PUNCTURE_PARAMS, shift=shift))
    host_lib.host_tap_slots(ctypes.byref(P), ctypes.byref(nf), ctypes.byref(nd), ctypes.byref(mf), ctypes.byref(md))
    assert 0 < nf.value <= mf.value and 0 < nd.value <= md.value, (nf.value, nd.value)
    if shift == "gamma-driver":   # the larger case (the b equation's differences): not much room wasted
        assert mf.value - nf.value < 8 and md.value - nd.value < 4, (nf.value, nd.value)
