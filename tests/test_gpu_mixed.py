"""The mixed-precision path (FP64 state, 1/phi terms and update; stencil
differences on split FP32 pairs with FP64 accuracy; FP32 pointwise algebra)
against the FP64 oracle and the FP64 path.

There is no bit-level parity to ask of FP32 algebra: the bar is an error
bound derived from single-precision rounding. The algebra of one point
chains a few thousand operations whose terms reach ~100x the size of the
result (the Ricci tensor and the Gamma-hat source), so with the FP32 unit
roundoff 6e-8 the right-hand side is expected to agree with FP64 to
~1e-5 of each field's scale; evolved states carry that error times dt per
stage."""
import numpy as np
import pytest

import oracle as O
from gpu_common import both_params, ko_pieces, make_pair, offset_state, random_state, rel_err
from paper_2406_11626_gb300 import inputs as I

pytestmark = pytest.mark.gpu

RHS_TOL = 2e-5
PUNC = dict(I.PUNCTURE_PARAMS)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available()


@pytest.mark.parametrize("bc,base", [("periodic", "flat"), ("sommerfeld", "puncture")])
def test_mixed_rhs_within_single_precision_bound(bc, base):
    p, npv = 6, (3, 2, 2)
    dx = 1.0 / 18 if base == "flat" else 0.4
    origin = (-0.5 * npv[0] * p * dx, -0.5 * npv[1] * p * dx - 0.013, -0.5 * npv[2] * p * dx + 0.021)
    gg, og, ijk = make_pair(p, npv, origin, dx, bc, permute_seed=2)
    U, G = random_state(p, npv, origin, dx, ijk, seed=4, bc=bc, base=base)
    cp, op = both_params(**dict(I.PUNCTURE_PARAMS, precision="mixed"))
    gg.upload(U, G)
    if gg.n_ghost:
        gg.upload(U, G, buf="INI")
    gg.rhs(cp, "U", "RHS")
    rU, rG = gg.download("RHS")
    oU, oG = og.rhs(op, U, G, G)
    e = rel_err(rU, oU)
    assert e.max() < RHS_TOL, dict(zip(I.FIELDS, e))
    assert e.max() > 1e-12   # the algebra really ran in single precision
    assert rel_err(rG, oG).max() < 1e-12   # ghost cells stay FP64


@pytest.mark.slow
def test_mixed_puncture_evolution_tracks_fp64():
    """A small single-puncture run (same physics and dx ratio as the 144^3
    workload): after 20 RK4 steps every field of the mixed run is within
    1e-5 of the FP64 run (relative to the field's scale), and the
    constraint norms agree within 2x."""
    from paper_2406_11626_gb300 import ccz4 as C
    cfg = I.single_puncture_config(p=9, n_side=4, half_width=2.0)
    g64 = C.Grid.from_config(cfg)
    g32 = C.Grid.from_config(cfg)
    U, G = I.initial_state(cfg)
    for g in (g64, g32):
        g.upload(U, G)
        g.upload(U, G, buf="INI")
    P64 = C.make_params(**cfg.params)
    P32 = C.make_params(**dict(cfg.params, precision="mixed"))
    g64.step(P64, cfg.dt, 20)
    g32.step(P32, cfg.dt, 20)
    a, _ = g64.download("U")
    b, _ = g32.download("U")
    e = rel_err(b, a)
    assert e.max() < 1e-5, dict(zip(I.FIELDS, e))
    c64 = g64.constraints("U")
    c32 = g32.constraints("U")
    assert 0.5 < c32[0] / c64[0] < 2.0 and 0.5 < c32[1] / c64[1] < 2.0


def test_mixed_fill_keeps_fp32_slots_for_the_fp32_algebra():
    """For the mixed path the halo fill takes the mixed derivatives of g~ and
    beta (used in FP32 by the mixed stage kernel) with inner differences on
    the split pairs and FP32 weights and outer differences, and stores them
    as FP32 in the first 27 float slots of the
    buffer; those of alpha and phi (used in FP64 next to 1/phi) stay FP64 and
    equal the FP64 fill bit for bit. The tiles of alpha and phi equal the
    FP64 fill's; every other field's tile holds the split pair of the FP64
    value u: hi = u rounded to FP32 (ties away from zero) and lo = u - hi
    rounded to FP32 (to nearest even), so hi + lo = u within 2^-48 |u|."""
    from paper_2406_11626_gb300 import ccz4 as C
    p, npv, dx = 9, (2, 2, 2), 0.35
    origin = (-3.15, -3.1, -3.2)
    gg, og, ijk = make_pair(p, npv, origin, dx, "sommerfeld", permute_seed=3)
    U, G = random_state(p, npv, origin, dx, ijk, seed=5, bc="sommerfeld", base="puncture")
    gg.upload(U, G)
    gg.fill_halos("U", P=C.make_params(**PUNC, precision="fp64"))
    t64, m64 = gg.download("TILE"), gg.download("MIX")
    gg.fill_halos("U", P=C.make_params(**PUNC, precision="mixed"))
    t32, raw = gg.download("TILE"), gg.download("MIX")
    for v, name in enumerate(I.FIELDS):
        if name in ("alpha", "phi"):
            np.testing.assert_array_equal(t32[v], t64[v])
            continue
        u = t64[v].reshape(-1)
        pair = np.ascontiguousarray(t32[v]).reshape(-1).view(np.float32).reshape(-1, 2)
        hi, lo = pair[:, 0], pair[:, 1]
        # hi: the nearest FP32 number; where two are nearest, the one of larger magnitude
        rne = u.astype(np.float32)
        tie = hi != rne
        assert np.all(np.abs(hi[tie].astype(np.float64)) > np.abs(u[tie])), name
        assert np.all(np.abs(hi[tie] - u[tie]) == np.abs(rne[tie] - u[tie])), name
        np.testing.assert_array_equal(lo, (u - hi.astype(np.float64)).astype(np.float32), err_msg=name)
        rec = hi.astype(np.float64) + lo.astype(np.float64)
        assert np.all(np.abs(rec - u) <= 2.0 ** -48 * np.abs(u)), name
    n = gg.n_points
    f32 = np.ascontiguousarray(raw).reshape(-1).view(np.float32)[:27 * n].reshape(27, n)
    for s in list(range(18)) + list(range(21, 30)):
        ref = m64[s]
        got = f32[s if s < 18 else s - 3].astype(np.float64)
        assert np.abs(got - ref).max() <= 1e-6 * max(np.abs(ref).max(), 1e-30), s
    for s in (18, 19, 20, 30, 31, 32):
        np.testing.assert_array_equal(raw[s], m64[s])


def test_split_pair_differences_keep_fp64_accuracy_on_a_large_offset():
    """The mixed path takes stencil differences on split FP32 pairs with the
    accuracy of FP64 differences. With the zero-shift option the right-hand
    sides of beta and b are their Kreiss-Oliger dissipation alone, and
    dissipation is blind to a constant: on beta = 1000 + s and b = -500 + s
    (s a smooth perturbation of size 1e-3) the mixed path must match the
    FP64 oracle to within the FP32 rounding of the combination of the
    second differences, about 4 x 2^-24 x 144 x eps/(64 dx) x max |second
    difference|. Differences of values rounded to FP32 would miss that bar
    by orders of magnitude (checked below on the same tiles in numpy)."""
    p, npv, dx = 6, (3, 2, 2), 1.0 / 18
    origin = (-0.5 * npv[0] * p * dx, -0.5 * npv[1] * p * dx, -0.5 * npv[2] * p * dx)
    gg, og, ijk = make_pair(p, npv, origin, dx, "periodic", permute_seed=6)
    U, G, offset = offset_state(p, npv, origin, dx, ijk)
    kw = dict(PUNC, shift="zero", ko_eps=0.3)
    cp, op = both_params(**dict(kw, precision="mixed"))
    gg.upload(U, G)
    gg.rhs(cp, "U", "RHS")
    rU, _ = gg.download("RHS")
    oU, _ = og.rhs(op, U, G, G)
    tiles = og.fill_tiles(U, G)
    cko = kw["ko_eps"] / (64.0 * dx)
    eps32 = 2.0 ** -24
    for name in offset:
        v = I.IDX[name]
        b1, ko_naive = ko_pieces(tiles, v, p)
        bar = 4.0 * eps32 * 144.0 * cko * b1
        err = np.abs(rU[v] - oU[v]).max()
        assert np.abs(oU[v]).max() > 100.0 * bar, name      # the dissipation itself is resolved
        assert err <= bar, (name, err, bar)
        naive = np.abs(cko * ko_naive.astype(np.float64) - oU[v]).max()
        assert naive > 100.0 * bar, (name, naive, bar)      # rounding the values first fails
