"""The first-order formulation and the second order with reconstruction on
the GPU (ccz4_fo_* through the C ABI) against the oracle's (og_fo_*), per
field in the relative max-norm ||gpu - oracle||_inf / max(||oracle||_inf, 1)
at 1e-11 (the GPU contracts to fused multiply-adds, the oracle does not):
the right-hand side of all 58 variables with and without the red terms on
perturbed puncture data with a Sommerfeld ghost shell and on a shuffled
periodic grid, the reconstruction of the auxiliary variables, and RK4 steps
of both formulations (ten gauge-wave steps, and puncture steps through the
ghost shell)."""
import numpy as np
import pytest

import oracle as O
from paper_2406_11626_gb300 import inputs as I

pytestmark = pytest.mark.gpu

NVF = I.NV_FO
TOL = 1e-11
PARAMS = dict(kappa1=0.3, kappa2=0.7, kappa3=0.45, e=1.7, c=1.3, tau=0.8, mu=0.35, f=0.6, eta=2.3, s=1.0,
              K0=0.0, ko_eps=0.1)


def rel(a, b):
    a = np.asarray(a).reshape(NVF, -1)
    b = np.asarray(b).reshape(NVF, -1)
    if a.shape[1] == 0:
        return np.zeros(NVF)
    return np.abs(a - b).max(axis=1) / np.maximum(np.abs(b).max(axis=1), 1.0)


def _perturbed(cfg, seed, amp=1e-2):
    """The configuration's 58-variable data with a smooth perturbation in
    every variable (auxiliary ones too, so they are not derivatives of the
    primaries: every term of every equation is exercised)."""
    U, G = I.fo_initial_state(cfg)
    x, y, z = I.point_coords(cfg.p, cfg.ijk(), cfg.origin, cfg.dx)
    box = 2.0 * abs(cfg.origin[0])
    rng = np.random.default_rng(seed)
    for v in range(NVF):
        k = rng.integers(-2, 3, size=3)
        k[0] = k[0] or 1
        ph, a = rng.uniform(0, 2 * np.pi), rng.uniform(-amp, amp)
        U[v] += a * np.sin(2 * np.pi * (k[0] * x + k[1] * y + k[2] * z) / box + ph)
        if G.shape[1]:
            gx, gy, gz = I.ghost_positions(cfg.N, cfg.origin, cfg.dx)
            G[v] += a * np.sin(2 * np.pi * (k[0] * gx + k[1] * gy + k[2] * gz) / box + ph)
    return U, G


def _pair(cfg, variant):
    from paper_2406_11626_gb300 import ccz4 as C
    g = C.Grid.from_config(cfg)
    fo = C.FirstOrder(g, variant)
    og = O.Grid(cfg.p, cfg.np, cfg.ijk(), cfg.origin, cfg.dx, cfg.bc)
    return g, fo, og


@pytest.mark.parametrize("variant", ["fo", "so-recon"])
@pytest.mark.parametrize("gauge", [("1+log", "gamma-driver"), ("harmonic", "zero")])
def test_rhs_matches_oracle_on_perturbed_puncture_data(variant, gauge):
    from paper_2406_11626_gb300 import ccz4 as C
    cfg = I.single_puncture_config(p=6, n_side=3, half_width=1.5, permute_seed=2)
    g, fo, og = _pair(cfg, variant)
    U, G = _perturbed(cfg, 1)
    fo.upload(U, G)
    fo.upload(U, G, buf="INI")
    kw = dict(PARAMS, slicing=gauge[0], shift=gauge[1])
    fo.rhs(C.make_params(**kw), "U", "RHS")
    rU, rG = fo.download("RHS")
    oU, oG = og.fo_rhs(O.make_params(**kw), U, G, G, red=(variant == "fo"))
    e = rel(rU, oU)
    assert e.max() < TOL, (I.FO_FIELDS[int(e.argmax())], e.max())
    assert rel(rG, oG).max() < TOL


def test_rhs_matches_oracle_on_a_shuffled_periodic_gauge_wave():
    from paper_2406_11626_gb300 import ccz4 as C
    cfg = I.gauge_wave_config(p=6, np_=(3, 3, 3), permute_seed=5)
    g, fo, og = _pair(cfg, "fo")
    U, _ = _perturbed(cfg, 3)
    fo.upload(U)
    fo.rhs(C.make_params(**I.GAUGE_WAVE_PARAMS), "U", "RHS")
    rU, _ = fo.download("RHS")
    oU, _ = og.fo_rhs(O.make_params(**I.GAUGE_WAVE_PARAMS), U, red=True)
    assert rel(rU, oU).max() < TOL


def test_reconstruction_matches_oracle():
    cfg = I.single_puncture_config(p=6, n_side=3, half_width=1.5, permute_seed=4)
    g, fo, og = _pair(cfg, "so-recon")
    U, G = _perturbed(cfg, 6)
    fo.upload(U, G)
    fo.reconstruct("U")
    gU, gG = fo.download("U")
    oU = og.fo_reconstruct(U, G)
    assert np.array_equal(gU[:I.NV], U[:I.NV]) and np.array_equal(gG, G)
    assert rel(gU, oU).max() < 1e-12


@pytest.mark.parametrize("variant", ["fo", "so-recon"])
def test_ten_gauge_wave_steps_match_oracle(variant):
    """The gauge-wave configuration (27^3 points as 3^3 patches of 9^3,
    periodic, harmonic slicing, RK4, dt = 0.1 dx), ten steps."""
    from paper_2406_11626_gb300 import ccz4 as C
    cfg = I.gauge_wave_config()
    g, fo, og = _pair(cfg, variant)
    U, G = I.fo_initial_state(cfg)
    if variant == "so-recon":
        U = og.fo_reconstruct(U)
    fo.upload(U)
    fo.step(C.make_params(**cfg.params), cfg.dt, 10)
    gU, _ = fo.download("U")
    P = O.make_params(**cfg.params)
    oU = U
    for _ in range(10):
        oU, _ = og.fo_rk4_step(P, cfg.dt, oU, variant=variant)
    e = rel(gU, oU)
    assert e.max() < TOL, (I.FO_FIELDS[int(e.argmax())], e.max())


@pytest.mark.parametrize("variant", ["fo", "so-recon"])
def test_puncture_steps_through_the_ghost_shell_match_oracle(variant):
    from paper_2406_11626_gb300 import ccz4 as C
    cfg = I.single_puncture_config(p=6, n_side=3, half_width=1.5)
    g, fo, og = _pair(cfg, variant)
    U, G = I.fo_initial_state(cfg)
    U, G = U.copy(), G.copy()
    x, y, z = I.point_coords(cfg.p, cfg.ijk(), cfg.origin, cfg.dx)
    U[I.IDX["betax"]] += 0.01 * np.sin(2 * np.pi * y / 3.0)   # a shift to advect with
    fo.upload(U, G)
    fo.upload(U, G, buf="INI")
    Pg = C.make_params(**cfg.params)
    fo.step(Pg, cfg.dt, 2)
    gU, gG = fo.download("U")
    oU, oG = U, G
    P = O.make_params(**cfg.params)
    for _ in range(2):
        oU, oG = og.fo_rk4_step(P, cfg.dt, oU, oG, G, variant=variant)
    e = rel(gU, oU)
    assert e.max() < TOL, (I.FO_FIELDS[int(e.argmax())], e.max())
    assert rel(gG, oG).max() < TOL


def test_refined_mesh_and_bad_arguments_are_refused():
    from paper_2406_11626_gb300 import ccz4 as C
    cfg = I.multilevel_puncture_config(p=6, n_side=4, half_width=2.0, boxes=[((1, 1, 1), (3, 3, 3))])
    gm = C.Grid.from_config(cfg)
    with pytest.raises(C.CCZ4Error) as e:
        C.FirstOrder(gm, "fo")
    assert e.value.code == C.ERR_INVALID and "single uniform level" in str(e.value)
    g = C.Grid.from_config(I.gauge_wave_config(p=6))
    fo = C.FirstOrder(g, "fo")
    with pytest.raises(C.CCZ4Error):
        fo.rhs(C.make_params(), "U", "U")
    with pytest.raises(C.CCZ4Error):
        fo.rk_stage(C.make_params(), 4, 0.1)
