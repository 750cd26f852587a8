"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bar: halo fill and index mapping bit-exact; floating point within 1e-11 in
the per-field relative max-norm ||gpu - oracle||_inf / max(||oracle||_inf, 1)
(the FP64 parity bar of the method; the GPU contracts to FMA and reorders
sums, the oracle does neither)."""
import numpy as np
import pytest

import oracle as O
from gpu_common import both_params, make_pair, random_state, rel_err
from paper_2406_11626_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-11
PUNC = dict(I.PUNCTURE_PARAMS)
GW = dict(I.GAUGE_WAVE_PARAMS)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available()
    from paper_2406_11626_gb300 import ccz4
    ccz4.lib()


@pytest.mark.parametrize("bc", ["periodic", "copy", "sommerfeld"])
@pytest.mark.parametrize("p,npv", [(6, (2, 3, 2)), (9, (3, 2, 2)), (12, (2, 2, 1)), (17, (1, 2, 2)),
                                   (1, (4, 5, 3)), (2, (3, 3, 3))])
def test_halo_fill_is_bit_exact(bc, p, npv):
    dx = 0.1
    origin = (-0.5 * npv[0] * p * dx, -0.3, -0.2)
    gg, og, ijk = make_pair(p, npv, origin, dx, bc, permute_seed=4)
    rng = np.random.default_rng(1)
    U = rng.standard_normal(og.ushape)
    G = rng.standard_normal(og.gshape)
    gg.upload(U, G)
    gg.fill_halos("U")
    np.testing.assert_array_equal(gg.download("TILE"), og.fill_tiles(U, G))


@pytest.mark.parametrize("bc,base,gauge", [("periodic", "flat", ("harmonic", "zero")),
                                           ("periodic", "flat", ("1+log", "gamma-driver")),
                                           ("copy", "flat", ("1+log", "gamma-driver")),
                                           ("sommerfeld", "puncture", ("1+log", "gamma-driver"))])
@pytest.mark.parametrize("p,npv", [(6, (3, 2, 2)), (9, (2, 2, 2)), (5, (2, 3, 1))])
def test_rhs_matches_oracle(bc, base, gauge, p, npv):
    dx = 1.0 / (npv[0] * p) if base == "flat" else 0.45
    origin = (-0.5 * npv[0] * p * dx, -0.5 * npv[1] * p * dx - 0.013, -0.5 * npv[2] * p * dx + 0.021)
    gg, og, ijk = make_pair(p, npv, origin, dx, bc, permute_seed=2)
    U, G = random_state(p, npv, origin, dx, ijk, seed=p, bc=bc, base=base)
    Gini = G * 0.999
    cp, op = both_params(**dict(PUNC, slicing=gauge[0], shift=gauge[1], ko_eps=0.3))
    gg.upload(U, G)
    if gg.n_ghost:
        gg.upload(U, Gini, buf="INI")   # only the ghost part of INI is read
    gg.rhs(cp, "U", "RHS")
    rU, rG = gg.download("RHS")
    oU, oG = og.rhs(op, U, G, Gini)
    assert rel_err(rU, oU).max() < TOL
    assert rel_err(rG, oG).max() < TOL
    assert np.abs(oU).max() > 1e-3   # the data exercise the equations


def test_rhs_on_exact_gauge_wave_matches_oracle():
    cfg = I.gauge_wave_config(permute_seed=3)
    gg, og, ijk = make_pair(cfg.p, cfg.np, cfg.origin, cfg.dx, cfg.bc, permute_seed=3)
    U, _ = I.initial_state(cfg)
    cp, op = both_params(**cfg.params)
    gg.upload(U)
    gg.rhs(cp, "U", "RHS")
    rU, _ = gg.download("RHS")
    oU, _ = og.rhs(op, U)
    assert rel_err(rU, oU).max() < TOL


@pytest.mark.slow
def test_gauge_wave_ten_steps_match_oracle():
    """The gauge-wave workload (27^3 points as 3^3 patches of 9^3, RK4, CFL 0.1,
    10 steps): the state after 10 steps agrees with the oracle within 1e-11 in
    every field, and both stay close to the exact travelling wave."""
    cfg = I.gauge_wave_config(permute_seed=5)
    gg, og, ijk = make_pair(cfg.p, cfg.np, cfg.origin, cfg.dx, cfg.bc, permute_seed=5)
    U0, _ = I.initial_state(cfg)
    cp, op = both_params(**cfg.params)
    gg.upload(U0)
    gg.step(cp, cfg.dt, cfg.steps)
    gU, _ = gg.download("U")
    oU = U0
    for _ in range(cfg.steps):
        oU, _ = og.rk4_step(op, cfg.dt, oU)
    e = rel_err(gU, oU)
    assert e.max() < TOL, dict(zip(I.FIELDS, e))
    x, _, _ = I.point_coords(cfg.p, ijk, cfg.origin, cfg.dx)
    exact = I.gauge_wave(x, cfg.dt * cfg.steps)
    assert np.abs(oU - exact).max() < 1e-4


@pytest.mark.parametrize("bc", ["periodic", "sommerfeld"])
def test_rk4_stages_match_oracle_step(bc):
    """The four fused stage kernels make one oracle RK4 step, ghost cells and
    enforcement included."""
    p, npv, dx = 6, (3, 3, 2), 0.3
    origin = (-2.7, -2.65, -1.75)
    gg, og, ijk = make_pair(p, npv, origin, dx, bc, permute_seed=8)
    U, G = random_state(p, npv, origin, dx, ijk, seed=3, bc=bc, base="puncture", amp=0.01)
    Gini = G.copy()
    cp, op = both_params(**PUNC)
    gg.upload(U, G)
    if gg.n_ghost:
        gg.upload(U, Gini, buf="INI")
    dt = 0.1 * dx
    for s in range(4):
        gg.rk_stage(cp, s, dt)
    gU, gG = gg.download("U")
    oU, oG = og.rk4_step(op, dt, U, G, Gini)
    assert rel_err(gU, oU).max() < TOL
    assert rel_err(gG, oG).max() < TOL


def test_constraints_match_oracle_and_are_deterministic():
    import torch
    p, npv, dx = 6, (3, 2, 2), 0.35
    origin = (-3.1, -2.0, -2.2)
    gg, og, ijk = make_pair(p, npv, origin, dx, "sommerfeld", permute_seed=1)
    U, G = random_state(p, npv, origin, dx, ijk, seed=7, bc="sommerfeld", base="puncture")
    gg.upload(U, G)
    H = torch.zeros(gg.n_points, dtype=torch.float64, device="cuda")
    M = torch.zeros(3 * gg.n_points, dtype=torch.float64, device="cuda")
    out = gg.constraints("U", H.data_ptr(), M.data_ptr())
    out2 = gg.constraints("U")
    np.testing.assert_array_equal(out, out2)
    oH, oM, oout = og.constraints(U, G)
    h = H.cpu().numpy()
    m = M.cpu().numpy().reshape(3, -1)
    assert np.abs(h - oH.ravel()).max() / max(np.abs(oH).max(), 1.0) < TOL
    assert np.abs(m - oM.reshape(3, -1)).max() / max(np.abs(oM).max(), 1.0) < TOL
    np.testing.assert_allclose(out[:4], oout[:4], rtol=1e-12)
    assert out[4] == 0.0


def test_enforce_matches_oracle():
    p, npv, dx = 5, (2, 2, 2), 0.2
    gg, og, ijk = make_pair(p, npv, (0, 0, 0), dx, "periodic")
    rng = np.random.default_rng(9)
    U = I.flat(og.ushape[1:]) + rng.uniform(-0.1, 0.1, size=og.ushape)
    gg.upload(U)
    gg.enforce("U")
    gU, _ = gg.download("U")
    assert rel_err(gU, og.enforce(U)).max() < 1e-14


def test_nonfinite_state_is_reported():
    from paper_2406_11626_gb300 import ccz4 as C
    gg, og, ijk = make_pair(4, (2, 1, 1), (0, 0, 0), 0.25, "periodic")
    U = I.flat(og.ushape[1:])
    U[I.IDX["K"], 1, 2, 2, 2] = np.nan
    gg.upload(U)
    with pytest.raises(C.CCZ4Error) as e:
        gg.constraints("U")
    assert e.value.code == C.ERR_NONFINITE
    out = gg.constraints("U", raise_nonfinite=False)
    assert out[4] > 0 and np.isfinite(out[0])


def test_invalid_arguments_are_rejected_without_launch():
    from paper_2406_11626_gb300 import ccz4 as C
    with pytest.raises(C.CCZ4Error):
        C.Grid(4, (2, 2, 2), np.zeros((8, 3), dtype=np.int32), (0, 0, 0), 0.1)   # duplicate slots
    with pytest.raises(C.CCZ4Error):
        C.Grid(4, (2, 2, 2), I.patch_ijk((2, 2, 1)), (0, 0, 0), 0.1)             # count mismatch
    with pytest.raises(C.CCZ4Error):
        C.Grid(4, (1, 1, 1), I.patch_ijk((1, 1, 1)), (0, 0, 0), -0.1)            # dx <= 0
    g = C.Grid(4, (1, 1, 1), I.patch_ijk((1, 1, 1)), (0, 0, 0), 0.1)
    P = C.make_params()
    with pytest.raises(C.CCZ4Error):
        g.rk_stage(P, 4, 0.01)
    with pytest.raises(C.CCZ4Error):
        g.rhs(P, "U", "U")
    with pytest.raises(C.CCZ4Error):
        g.fill_halos("TILE")
    g.step(P, 0.01, 0)   # zero steps: a no-op


def test_evolve_host_equals_device_steps():
    cfg = I.gauge_wave_config(p=6, np_=(2, 2, 2), permute_seed=1)
    from paper_2406_11626_gb300 import ccz4 as C
    g = C.Grid.from_config(cfg)
    U0, _ = I.initial_state(cfg)
    P = C.make_params(**cfg.params)
    Uh, _ = g.evolve_host(P, cfg.dt, 3, U0)
    g.upload(U0)
    g.step(P, cfg.dt, 3)
    Ud, _ = g.download("U")
    np.testing.assert_array_equal(Uh, Ud)


def test_pinned_host_buffers_take_the_copy_kernel_with_the_same_result():
    """Pinned (mapped) host state, interior and Sommerfeld ghost cells, is
    moved by the library's copy kernel instead of the copy engine: the same
    values either way, in both directions."""
    import torch
    from paper_2406_11626_gb300 import ccz4 as C
    cfg = I.single_puncture_config(p=6, n_side=3, half_width=1.5)
    g = C.Grid.from_config(cfg)
    U0, G0 = I.initial_state(cfg)
    U0 = np.ascontiguousarray(U0).reshape(I.NV, -1)
    G0 = np.ascontiguousarray(G0).reshape(I.NV, -1)
    P = C.make_params(**cfg.params)
    pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
    Up, Gp = pin(U0), pin(G0)
    Uo, Go = pin(np.zeros_like(U0)), pin(np.zeros_like(G0))
    g.evolve_host(P, cfg.dt, 2, Up, Gp, Uo, Go)       # pinned: copy kernel
    Ua, Ga = g.evolve_host(P, cfg.dt, 2, U0, G0)     # pageable: copy engine
    np.testing.assert_array_equal(Uo.reshape(Ua.shape), Ua)
    np.testing.assert_array_equal(Go, Ga)
    g.upload(Up, Gp)                                  # and the plain upload / download
    Ud, Gd = g.download("U")
    np.testing.assert_array_equal(Ud.reshape(I.NV, -1), U0)
    np.testing.assert_array_equal(Gd, G0)


@pytest.mark.slow
def test_single_puncture_full_size_sampled_parity():
    """The 144^3 single-puncture workload in the launch configuration the
    benchmark times: after one fused RK stage, the accumulator holds k0 at
    every point; sampled interior points (including the patches next to the
    puncture and the outer boundary) and every ghost cell kind agree with
    the oracle evaluated point by point."""
    cfg = I.single_puncture_config()
    from paper_2406_11626_gb300 import ccz4 as C
    g = C.Grid.from_config(cfg)
    og = O.Grid(cfg.p, cfg.np, cfg.ijk(), cfg.origin, cfg.dx, cfg.bc)
    U, G = I.initial_state(cfg)
    x, y, z = I.point_coords(cfg.p, cfg.ijk(), cfg.origin, cfg.dx)
    U = I.smooth_perturbation(x, y, z, seed=3, amp=1e-3, box=16.0, base=U)
    g.upload(U, G)
    g.upload(U, G, buf="INI")
    P = C.make_params(**cfg.params)
    g.rk_stage(P, 0, cfg.dt)
    acc, accG = g.download("ACC")
    r = np.sqrt(x ** 2 + y ** 2 + z ** 2).ravel()
    rng = np.random.default_rng(0)
    pts = np.concatenate([rng.choice(len(r), 300, replace=False), np.argsort(r)[:40],
                          np.argsort(-np.abs(x).ravel())[:30]])
    ref = og.rhs_points(O.make_params(**cfg.params), U, G, pts)
    got = acc.reshape(I.NV, -1)[:, pts].T
    scale = np.maximum(np.abs(ref).max(axis=0), 1.0)
    assert (np.abs(got - ref) / scale).max() < TOL
    # every ghost cell of the Sommerfeld shell
    oG = og.ghost_rhs(O.make_params(**cfg.params), U, G, G)
    assert rel_err(accG, oG).max() < TOL


def test_graph_steps_are_bit_identical_to_plain_steps():
    """A time step captured as a CUDA graph and replayed gives exactly the
    state of the same steps launched one by one; changing dt re-captures."""
    from paper_2406_11626_gb300 import ccz4 as C
    cfg = I.single_puncture_config(p=6, n_side=3, half_width=2.0)
    U0, G0 = I.initial_state(cfg)
    out = []
    for use_graph in (False, True):
        g = C.Grid.from_config(cfg)
        g.upload(U0, G0)
        g.upload(U0, G0, buf="INI")
        P = C.make_params(**cfg.params)
        for dt in (cfg.dt, 0.5 * cfg.dt):
            if use_graph:
                g.step_graph(P, dt, 3)
            else:
                g.step(P, dt, 3)
        out.append(g.download("U"))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("bc,p,npv", [("sommerfeld", 9, (2, 2, 2)), ("periodic", 6, (3, 2, 2)), ("copy", 17, (1, 2, 1)),
                                      ("periodic", 2, (3, 3, 2))])
def test_mixed_derivatives_from_the_halo_fill_match_oracle(bc, p, npv):
    """The halo fill forms d_x d_y, d_x d_z, d_y d_z of g~, alpha, beta and phi
    from first derivatives shared in shared memory; they equal the oracle's
    tensor-product stencil at every point (buffer CCZ4_BUF_MIX)."""
    dx = 0.3
    origin = (-0.5 * npv[0] * p * dx, -0.5 * npv[1] * p * dx - 0.011, -0.5 * npv[2] * p * dx + 0.017)
    gg, og, ijk = make_pair(p, npv, origin, dx, bc, permute_seed=6)
    U, G = random_state(p, npv, origin, dx, ijk, seed=2, bc=bc, base="puncture" if bc == "sommerfeld" else "flat")
    gg.upload(U, G)
    gg.fill_halos("U")
    n = gg.n_points
    tiles = gg.download("TILE")
    mix = gg.download("MIX")
    assert mix.shape == (33, n)
    slots = [(I.IDX[f], 3 * k) for k, f in enumerate(["gxx", "gxy", "gxz", "gyy", "gyz", "gzz"])]
    slots += [(I.IDX["alpha"], 18), (I.IDX["betax"], 21), (I.IDX["betay"], 24), (I.IDX["betaz"], 27), (I.IDX["phi"], 30)]
    rng = np.random.default_rng(0)
    pts = rng.choice(n, min(n, 200), replace=False)
    for pt in pts:
        _, d2, _ = og.point_derivs(U, G, int(pt))
        for v, s in slots:
            ref = np.array([d2[v, 0, 1], d2[v, 0, 2], d2[v, 1, 2]])
            got = mix[s:s + 3, pt]
            assert np.abs(got - ref).max() <= 1e-11 * max(np.abs(ref).max(), 1.0), (pt, v)
    np.testing.assert_array_equal(tiles, og.fill_tiles(U, G))
