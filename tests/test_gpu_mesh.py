"""Parity of the CUDA path with the oracle on statically refined ratio-3
meshes (appendix "refinement transition"): halo fill with coarse-to-fine
interpolation (bit-exact), right-hand side with per-level spacing, RK4 steps
with restriction, leaf-only constraint norms, mixed precision, and the
three-level puncture workload at full size on sampled points."""
import numpy as np
import pytest

import oracle as O
from gpu_common import both_params, rel_err
from paper_2406_11626_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-11
PUNC = dict(I.PUNCTURE_PARAMS)

MESHES = {
    "two": (6, (4, 4, 4), [((1, 1, 1), (3, 3, 3))]),
    "three": (6, (4, 4, 4), [((1, 1, 1), (3, 3, 3)), ((5, 5, 5), (7, 7, 7))]),
    "small_p": (3, (5, 4, 4), [((1, 1, 1), (4, 3, 3)), ((4, 4, 4), (6, 5, 5))]),
    "p9": (9, (3, 3, 3), [((1, 1, 1), (2, 2, 2))]),
    # the largest patch edge the fill takes: 24^3 tiles, up to 4044 separable
    # x and y interpolations per patch in its shared memory
    "p18": (18, (3, 3, 3), [((1, 1, 1), (2, 2, 2))]),
}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available()
    from paper_2406_11626_gb300 import ccz4
    ccz4.lib()


def mesh_pair(name, bc, dx=0.3, shuffle=0):
    from paper_2406_11626_gb300 import ccz4 as C
    p, np_, boxes = MESHES[name]
    lev, ijk = I.refined_mesh(np_, boxes)
    if shuffle:
        perm = np.random.default_rng(shuffle).permutation(len(lev))
        lev, ijk = lev[perm], ijk[perm]
    origin = tuple(-0.5 * n * p * dx + o for n, o in zip(np_, (0.0, -0.013, 0.021)))
    gg = C.Grid(p, np_, ijk, origin, dx, bc, level=lev)
    og = O.Grid(p, np_, ijk, origin, dx, bc, level=lev)
    return gg, og, lev, ijk, origin


def mesh_state(gg, lev, ijk, origin, dx, bc, seed, base, amp=0.02):
    p = gg.p
    x, y, z = I.mesh_point_coords(p, lev, ijk, origin, dx)
    box = gg.np[0] * p * dx
    U0 = I.brill_lindquist(x, y, z) if base == "puncture" else I.flat(x.shape)
    U = I.smooth_perturbation(x, y, z, seed, amp=amp, box=box, base=U0)
    G = np.zeros((I.NV, 0))
    if bc == "sommerfeld":
        N = tuple(n * p for n in gg.np)
        gx, gy, gz = I.ghost_positions(N, origin, dx)
        G0 = I.brill_lindquist(gx, gy, gz) if base == "puncture" else I.flat(gx.shape)
        G = I.smooth_perturbation(gx, gy, gz, seed, amp=amp, box=box, base=G0)
    return np.ascontiguousarray(U), np.ascontiguousarray(G)


@pytest.mark.parametrize("name,bc", [("two", "periodic"), ("two", "copy"), ("three", "sommerfeld"),
                                     ("small_p", "periodic"), ("p9", "sommerfeld"), ("p18", "sommerfeld")])
def test_mesh_halo_fill_is_bit_exact(name, bc):
    """Same-level copies, level-0 boundary rules and the interpolated halo
    of refined patches all equal the oracle bit for bit (the kernel rounds
    every product and sum of the interpolation on its own, in the oracle's
    order)."""
    gg, og, lev, ijk, origin = mesh_pair(name, bc, shuffle=3)
    rng = np.random.default_rng(1)
    U = rng.standard_normal(og.ushape)
    G = rng.standard_normal((I.NV, og.n_ghost))
    gg.upload(U, G)
    gg.fill_halos("U")
    np.testing.assert_array_equal(gg.download("TILE"), og.fill_tiles(U, G))


@pytest.mark.parametrize("name,bc,base", [("two", "periodic", "flat"), ("three", "sommerfeld", "puncture"),
                                          ("small_p", "copy", "flat")])
def test_mesh_rhs_matches_oracle(name, bc, base):
    dx = 0.3
    gg, og, lev, ijk, origin = mesh_pair(name, bc, dx=dx, shuffle=5)
    U, G = mesh_state(gg, lev, ijk, origin, dx, bc, seed=4, base=base)
    Gini = G * 0.999
    cp, op = both_params(**dict(PUNC, ko_eps=0.3))
    gg.upload(U, G)
    if gg.n_ghost:
        gg.upload(U, Gini, buf="INI")
    gg.rhs(cp, "U", "RHS")
    rU, rG = gg.download("RHS")
    oU, oG = og.rhs(op, U, G, Gini)
    assert rel_err(rU, oU).max() < TOL
    assert rel_err(rG, oG).max() < TOL
    assert np.abs(oU).max() > 1e-3


def test_mesh_restriction_is_bit_exact():
    gg, og, lev, ijk, origin = mesh_pair("three", "copy", shuffle=2)
    U = np.random.default_rng(9).standard_normal(og.ushape)
    gg.upload(U)
    gg.restrict("U")
    gU, _ = gg.download("U")
    np.testing.assert_array_equal(gU, og.restrict(U))


@pytest.mark.parametrize("name,bc", [("three", "sommerfeld"), ("two", "periodic")])
def test_mesh_rk4_steps_match_oracle(name, bc):
    """Three RK4 steps (halo interpolation at every stage, enforcement and
    restriction after every step, one global dt from the finest level)."""
    dx = 0.3
    gg, og, lev, ijk, origin = mesh_pair(name, bc, dx=dx, shuffle=7)
    U, G = mesh_state(gg, lev, ijk, origin, dx, bc, seed=6, base="puncture" if bc == "sommerfeld" else "flat",
                      amp=0.01)
    cp, op = both_params(**PUNC)
    gg.upload(U, G)
    if gg.n_ghost:
        gg.upload(U, G, buf="INI")
    dt = 0.1 * I.level_spacing(dx, og.n_levels)[-1]
    gg.step(cp, dt, 3)
    gU, gG = gg.download("U")
    oU, oG = U, G
    for _ in range(3):
        oU, oG = og.rk4_step(op, dt, oU, oG, G)
    assert rel_err(gU, oU).max() < TOL
    assert rel_err(gG, oG).max() < TOL
    # graph replay is bit-identical to the plain launches
    gg.upload(U, G)
    gg.step_graph(cp, dt, 3)
    hU, hG = gg.download("U")
    np.testing.assert_array_equal(hU, gU)
    np.testing.assert_array_equal(hG, gG)


def test_mesh_constraints_count_leaf_points_only():
    import torch
    dx = 0.3
    gg, og, lev, ijk, origin = mesh_pair("three", "sommerfeld", dx=dx, shuffle=1)
    U, G = mesh_state(gg, lev, ijk, origin, dx, "sommerfeld", seed=8, base="puncture")
    gg.upload(U, G)
    H = torch.zeros(gg.n_points, dtype=torch.float64, device="cuda")
    M = torch.zeros(3 * gg.n_points, dtype=torch.float64, device="cuda")
    out = gg.constraints("U", H.data_ptr(), M.data_ptr())
    oH, oM, oout = og.constraints(U, G)
    h = H.cpu().numpy()
    m = M.cpu().numpy().reshape(3, -1)
    assert np.abs(h - oH.ravel()).max() / max(np.abs(oH).max(), 1.0) < TOL
    assert np.abs(m - oM.reshape(3, -1)).max() / max(np.abs(oM).max(), 1.0) < TOL
    np.testing.assert_allclose(out[:4], oout[:4], rtol=1e-12)
    assert gg.n_leaf_points < gg.n_points


def test_mesh_mixed_precision_tracks_fp64():
    """The mixed path on a mesh stays within the mixed tolerance of FP64."""
    from paper_2406_11626_gb300 import ccz4 as C
    dx = 0.3
    out = []
    for prec in ("fp64", "mixed"):
        gg, og, lev, ijk, origin = mesh_pair("three", "sommerfeld", dx=dx)
        U, G = mesh_state(gg, lev, ijk, origin, dx, "sommerfeld", seed=6, base="puncture", amp=0.01)
        gg.upload(U, G)
        gg.upload(U, G, buf="INI")
        P = C.make_params(**PUNC, precision=prec)
        gg.step(P, 0.1 * I.level_spacing(dx, 3)[-1], 3)
        out.append(gg.download("U")[0])
    assert rel_err(out[1], out[0]).max() < 1e-5


def test_mesh_rejected_on_invalid_nesting():
    from paper_2406_11626_gb300 import ccz4 as C
    lev, ijk = I.refined_mesh((4, 4, 4), [((0, 1, 1), (2, 3, 3))])
    with pytest.raises(C.CCZ4Error) as e:
        C.Grid(6, (4, 4, 4), ijk, (0, 0, 0), 0.1, "copy", level=lev)
    assert e.value.code == C.ERR_INVALID


@pytest.mark.slow
def test_three_level_puncture_full_size_sampled_parity():
    """The three-level puncture workload (7552 patches of 9^3, levels at
    dx = 1/9, 1/27, 1/81) in the launch configuration the benchmark times:
    after one fused RK stage the accumulator holds k0; sampled points of
    every level, including those whose stencils reach interpolated halos,
    agree with the oracle evaluated point by point."""
    from paper_2406_11626_gb300 import ccz4 as C
    cfg = I.multilevel_puncture_config()
    g = C.Grid.from_config(cfg)
    og = O.Grid(cfg.p, cfg.np, cfg.ijk(), cfg.origin, cfg.dx, cfg.bc, level=cfg.level)
    U, G = I.initial_state(cfg)
    g.upload(U, G)
    g.upload(U, G, buf="INI")
    P = C.make_params(**cfg.params)
    g.rk_stage(P, 0, cfg.dt)
    acc, _ = g.download("ACC")
    p3 = cfg.p ** 3
    rng = np.random.default_rng(0)
    pts = []
    for l in range(3):
        on = np.nonzero(np.repeat(cfg.level == l, p3))[0]
        pts.append(rng.choice(on, 120, replace=False))
        # points of boundary patches of the level (their stencils reach the interpolated halo)
        sl = cfg.ijk()[cfg.level == l]
        lo, hi = sl.min(axis=0), sl.max(axis=0)
        edge = np.nonzero((cfg.level == l) & ((cfg.ijk() == lo) | (cfg.ijk() == hi)).any(axis=1))[0]
        pts.append(rng.choice(edge, 8, replace=False) * p3 + rng.integers(0, p3, 8))
    pts = np.concatenate(pts)
    ref = og.rhs_points(O.make_params(**cfg.params), U, G, pts)
    got = acc.reshape(I.NV, -1)[:, pts].T
    scale = np.maximum(np.abs(ref).max(axis=0), 1.0)
    assert (np.abs(got - ref) / scale).max() < TOL


@pytest.mark.slow
def test_binary_puncture_full_size_sampled_parity():
    """The four-level binary puncture workload (20296 patches, Bowen-York
    data from the GPU solve) in the bench's launch configuration: after one
    fused RK stage, sampled points of every level (including those next to
    interpolated halos and the punctures' patches) agree with the oracle
    evaluated point by point on the same state."""
    from paper_2406_11626_gb300 import ccz4 as C
    from paper_2406_11626_gb300 import initial_data as ID
    cfg = I.binary_puncture_config(id_n=96, id_tol=1e-8, id_omega=1.97)
    g = C.Grid.from_config(cfg)
    s, B, k = ID.solve_config(cfg)
    assert k > 0
    s.assemble(B, g, "U")
    s.assemble(B, g, "INI")
    U, G = g.download("U")
    og = O.Grid(cfg.p, cfg.np, cfg.ijk(), cfg.origin, cfg.dx, cfg.bc, level=cfg.level)
    P = C.make_params(**cfg.params)
    g.rk_stage(P, 0, cfg.dt)
    acc, _ = g.download("ACC")
    p3 = cfg.p ** 3
    rng = np.random.default_rng(1)
    pts = []
    for l in range(4):
        on = np.nonzero(np.repeat(cfg.level == l, p3))[0]
        pts.append(rng.choice(on, 60, replace=False))
        sl = cfg.ijk()[cfg.level == l]
        lo, hi = sl.min(axis=0), sl.max(axis=0)
        edge = np.nonzero((cfg.level == l) & ((cfg.ijk() == lo) | (cfg.ijk() == hi)).any(axis=1))[0]
        pts.append(rng.choice(edge, 8, replace=False) * p3 + rng.integers(0, p3, 8))
    x, y, z = I.mesh_point_coords(cfg.p, cfg.level, cfg.ijk(), cfg.origin, cfg.dx)
    r = np.minimum(np.sqrt((x - 3) ** 2 + y ** 2 + z ** 2), np.sqrt((x + 3) ** 2 + y ** 2 + z ** 2)).ravel()
    pts.append(np.argsort(r)[:20])
    pts = np.concatenate(pts)
    ref = og.rhs_points(O.make_params(**cfg.params), U, G, pts)
    got = acc.reshape(I.NV, -1)[:, pts].T
    scale = np.maximum(np.abs(ref).max(axis=0), 1.0)
    assert (np.abs(got - ref) / scale).max() < TOL


@pytest.mark.parametrize("name,bc,prec", [("three", "sommerfeld", "fp64"), ("two", "periodic", "fp64"),
                                          ("three", "sommerfeld", "mixed")])
def test_separable_interpolation_equals_entry_by_entry(name, bc, prec, monkeypatch):
    """The halo fill's separable evaluation of the coarse-to-fine
    interpolations (x, y, z passes sharing their results) gives the same
    tiles, bit for bit, as the point-by-point evaluation, and so the same
    states after RK4 steps (in the mixed path the tiles of split pairs and
    the FP32 mixed derivatives taken from interpolated points read back
    from them)."""
    from paper_2406_11626_gb300 import ccz4 as C
    dx = 0.3
    gg, _, lev, ijk, origin = mesh_pair(name, bc, dx=dx, shuffle=5)
    U, G = mesh_state(gg, lev, ijk, origin, dx, bc, seed=4, base="puncture", amp=0.01)
    dt, P = 0.1 * I.level_spacing(dx, int(np.max(lev)) + 1)[-1], C.make_params(**dict(PUNC, precision=prec))
    out = []
    for by_entry in ("0", "1"):
        monkeypatch.setenv("CCZ4_MESH_INTERP_BY_ENTRY", by_entry)
        g = C.Grid(gg.p, gg.np, ijk, origin, dx, bc, level=lev)
        g.upload(U, G)
        if bc == "sommerfeld":
            g.upload(U, G, buf="INI")
        g.fill_halos("U", P=P)
        tiles = g.download("TILE")
        g.step(P, dt, 2)
        out.append((tiles, g.download("U")))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1][0], out[1][1][0])
    np.testing.assert_array_equal(out[0][1][1], out[1][1][1])


@pytest.mark.parametrize("mesh", [None, "three"])
def test_queue_launch_is_bit_identical_to_flat(mesh):
    """The persistent work-queue launch of the stage kernel computes every
    point exactly as the flat launch (plain steps and graph replays)."""
    from paper_2406_11626_gb300 import ccz4 as C
    if mesh is None:
        cfg = I.single_puncture_config(p=6, n_side=4, half_width=2.0)
        make = lambda: C.Grid.from_config(cfg)
        U, G = I.initial_state(cfg)
        dt, P = cfg.dt, C.make_params(**cfg.params)
    else:
        dx = 0.3
        gg, _, lev, ijk, origin = mesh_pair(mesh, "sommerfeld", dx=dx)
        U, G = mesh_state(gg, lev, ijk, origin, dx, "sommerfeld", seed=2, base="puncture", amp=0.01)
        make = lambda: C.Grid(6, (4, 4, 4), ijk, origin, dx, "sommerfeld", level=lev)
        dt, P = 0.1 * I.level_spacing(dx, 3)[-1], C.make_params(**PUNC)
    out = []
    for launch in ("flat", "queue"):
        for graph in (False, True):
            g = make()
            g.set_launch(launch)
            g.upload(U, G)
            g.upload(U, G, buf="INI")
            (g.step_graph if graph else g.step)(P, dt, 2)
            out.append(g.download("U"))
    for o in out[1:]:
        np.testing.assert_array_equal(o[0], out[0][0])
        np.testing.assert_array_equal(o[1], out[0][1])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("mesh", [False, True])
def test_fixed_edge_stage_kernel_is_bit_identical_to_the_general_one(prec, mesh):
    """Grids of 9^3 patches take the stage kernel compiled for that edge on
    the flat default launch; the queue launch and the other launch shapes
    take the general one; the fused launch runs the fill and the stage of
    that edge in one cooperative kernel. All compute the same steps bit for
    bit."""
    from paper_2406_11626_gb300 import ccz4 as C
    if mesh:
        cfg = I.multilevel_puncture_config(p=9, n_side=4, half_width=2.0, boxes=[((1, 1, 1), (3, 3, 3))])
    else:
        cfg = I.single_puncture_config(p=9, n_side=3, half_width=1.5)
    U, G = I.initial_state(cfg)
    P = C.make_params(**cfg.params, precision=prec)
    out = []
    for launch, shape in (("flat", 0), ("queue", 0), ("flat", 1), ("fused", 0)):
        g = C.Grid.from_config(cfg)
        g.set_launch(launch)
        g.set_tuning(shape, 0)
        g.upload(U, G)
        g.upload(U, G, buf="INI")
        g.step_graph(P, cfg.dt, 2)
        out.append(g.download("U"))
        g.close()
    for o in out[1:]:
        np.testing.assert_array_equal(o[0], out[0][0])
        np.testing.assert_array_equal(o[1], out[0][1])


def test_constraint_norms_away_from_the_punctures_match_oracle():
    """ccz4_constraints_excluding on the per-point monitors of a shuffled
    three-level mesh against og_constraints_excluding: the point counts are
    equal and the norms agree to the monitors' own parity."""
    import torch
    dx = 0.3
    gg, og, lev, ijk, origin = mesh_pair("three", "sommerfeld", dx=dx, shuffle=3)
    U, G = mesh_state(gg, lev, ijk, origin, dx, "sommerfeld", seed=5, base="puncture")
    gg.upload(U, G)
    H = torch.zeros(gg.n_points, dtype=torch.float64, device="cuda")
    M = torch.zeros(3 * gg.n_points, dtype=torch.float64, device="cuda")
    out = gg.constraints("U", H.data_ptr(), M.data_ptr())
    oH, oM, _ = og.constraints(U, G)
    centres = [(0.0, 0.0, 0.0), (0.9, -0.3, 0.2)]
    for radius in (0.0, 0.6, 1.0):
        e = gg.constraints_excluding(H.data_ptr(), M.data_ptr(), centres, radius)
        oe = og.constraints_excluding(oH, oM, centres, radius)
        assert e[4] == oe[4] and e[4] > 0
        np.testing.assert_allclose(e[:4], oe[:4], rtol=1e-10)
    np.testing.assert_allclose(gg.constraints_excluding(H.data_ptr(), M.data_ptr(), centres, 0.0)[:4], out[:4],
                               rtol=1e-13)
    # repeated calls agree bit for bit (fixed reduction order)
    a = gg.constraints_excluding(H.data_ptr(), M.data_ptr(), centres, 0.6)
    b = gg.constraints_excluding(H.data_ptr(), M.data_ptr(), centres, 0.6)
    assert np.array_equal(a, b)


@pytest.mark.slow
def test_binary_mixed_run_tracks_fp64():
    """The four-level binary puncture workload itself: 20 RK4 steps in FP64
    and in the mixed precision from the same Bowen-York data; every field of
    the mixed state is within 1e-5 of the FP64 one (relative to its scale)
    and the constraint norms, over all leaf points and away from the
    punctures (r >= 1), agree within a factor of 2 (measured: to ~1e-7)."""
    import torch
    from paper_2406_11626_gb300 import ccz4 as C
    from paper_2406_11626_gb300 import initial_data as ID
    cfg = I.binary_puncture_config(id_n=96, id_tol=1e-8, id_omega=1.97)
    s, B, _ = ID.solve_config(cfg)
    res = {}
    for prec in ("fp64", "mixed"):
        g = C.Grid.from_config(cfg)
        s.assemble(B, g, "U")
        s.assemble(B, g, "INI")
        g.step_graph(C.make_params(**cfg.params, precision=prec), cfg.dt, 20)
        H = torch.zeros(g.n_points, dtype=torch.float64, device="cuda")
        M = torch.zeros(3 * g.n_points, dtype=torch.float64, device="cuda")
        out = g.constraints("U", H.data_ptr(), M.data_ptr())
        ex = g.constraints_excluding(H.data_ptr(), M.data_ptr(), [(-3.0, 0, 0), (3.0, 0, 0)], 1.0)
        res[prec] = (g.download("U")[0], out, ex)
        g.close()
    assert rel_err(res["mixed"][0], res["fp64"][0]).max() < 1e-5
    for k in (1, 2):
        for q in (0, 1):
            a, b = res["mixed"][k][q], res["fp64"][k][q]
            assert 0.5 < a / b < 2.0 and abs(a / b - 1.0) < 1e-4


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("graph", [False, True])
def test_fused_stage_launch_with_more_patches_than_blocks_is_bit_identical(prec, graph):
    """The fused launch on 12^3 patches of 9^3 (more patches than resident
    blocks, so each block fills several, and more 32-point items than warps)
    with Sommerfeld ghost cells: plain steps and a replayed step graph equal
    the separate fill and stage launches bit for bit."""
    from paper_2406_11626_gb300 import ccz4 as C
    cfg = I.single_puncture_config(p=9, n_side=12, half_width=6.0)
    U, G = I.initial_state(cfg)
    P = C.make_params(**cfg.params, precision=prec)
    out = []
    for launch in ("flat", "fused"):
        g = C.Grid.from_config(cfg)
        g.set_launch(launch)
        g.upload(U, G)
        g.upload(U, G, buf="INI")
        (g.step_graph if graph else g.step)(P, cfg.dt, 3)
        out.append(g.download("U"))
        g.close()
    np.testing.assert_array_equal(out[1][0], out[0][0])
    np.testing.assert_array_equal(out[1][1], out[0][1])


def test_fused_stage_launch_needs_9_cubed_patches():
    from paper_2406_11626_gb300 import ccz4 as C
    cfg = I.single_puncture_config(p=6, n_side=4, half_width=2.0)
    g = C.Grid.from_config(cfg)
    with pytest.raises(C.CCZ4Error, match="9\\^3"):
        g.set_launch("fused")
    g.set_launch("flat")
    g.close()
