"""Particle tracers and puncture trackers on the GPU (ccz4_tracers_* through
the C ABI) against the oracle's tracers: the projected values and the
positions after several Euler moves are bit-identical (both sides round
every product and sum of the same formula on its own), on a uniform
Sommerfeld grid (tracers reaching into the ghost shell), a periodic grid
(corners across the wrap) and a three-level mesh (the finest level holding
all corners). A tracer outside the grid is reported as CCZ4_ERR_BOUNDS and
left in place, without any out-of-bounds access."""
import numpy as np
import pytest

import oracle as O
from paper_2406_11626_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _perturbed(cfg, seed):
    U, G = I.initial_state(cfg)
    if isinstance(cfg, I.MeshConfig):
        x, y, z = I.mesh_point_coords(cfg.p, cfg.level, cfg.ijk(), cfg.origin, cfg.dx)
    else:
        x, y, z = I.point_coords(cfg.p, cfg.ijk(), cfg.origin, cfg.dx)
    # a shift that moves the tracers
    U = I.smooth_perturbation(x, y, z, seed=seed, amp=5e-2, box=2.0 * abs(cfg.origin[0]), base=U)
    return U, G


def _run(cfg, U, G, pos, steps, dt):
    from paper_2406_11626_gb300 import ccz4 as C
    g = C.Grid.from_config(cfg)
    g.upload(U, G)
    og = O.Grid(cfg.p, cfg.np, cfg.ijk(), cfg.origin, cfg.dx, cfg.bc, level=getattr(cfg, "level", None))
    tr = C.Tracers(g, pos, velocity="shift")
    q = np.array(pos, dtype=np.float64)
    for _ in range(steps):
        tr.step("U", dt)
        q, vo, bad = og.tracers_step(U, G, q, dt, I.IDX["betax"], -1.0)
        assert bad == 0
        pg, vg = tr.read()
        assert np.array_equal(vg, vo)
        assert np.array_equal(pg, q)
    return q


def test_tracers_match_oracle_on_a_sommerfeld_grid_bit_for_bit():
    cfg = I.single_puncture_config(p=6, n_side=3, half_width=1.5)
    U, G = _perturbed(cfg, 1)
    rng = np.random.default_rng(2)
    dx = cfg.dx
    pos = rng.uniform(cfg.origin[0] - 2.4 * dx, -cfg.origin[0] + 2.4 * dx, size=(257, 3))   # ragged count
    q = _run(cfg, U, G, pos, 4, 0.3)
    assert np.abs(q - pos).max() > 1e-3   # they moved


def test_tracers_match_oracle_across_the_periodic_wrap():
    cfg = I.gauge_wave_config(p=6, np_=(3, 3, 3), permute_seed=4)
    U, G = _perturbed(cfg, 3)
    rng = np.random.default_rng(5)
    pos = rng.uniform(-0.5, 0.5, size=(64, 3))
    pos[:8, 0] = -0.5 + rng.uniform(0.0, 0.5, 8) / 18.0   # between the last cell and the first
    _run(cfg, U, G, pos, 3, 0.05)


def test_tracers_match_oracle_on_a_three_level_mesh():
    cfg = I.multilevel_puncture_config(p=6, n_side=4, half_width=2.0,
                                       boxes=[((1, 1, 1), (3, 3, 3)), ((4, 4, 4), (6, 6, 5))])
    U, G = _perturbed(cfg, 7)
    rng = np.random.default_rng(8)
    pos = np.concatenate([rng.uniform(-1.9, 1.9, size=(100, 3)),
                          rng.uniform((-0.75, -0.75, -0.7), (0.05, 0.05, -0.3), size=(100, 3))])
    _run(cfg, U, G, pos, 3, 0.1)


def test_tracer_outside_the_grid_is_reported_and_left_in_place():
    from paper_2406_11626_gb300 import ccz4 as C
    cfg = I.single_puncture_config(p=6, n_side=3, half_width=1.5)
    U, G = _perturbed(cfg, 9)
    g = C.Grid.from_config(cfg)
    g.upload(U, G)
    pos = np.array([[0.1, 0.2, 0.3], [9.0, 0.0, 0.0], [0.0, 0.0, -0.2]])
    tr = C.Tracers(g, pos, velocity="shift")
    tr.step("U", 0.1)
    with pytest.raises(C.CCZ4Error) as e:
        tr.read()
    assert e.value.code == C.ERR_BOUNDS and "outside the grid" in str(e.value)
    p, v = tr.read(raise_bounds=False)
    assert np.array_equal(p[1], pos[1]) and np.isnan(v[1]).all()
    og = O.Grid(cfg.p, cfg.np, cfg.ijk(), cfg.origin, cfg.dx, cfg.bc)
    q, vo, bad = og.tracers_step(U, G, pos, 0.1, I.IDX["betax"], -1.0)
    assert bad == 1 and np.array_equal(p, q) and np.array_equal(v[[0, 2]], vo[[0, 2]])
    # invalid arguments are refused on the host
    with pytest.raises(C.CCZ4Error):
        C.Tracers(g, pos, vel_field=23)
