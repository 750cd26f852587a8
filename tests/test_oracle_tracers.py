"""Pins of the oracle's particle tracers (Sec. "Particle Tracers as Data
Probes": trilinear projection from the 2^3 closest sample points, explicit
Euler moves with a projected velocity; puncture trackers use the opposite
shift). Each pin holds against mathematics, not against the oracle itself:

- trilinear interpolation reproduces every trilinear function exactly, so a
  wrong weight, a transposed axis or an off-by-one corner fails it;
- on a refined mesh the finest level that holds all eight corners is used,
  found here by brute force over the patch slots of each level;
- an Euler step with a linear shift field moves a tracer to x - dt beta(x);
- a periodic wrap takes the corner across the boundary (brute force on the
  global array);
- a tracer outside what level 0 resolves is reported and stays in place.
"""
import numpy as np

import oracle as O
from paper_2406_11626_gb300 import inputs as I

NV = I.NV


def _trilinear_coeffs(seed):
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=(NV, 8))


def _trilinear(c, x, y, z):
    """(NV, ...) values of c0 + c1 x + c2 y + c3 z + c4 xy + c5 xz + c6 yz + c7 xyz."""
    x, y, z = (np.asarray(v, dtype=np.float64) for v in (x, y, z))
    terms = np.stack([np.ones_like(x), x, y, z, x * y, x * z, y * z, x * y * z])
    return np.tensordot(c, terms, axes=(1, 0))


def _uniform(bc="sommerfeld", p=6, n=3, half=1.5):
    ijk = I.patch_ijk((n, n, n), permute_seed=3)
    dx = 2.0 * half / (n * p)
    origin = (-half,) * 3
    return O.Grid(p, (n, n, n), ijk, origin, dx, bc), ijk, origin, dx


def test_trilinear_data_is_reproduced_exactly_including_the_ghost_shell():
    g, ijk, origin, dx = _uniform()
    c = _trilinear_coeffs(0)
    U = _trilinear(c, *I.point_coords(g.p, ijk, origin, dx))
    N = (g.p * 3,) * 3
    G = _trilinear(c, *I.ghost_positions(N, origin, dx))
    rng = np.random.default_rng(1)
    # corners may reach the outermost ghost cells: positions within the shell's centres
    lo, hi = origin[0] - 2.5 * dx, origin[0] + (N[0] + 2.5) * dx
    pos = rng.uniform(lo, hi, size=(200, 3))
    new, vals, bad = g.tracers_step(U, G, pos)
    assert bad == 0 and np.array_equal(new, pos)
    exact = _trilinear(c, pos[:, 0], pos[:, 1], pos[:, 2]).T
    assert np.abs(vals - exact).max() <= 1e-13 * max(np.abs(exact).max(), 1.0)


def _level_by_brute_force(level, ijk, p, origin, dx, x):
    """Finest level whose patches hold all eight sample points around x."""
    hs = I.level_spacing(dx, int(level.max()) + 1)
    for l in range(len(hs) - 1, 0, -1):
        slots = {tuple(s) for s in ijk[level == l]}
        i0 = np.floor((np.asarray(x) - np.asarray(origin)) / hs[l] - 0.5).astype(int)
        corners = [i0 + np.array([a, b, c]) for c in (0, 1) for b in (0, 1) for a in (0, 1)]
        if all(tuple(k // p) in slots and (k >= 0).all() for k in corners):
            return l
    return 0


def test_mesh_projection_uses_the_finest_level_holding_all_corners():
    lev, ijk = I.refined_mesh((4, 4, 4), [((1, 1, 1), (3, 3, 3)), ((4, 4, 4), (6, 6, 5))], permute_seed=2)
    p, origin, dx = 6, (-2.0, -2.0, -2.0), 1.0 / 6.0
    g = O.Grid(p, (4, 4, 4), ijk, origin, dx, "sommerfeld", level=lev)
    c = _trilinear_coeffs(4)
    x, y, z = I.mesh_point_coords(p, lev, ijk, origin, dx)
    # trilinear data plus 1000 x (level of the patch): the projection tells its level apart
    U = _trilinear(c, x, y, z) + 1000.0 * lev.reshape(1, -1, 1, 1, 1)
    G = _trilinear(c, *I.ghost_positions((24, 24, 24), origin, dx))
    rng = np.random.default_rng(5)
    pos = np.concatenate([rng.uniform(-1.9, 1.9, size=(300, 3)),
                          # around the finest level's box, [-2/3, 0]^2 x [-2/3, -1/3], and its edges
                          rng.uniform((-0.75, -0.75, -0.7), (0.05, 0.05, -0.3), size=(300, 3))])
    _, vals, bad = g.tracers_step(U, G, pos)
    assert bad == 0
    L = np.array([_level_by_brute_force(lev, ijk, p, origin, dx, q) for q in pos])
    assert set(L) == {0, 1, 2}
    exact = _trilinear(c, pos[:, 0], pos[:, 1], pos[:, 2]).T + 1000.0 * L[:, None]
    assert np.abs(vals - exact).max() <= 1e-11


def test_euler_step_with_a_linear_shift_and_static_probes():
    g, ijk, origin, dx = _uniform(bc="periodic")
    rng = np.random.default_rng(7)
    b0, B = rng.uniform(-0.3, 0.3, 3), rng.uniform(-0.2, 0.2, (3, 3))
    x, y, z = I.point_coords(g.p, ijk, origin, dx)
    U = np.zeros((NV,) + x.shape)
    for i in range(3):
        U[I.IDX["betax"] + i] = b0[i] + B[i, 0] * x + B[i, 1] * y + B[i, 2] * z
    pos = rng.uniform(-1.0, 1.0, size=(50, 3))
    dt = 0.037
    new, vals, bad = g.tracers_step(U, None, pos, dt, I.IDX["betax"], -1.0)
    assert bad == 0
    beta = b0[None, :] + pos @ B.T
    assert np.abs(vals[:, I.IDX["betax"]:I.IDX["betax"] + 3] - beta).max() < 1e-14
    assert np.abs(new - (pos - dt * beta)).max() < 1e-15
    # a static probe records the values and does not move
    same, _, _ = g.tracers_step(U, None, pos, dt, -1)
    assert np.array_equal(same, pos)


def test_periodic_wrap_takes_the_corner_across_the_boundary():
    g, ijk, origin, dx = _uniform(bc="periodic")
    rng = np.random.default_rng(9)
    U = rng.standard_normal((NV, len(ijk), g.p, g.p, g.p))
    # the global array Q[v][z][y][x] of the patches
    n = 3 * g.p
    Q = np.empty((NV, n, n, n))
    for k, (a, b, c) in enumerate(ijk):
        Q[:, c * g.p:(c + 1) * g.p, b * g.p:(b + 1) * g.p, a * g.p:(a + 1) * g.p] = U[:, k]
    pos = np.array([[origin[0] + 0.2 * dx, 0.31, -0.42],          # between x_{N-1} (wrapped) and x_0
                    [origin[0] + (n - 0.3) * dx, origin[1] + 0.1 * dx, origin[2] + (n - 0.05) * dx]])
    _, vals, bad = g.tracers_step(U, None, pos)
    assert bad == 0
    for s, x in enumerate(pos):
        sv = (x - np.asarray(origin)) / dx - 0.5
        i0 = np.floor(sv).astype(int)
        t = sv - i0
        want = np.zeros(NV)
        for c in (0, 1):
            for b in (0, 1):
                for a in (0, 1):
                    w = (t[0] if a else 1 - t[0]) * (t[1] if b else 1 - t[1]) * (t[2] if c else 1 - t[2])
                    want += w * Q[:, (i0[2] + c) % n, (i0[1] + b) % n, (i0[0] + a) % n]
        assert np.abs(vals[s] - want).max() < 1e-14


def test_tracer_outside_the_grid_is_reported_and_stays():
    g, ijk, origin, dx = _uniform()
    c = _trilinear_coeffs(11)
    U = _trilinear(c, *I.point_coords(g.p, ijk, origin, dx))
    G = _trilinear(c, *I.ghost_positions((18, 18, 18), origin, dx))
    pos = np.array([[0.0, 0.0, 0.0], [5.0, 0.0, 0.0], [0.0, np.nan, 0.0]])
    new, vals, bad = g.tracers_step(U, G, pos, 0.1, I.IDX["betax"], -1.0)
    assert bad == 2
    assert np.isfinite(vals[0]).all() and np.isnan(vals[1]).all() and np.isnan(vals[2]).all()
    assert np.array_equal(new[1], pos[1])
