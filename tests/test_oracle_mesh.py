"""Pins of the oracle's statically refined mesh (appendix "refinement
transition" of the paper): ratio-3 levels, coarse-to-fine interpolation of
the halo, fine-to-coarse restriction, per-level spacing and the leaf-only
constraint norms."""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2406_11626_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "refinement_transfer_matrices.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, *vals = line.split()
        out.setdefault(name, []).append([float(Fraction(v)) for v in vals])
    return {k: np.array(v) for k, v in out.items()}


def _two_level(p=6, np_=(4, 4, 4), dx=0.1, origin=(0.0, 0.0, 0.0), bc="copy"):
    lev, ijk = I.refined_mesh(np_, [((1, 1, 1), (3, 3, 3))])
    return O.Grid(p, np_, ijk, origin, dx, bc, level=lev), lev, ijk


def _three_level(p=6, np_=(4, 4, 4), dx=0.1, origin=(0.0, 0.0, 0.0), bc="copy"):
    lev, ijk = I.refined_mesh(np_, [((1, 1, 1), (3, 3, 3)), ((4, 4, 4), (5, 5, 5))])
    return O.Grid(p, np_, ijk, origin, dx, bc, level=lev), lev, ijk


def _patch_of(g, lev, ijk, l, slot):
    for n in range(g.n_patches):
        if lev[n] == l and tuple(ijk[n]) == tuple(slot):
            return n
    raise KeyError(slot)


def _tile_value(tiles, g, ijk, n, v, x, y, z):
    """Tile entry of patch n at global point (x, y, z) of the patch's level."""
    p = g.p
    lx, ly, lz = (c - ijk[n][d] * p + 3 for d, c in enumerate((x, y, z)))
    return tiles[v, n, lz, ly, lx]


def _coarse_set(U, g, lev, ijk, l, fn):
    """U[v] on every level-l point <- fn(x, y, z) of its global level-l coordinates."""
    p = g.p
    r = np.arange(p)
    for n in np.nonzero(lev == l)[0]:
        a, b, c = ijk[n]
        X = (a * p + r)[None, None, :]
        Y = (b * p + r)[None, :, None]
        Z = (c * p + r)[:, None, None]
        U[:, n] = fn(X, Y, Z)


def test_mesh_rules_are_enforced():
    """Refined patches come in complete child sets, keep two coarse cells of
    coarse data around their halo and stay away from the domain boundary."""
    _two_level()
    _three_level()
    for boxes in ([((0, 1, 1), (2, 3, 3))], [((1, 1, 1), (4, 3, 3))],
                  [((1, 1, 1), (3, 3, 3)), ((3, 4, 4), (4, 5, 5))]):
        lev, ijk = I.refined_mesh((4, 4, 4), boxes)
        with pytest.raises(ValueError):
            O.Grid(6, (4, 4, 4), ijk, (0, 0, 0), 0.1, "copy", level=lev)
    lev, ijk = I.refined_mesh((4, 4, 4), [((1, 1, 1), (3, 3, 3))])
    keep = np.ones(len(lev), bool)
    keep[np.nonzero(lev == 1)[0][5]] = False  # an incomplete child set
    with pytest.raises(ValueError):
        O.Grid(6, (4, 4, 4), ijk[keep], (0, 0, 0), 0.1, "copy", level=lev[keep])


def test_interpolation_weights_are_the_printed_P_perp_columns():
    """A plane impulse on coarse layer c_j (constant along the face) reaches
    the fine ghost layers f0, f1, f2 with the weights of column j of P^perp."""
    P = _golden()["P_perp"]
    g, lev, ijk = _two_level()
    n = _patch_of(g, lev, ijk, 1, (3, 4, 4))  # lower-x face of the refined block
    for j in range(6):
        U = np.zeros(g.ushape)
        _coarse_set(U, g, lev, ijk, 0, lambda X, Y, Z: np.broadcast_to(
            (X == 3 + j).astype(float), (I.NV, 6, 6, 6)))
        tiles = g.fill_tiles(U)
        for row, fx in enumerate((15, 16, 17)):
            for fy, fz in ((25, 26), (27, 28), (24, 29)):
                got = _tile_value(tiles, g, ijk, n, 4, fx, fy, fz)
                assert got == pytest.approx(P[row, j], abs=1e-15), (j, row)


def test_interpolation_weights_are_the_printed_P_par_rows():
    """Along the face, a plane impulse on coarse cell j of the face reaches
    fine cell i (i = 1..5 from the face start) with P^par[i][j]."""
    P = _golden()["P_par"]
    g, lev, ijk = _two_level()
    n = _patch_of(g, lev, ijk, 1, (3, 3, 4))
    Y0 = 6  # first coarse y cell of the refined block; fine y = 3 * Y0 + i
    for j in range(3):
        U = np.zeros(g.ushape)
        _coarse_set(U, g, lev, ijk, 0, lambda X, Y, Z: np.broadcast_to(
            (Y == Y0 + j).astype(float), (I.NV, 6, 6, 6)))
        tiles = g.fill_tiles(U)
        for i in range(1, 6):
            # fine x = 16 is ghost layer f1 (weight one on c2), fine z = 28 inside
            got = _tile_value(tiles, g, ijk, n, 0, 16, 3 * Y0 + i, 28)
            assert got == pytest.approx(P[i - 1, j], abs=1e-15), (i, j)


def test_restriction_weights_are_the_printed_R_average_product():
    """An impulse on one fine cell restricts to R[x] R[y] R[z] on the coarse
    cell above it, and to zero on the other coarse cells of the block;
    coarse cells outside the refined block are untouched."""
    R = _golden()["R_avg"]
    g, lev, ijk = _two_level()
    rng = np.random.default_rng(4)
    for fx, fy, fz in ((19, 22, 25), (18, 18, 18), (35, 30, 20)):
        U = rng.standard_normal(g.ushape)
        fine = lev == 1
        U[:, fine] = 0.0
        n = None
        for m in np.nonzero(fine)[0]:
            a, b, c = ijk[m]
            if a * 6 <= fx < a * 6 + 6 and b * 6 <= fy < b * 6 + 6 and c * 6 <= fz < c * 6 + 6:
                n = m
        U[:, n, fz - ijk[n][2] * 6, fy - ijk[n][1] * 6, fx - ijk[n][0] * 6] = 1.0
        out = g.restrict(U)
        X, Y, Z = fx // 3, fy // 3, fz // 3
        want = R[0, fx - 3 * X] * R[0, fy - 3 * Y] * R[0, fz - 3 * Z]
        for m in np.nonzero(lev == 0)[0]:
            a, b, c = ijk[m]
            refined = all(1 <= s < 3 for s in (a, b, c))
            if not refined:
                np.testing.assert_array_equal(out[:, m], U[:, m])
                continue
            blk = out[0, m].copy()
            if a * 6 <= X < a * 6 + 6 and b * 6 <= Y < b * 6 + 6 and c * 6 <= Z < c * 6 + 6:
                loc = (Z - c * 6, Y - b * 6, X - a * 6)
                assert blk[loc] == pytest.approx(want, rel=1e-15)
                blk[loc] = 0.0
            assert np.all(blk == 0.0)


def _has_children(lev, ijk):
    kids = {(int(l) - 1,) + tuple(int(c) // 3 for c in s) for l, s in zip(lev, ijk) if l > 0}
    return np.array([(int(l),) + tuple(int(c) for c in s) in kids for l, s in zip(lev, ijk)])


def _trilinear(seed):
    rng = np.random.default_rng(seed)
    coef = rng.uniform(-1, 1, (I.NV, 8))

    def f(x, y, z):
        terms = [np.ones_like(x), x, y, z, x * y, x * z, y * z, x * y * z]
        return np.stack([sum(c[k] * terms[k] for k in range(8)) for c in coef])
    return f


def _tile_positions(g, ijk, lev, n, origin, dx):
    h = I.level_spacing(dx, g.n_levels)[lev[n]]
    T = g.p + 6
    r = np.arange(T) - 3
    xs = origin[0] + (ijk[n][0] * g.p + r + 0.5) * h
    ys = origin[1] + (ijk[n][1] * g.p + r + 0.5) * h
    zs = origin[2] + (ijk[n][2] * g.p + r + 0.5) * h
    return (np.broadcast_to(xs[None, None, :], (T, T, T)), np.broadcast_to(ys[None, :, None], (T, T, T)),
            np.broadcast_to(zs[:, None, None], (T, T, T)))


@pytest.mark.parametrize("mesh", [_two_level, _three_level])
def test_interpolation_and_restriction_are_exact_for_trilinear_fields(mesh):
    """Linear interpolation between cell centres, applied along each axis,
    reproduces any polynomial of degree one in each variable; so does the
    27-cell mean (the midpoint rule along each axis). A wrong weight, a
    shifted coarse cell or a wrong level spacing breaks both."""
    origin, dx = (-1.3, -0.7, -0.2), 0.1
    g, lev, ijk = mesh(origin=origin, dx=dx)
    f = _trilinear(1)
    x, y, z = I.mesh_point_coords(g.p, lev, ijk, origin, dx)
    U = f(x, y, z)
    tiles = g.fill_tiles(U)
    for n in range(g.n_patches):
        if lev[n] == 0:
            continue
        X, Y, Z = _tile_positions(g, ijk, lev, n, origin, dx)
        np.testing.assert_allclose(tiles[:, n], f(X, Y, Z), rtol=0, atol=1e-13)
    # restriction: perturb the coarse points under fine patches, then restore
    V = U.copy()
    V[:, _has_children(lev, ijk)] += 0.37
    out = g.restrict(V)
    np.testing.assert_allclose(out, U, rtol=0, atol=1e-13)


def test_interpolation_error_of_a_quadratic_has_its_closed_form():
    """Linear interpolation of x^2 between nodes h apart, at fraction t of
    the way, overshoots by exactly h^2 t (1 - t); the tensor product adds
    these per axis. So for f = x^2 + 2 y^2 + 3 z^2 every interpolated ghost
    value of the fine level exceeds f by h_c^2 (e_x + 2 e_y + 3 e_z), e_d =
    t_d (1 - t_d) with t_d = ((i_d - 1) mod 3) / 3 for fine index i_d, and
    every covered tile point is exact."""
    origin, dx = (-1.1, -0.6, -0.9), 0.1
    g, lev, ijk = _two_level(origin=origin, dx=dx)
    x, y, z = I.mesh_point_coords(g.p, lev, ijk, origin, dx)

    def f(x, y, z):
        v = x * x + 2.0 * y * y + 3.0 * z * z
        return np.broadcast_to(v, (I.NV,) + v.shape)
    tiles = g.fill_tiles(f(x, y, z))
    T = g.p + 6
    lo, hi = 18, 54  # fine cells of the refined block along each axis
    n_interp = 0
    for n in np.nonzero(lev == 1)[0]:
        X, Y, Z = _tile_positions(g, ijk, lev, n, origin, dx)
        idx = [ijk[n][d] * g.p + np.arange(T) - 3 for d in range(3)]
        t = [((i - 1) % 3) / 3.0 for i in idx]
        e = [tt * (1.0 - tt) for tt in t]
        err = dx * dx * (e[0][None, None, :] + 2.0 * e[1][None, :, None] + 3.0 * e[2][:, None, None])
        outside = ((idx[0] < lo) | (idx[0] >= hi))[None, None, :] | ((idx[1] < lo) | (idx[1] >= hi))[None, :, None] | \
            ((idx[2] < lo) | (idx[2] >= hi))[:, None, None]
        want = f(X, Y, Z)[0] + np.where(outside, err, 0.0)
        np.testing.assert_allclose(tiles[0, n], want, rtol=0, atol=1e-13)
        n_interp += int(outside.sum())
    assert n_interp > 1000


def _trilinear_state(seed):
    """A CCZ4 state whose every field is a polynomial of degree one in each
    variable (the FD4 stencils are exact on it, the KO sum vanishes)."""
    f = _trilinear(seed)

    def state(x, y, z):
        U = 0.02 * f(x, y, z)
        for v in I._FLAT_ONES:
            U[v] += 1.0
        return U
    return state


@pytest.mark.parametrize("mesh", [_two_level, _three_level])
def test_rhs_on_the_mesh_equals_the_uniform_grid_of_each_level(mesh):
    """With trilinear data every tile value of every level is the data
    itself, so the right-hand side at a point of level l equals that of a
    uniform grid of spacing dx / 3^l around the same point: this pins the
    per-level spacing and the interpolated halo inside the full RHS."""
    origin, dx = (-1.2, -1.2, -1.2), 0.1
    g, lev, ijk = mesh(origin=origin, dx=dx)
    P = O.make_params(**I.PUNCTURE_PARAMS)
    st = _trilinear_state(2)
    x, y, z = I.mesh_point_coords(g.p, lev, ijk, origin, dx)
    U = st(x, y, z)
    rU, _ = g.rhs(P, U)
    hs = I.level_spacing(dx, g.n_levels)
    rng = np.random.default_rng(0)
    p3 = g.p ** 3
    N0 = g.p * 4
    for l in range(g.n_levels):
        cand = []
        for pt in np.nonzero(np.repeat(lev == l, p3))[0]:
            n, q = divmod(int(pt), p3)
            kz, r = divmod(q, g.p * g.p)
            ky, kx = divmod(r, g.p)
            gl = [ijk[n][0] * g.p + kx, ijk[n][1] * g.p + ky, ijk[n][2] * g.p + kz]
            # level 0: keep the stencil off the copied boundary layers
            if l > 0 or all(3 <= c < N0 - 3 for c in gl):
                cand.append((n, kz, ky, kx, gl))
        picks = list(rng.choice(len(cand), 6, replace=False))
        if l > 0:
            # and points whose stencil reaches the interpolated halo
            sl = ijk[lev == l]
            lo, hi = sl.min(axis=0) * g.p, (sl.max(axis=0) + 1) * g.p
            near = [k for k, c in enumerate(cand) if any(c[4][d] - lo[d] < 3 or hi[d] - 1 - c[4][d] < 3
                                                          for d in range(3))]
            picks += list(rng.choice(near, 6, replace=False))
        for k in picks:
            n, kz, ky, kx, _ = cand[k]
            pos = np.array([x[n, kz, ky, kx], y[n, kz, ky, kx], z[n, kz, ky, kx]])
            # a lone 7^3 patch centred on the point, spacing of level l
            h = hs[l]
            o = pos - 3.5 * h
            u = O.Grid(7, (1, 1, 1), [[0, 0, 0]], tuple(o), h, "copy")
            ux, uy, uz = I.point_coords(7, [[0, 0, 0]], tuple(o), h)
            Uu = st(ux, uy, uz)
            ref = u.rhs_points(P, Uu, None, [3 * 49 + 3 * 7 + 3])[0]
            got = rU[:, n, kz, ky, kx]
            np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-11)


def test_flat_space_stays_flat_on_a_refined_mesh():
    g, lev, ijk = _three_level(bc="sommerfeld")
    P = O.make_params(**I.PUNCTURE_PARAMS)
    U = I.flat(g.ushape[1:])
    G = I.flat((g.n_ghost,))
    U1, G1 = g.rk4_step(P, 0.01, U, G, G)
    np.testing.assert_array_equal(U1, U)
    np.testing.assert_array_equal(G1, G)


def test_constraint_norms_count_leaf_points_only():
    """H and M are returned for every point; the L2 norms run over the
    points of leaf patches only (a point a finer level covers is not counted
    twice)."""
    origin, dx = (-1.2, -1.2, -1.2), 0.1
    g, lev, ijk = _two_level(origin=origin, dx=dx)
    x, y, z = I.mesh_point_coords(g.p, lev, ijk, origin, dx)
    U = I.smooth_perturbation(x, y, z, seed=3, amp=1e-2, box=2.4)
    H, M, out = g.constraints(U)
    parent = _has_children(lev, ijk)
    assert parent.sum() == 8
    leaf = ~parent
    h = H[leaf].ravel()
    m2 = (M[:, leaf] ** 2).sum(axis=0).ravel()
    assert out[0] == pytest.approx(np.sqrt(np.mean(h ** 2)), rel=1e-12)
    assert out[1] == pytest.approx(np.sqrt(np.mean(m2)), rel=1e-12)
    assert np.abs(H[parent]).max() > 0.0  # written, just not counted


def _rotate_levels(U, g, lev, ijk, R):
    """Rotate a mesh state by the lattice rotation R about the domain centre.
    Every level's block is centred, so each level maps onto itself; the
    level's points are rotated as a cell-centred cube (scalars move, vectors
    and tensors rotate)."""
    from test_oracle_rhs_pins import _rotate_state
    p = g.p
    out = np.empty_like(U)
    for l in range(g.n_levels):
        sel = np.nonzero(lev == l)[0]
        lo = ijk[sel].min(axis=0)
        n = (ijk[sel].max(axis=0) - lo + 1) * p
        assert n[0] == n[1] == n[2]
        N = int(n[0])
        Q = np.full((I.NV, N, N, N), np.nan)
        for m in sel:
            a, b, c = (ijk[m] - lo) * p
            Q[:, c:c + p, b:b + p, a:a + p] = U[:, m]
        Qr = _rotate_state(Q, R, N)
        for m in sel:
            a, b, c = (ijk[m] - lo) * p
            out[:, m] = Qr[:, c:c + p, b:b + p, a:a + p]
    return out


@pytest.mark.parametrize("R", [np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]]),
                               np.array([[0, 0, 1], [1, 0, 0], [0, 1, 0]])])
def test_a_step_on_a_symmetric_mesh_is_rotation_covariant(R):
    """One RK4 step on a three-level mesh with centred blocks (halo
    interpolation, per-level spacing, enforcement and restriction all
    included) commutes with a lattice rotation of the data, up to rounding.
    A transposed axis or a one-sided index in the level transfer breaks it."""
    p, np_, dx = 6, (4, 4, 4), 0.25
    lev, ijk = I.refined_mesh(np_, [((1, 1, 1), (3, 3, 3)), ((5, 5, 5), (7, 7, 7))])
    origin = (-3.0, -3.0, -3.0)
    g = O.Grid(p, np_, ijk, origin, dx, "periodic", level=lev)
    x, y, z = I.mesh_point_coords(p, lev, ijk, origin, dx)
    U = I.smooth_perturbation(x, y, z, seed=5, amp=0.03, box=6.0)
    P = O.make_params(**I.PUNCTURE_PARAMS)
    dt = 0.1 * I.level_spacing(dx, 3)[-1]
    U1, _ = g.rk4_step(P, dt, U)
    Ur1, _ = g.rk4_step(P, dt, _rotate_levels(U, g, lev, ijk, R))
    expect = _rotate_levels(U1, g, lev, ijk, R)
    np.testing.assert_allclose(Ur1, expect, rtol=0, atol=1e-12 * np.abs(U1).max())
    assert np.abs(U1 - U).max() > 1e-6  # the step did move the data


def test_constraint_norms_away_from_the_punctures():
    """The norms that leave out the balls r < radius around the punctures:
    radius 0 gives the monitor's own leaf-point norms; otherwise they equal
    a brute-force mean over the leaf points outside every ball (positions
    from the cell centres of each level); a ball over everything leaves no
    point."""
    lev, ijk = I.refined_mesh((4, 4, 4), [((1, 1, 1), (3, 3, 3))], permute_seed=6)
    p, origin, dx = 6, (-2.0, -2.0, -2.0), 1.0 / 6.0
    g = O.Grid(p, (4, 4, 4), ijk, origin, dx, "sommerfeld", level=lev)
    x, y, z = I.mesh_point_coords(p, lev, ijk, origin, dx)
    U = I.smooth_perturbation(x, y, z, seed=4, amp=1e-2, box=4.0,
                              base=I.brill_lindquist(x, y, z, (0.5, 0.5), ((-0.7, 0.1, 0.0), (0.7, -0.1, 0.0))))
    gx, gy, gz = I.ghost_positions((24, 24, 24), origin, dx)
    G = I.brill_lindquist(gx, gy, gz, (0.5, 0.5), ((-0.7, 0.1, 0.0), (0.7, -0.1, 0.0)))
    H, M, out = g.constraints(U, G)
    centres = [(-0.7, 0.1, 0.0), (0.7, -0.1, 0.0)]
    e0 = g.constraints_excluding(H, M, centres, 0.0)
    np.testing.assert_allclose(e0[:4], out[:4], rtol=1e-13)
    # brute force: leaf patches (no children) and the points outside both balls
    kids = {tuple(c // 3) for c in ijk[lev == 1]}
    leaf = np.array([not (l == 0 and tuple(c) in kids) for l, c in zip(lev, ijk)])
    for radius in (0.5, 1.0):
        far = np.ones(x.shape, dtype=bool)
        for c in centres:
            far &= (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2 >= radius ** 2
        sel = far & leaf[:, None, None, None]
        h, m2 = H[sel], (M ** 2).sum(axis=0)[sel]
        e = g.constraints_excluding(H, M, centres, radius)
        assert e[4] == sel.sum() and 0 < e[4] < leaf.sum() * p ** 3
        np.testing.assert_allclose(e[:4], [np.sqrt(np.mean(h ** 2)), np.sqrt(np.mean(m2)), np.abs(h).max(),
                                           np.sqrt(m2).max()], rtol=1e-12)
    assert g.constraints_excluding(H, M, centres, 100.0)[4] == 0.0
