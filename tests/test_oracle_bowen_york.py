"""Pins of the Bowen-York initial-data oracle: the closed-form curvature of
one puncture, the constraints the Bowen-York curvature satisfies by
construction, the discrete operator and its fall-off ghosts, and the
Hamiltonian constraint of the solved data measured by the (independently
pinned) CCZ4 constraint monitor."""
import numpy as np
import pytest

import oracle as O
from paper_2406_11626_gb300 import inputs as I


def _rand_points(rng, m, c, rmin=0.5, rmax=3.0):
    d = rng.standard_normal((m, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    r = rng.uniform(rmin, rmax, m)
    return c + d * r[:, None], d, r


def test_momentum_curvature_has_its_closed_form():
    """One puncture with momentum P: Abar_ij Abar^ij = 9 P^2 / (2 r^4) (1 + 2 cos^2 t),
    t the angle between n and P (derived from the definition by hand)."""
    rng = np.random.default_rng(0)
    c = np.array([0.3, -0.2, 0.1])
    P = np.array([0.1, -0.25, 0.07])
    B = O.make_punctures([0.7], [c], [P])
    X, n, r = _rand_points(rng, 200, c)
    _, aa, psi = O.by_points(B, X[:, 0], X[:, 1], X[:, 2])
    cos = n @ P / np.linalg.norm(P)
    want = 9.0 * (P @ P) / (2.0 * r ** 4) * (1.0 + 2.0 * cos ** 2)
    np.testing.assert_allclose(aa, want, rtol=1e-12)
    np.testing.assert_allclose(psi, 1.0 + 0.7 / (2.0 * r), rtol=1e-13)


def test_spin_curvature_has_its_closed_form():
    """One puncture with spin S: Abar_ij Abar^ij = 18 S^2 sin^2 t / r^6."""
    rng = np.random.default_rng(1)
    c = np.array([-0.4, 0.0, 0.25])
    S = np.array([0.05, 0.2, -0.1])
    B = O.make_punctures([0.5], [c], None, [S])
    X, n, r = _rand_points(rng, 200, c)
    _, aa, _ = O.by_points(B, X[:, 0], X[:, 1], X[:, 2])
    cos = n @ S / np.linalg.norm(S)
    want = 18.0 * (S @ S) * (1.0 - cos ** 2) / r ** 6
    np.testing.assert_allclose(aa, want, rtol=1e-11, atol=1e-14)


def test_curvature_is_tracefree_and_divergence_free():
    """Bowen-York curvature solves the flat momentum constraint: tr Abar = 0
    and d_j Abar_ij = 0 away from the punctures (divergence by a fourth-order
    central difference, which converges to zero at fourth order)."""
    B = O.make_punctures([0.5, 0.4], [(1.0, 0.0, 0.0), (-1.0, 0.2, 0.0)],
                         [(0.0, 0.2, 0.05), (0.1, -0.2, 0.0)], [(0.0, 0.0, 0.1), (0.05, 0.1, 0.0)])
    rng = np.random.default_rng(2)
    X = rng.uniform(-3, 3, (60, 3))
    X = X[np.minimum(np.linalg.norm(X - [1, 0, 0], axis=1), np.linalg.norm(X - [-1, 0.2, 0], axis=1)) > 0.8]
    A, _, _ = O.by_points(B, X[:, 0], X[:, 1], X[:, 2])
    assert np.abs(A[:, 0] + A[:, 3] + A[:, 5]).max() < 1e-13 * np.abs(A).max()
    sym = [[0, 1, 2], [1, 3, 4], [2, 4, 5]]
    errs = []
    for h in (0.02, 0.01):
        div = np.zeros((len(X), 3))
        for j in range(3):
            e = np.zeros(3)
            e[j] = h
            Ap = [O.by_points(B, *(X + s * e).T)[0] for s in (-2, -1, 1, 2)]
            dA = (Ap[0] - 8 * Ap[1] + 8 * Ap[2] - Ap[3]) / (12 * h)
            for i in range(3):
                div[:, i] += dA[:, sym[i][j]]
        errs.append(np.abs(div).max())
    assert errs[1] < errs[0] / 12.0 and errs[1] < 1e-6, errs


def test_no_momentum_no_spin_gives_u_zero():
    """Without momenta and spins the source vanishes and u = 0 solves the
    discrete equation exactly (Brill-Lindquist data)."""
    B = O.make_punctures([0.5, 0.5], [(1.1, 0.0, 0.0), (-1.1, 0.0, 0.0)])
    u, k, r = O.by_solve(B, 12, 3.0)
    assert k == 0 and r == 0.0 and not u.any()


def test_discrete_operator_and_fall_off_ghosts():
    """Without source, the residual is the 7-point Laplacian: 2 + 4 + 6 = 12
    on x^2 + 2 y^2 + 3 z^2 at every cell away from the faces; for u = C / r
    the ghosts are exact, so boundary cells carry only the small truncation
    error of the interior stencil."""
    n, L = 12, 3.0
    B = O.make_punctures([0.5], [(0.05, 0.0, 0.0)])
    x, y, z = O.by_cell_coords(n, L)
    res, _ = O.by_residual(B, n, L, x * x + 2.0 * y * y + 3.0 * z * z)
    np.testing.assert_allclose(res[1:-1, 1:-1, 1:-1], 12.0, rtol=1e-12)
    r = np.sqrt(x * x + y * y + z * z)
    res, _ = O.by_residual(B, n, L, 0.3 / r)
    face = np.zeros((n, n, n), bool)
    face[[0, -1], :, :] = face[:, [0, -1], :] = face[:, :, [0, -1]] = True
    # a copied ghost (u_ghost = u_cell) would leave u (h / r) / h^2 there,
    # about 8 % of u / h^2 on these faces; a zero ghost all of it
    assert np.abs(res[face]).max() < 0.02 * (0.3 / r[face]).min() / (2 * L / n) ** 2


def test_solved_data_satisfy_the_hamiltonian_constraint():
    """The solved conformal factor, mapped to the CCZ4 variables (phi =
    psi^-2, A~_ij = psi^-6 Abar_ij, g~ = delta, K = 0), makes the CCZ4
    Hamiltonian monitor vanish at second order (the order of the 7-point
    solve) in a shell between the puncture and the outer boundary; with the
    source factor or power wrong it would not vanish."""
    m, c, P = 0.5, (0.02, -0.03, 0.01), (0.0, 0.3, 0.0)
    B = O.make_punctures([m], [c], [P])
    L = 3.0
    hs = []
    for n in (12, 24):
        u, k, r = O.by_solve(B, n, L, tol=1e-11, check=20)
        assert k > 0
        x, y, z = O.by_cell_coords(n, L)
        _, _, psi_bl = O.by_points(B, x, y, z)
        psi = (psi_bl + u.ravel()).reshape(n, n, n)
        # the same cells as a CCZ4 grid of 6^3 patches; the state by the
        # oracle's assembly (at cell centres the interpolation is the identity)
        p = 6
        npv = (n // p,) * 3
        ijk = I.patch_ijk(npv)
        g = O.Grid(p, npv, ijk, (-L, -L, -L), 2 * L / n, "copy")
        xs, ys, zs = I.point_coords(p, ijk, (-L, -L, -L), 2 * L / n)
        U = O.by_state(B, n, L, u, xs, ys, zs).reshape(g.ushape)
        phi = U[I.IDX["phi"]]
        for q, (a, b, cc) in enumerate(ijk):
            sl = (slice(cc * p, (cc + 1) * p), slice(b * p, (b + 1) * p), slice(a * p, (a + 1) * p))
            np.testing.assert_allclose(phi[q], psi[sl] ** -2.0, rtol=1e-14)
        H, _, _ = g.constraints(U)
        rr = np.sqrt((xs - c[0]) ** 2 + (ys - c[1]) ** 2 + (zs - c[2]) ** 2)
        shell = (rr > 1.0) & (rr < 1.8)
        hs.append(np.abs(H[shell]).max())
    assert hs[0] / hs[1] > 3.0, hs


def test_tricubic_interpolation_is_exact_for_cubics():
    """Lagrange interpolation through four cell centres per axis reproduces
    any polynomial of degree three in each variable, in the interior and
    near the faces (where the stencil shifts inwards)."""
    n, L = 10, 2.0
    rng = np.random.default_rng(5)
    c = rng.uniform(-1, 1, (4, 4, 4))

    def f(x, y, z):
        return sum(c[a, b, k] * x ** a * y ** b * z ** k for a in range(4) for b in range(4) for k in range(4))
    x, y, z = O.by_cell_coords(n, L)
    u = f(x, y, z)
    P = rng.uniform(-L, L, (300, 3))
    got = O.by_interp(n, L, u, P[:, 0], P[:, 1], P[:, 2])
    np.testing.assert_allclose(got, f(P[:, 0], P[:, 1], P[:, 2]), rtol=1e-10, atol=1e-10)
    # at the cell centres it is the identity
    np.testing.assert_allclose(O.by_interp(n, L, u, x, y, z), u.ravel(), rtol=1e-13, atol=1e-13)


def test_assembled_state_maps_the_conformal_factor():
    """phi = psi^-2, A~ = psi^-6 Abar, g~ = delta and the averaged lapse."""
    B = O.make_punctures([0.5, 0.4], [(1.0, 0, 0), (-1.0, 0, 0)], [(0, 0.1, 0), (0, -0.1, 0)])
    n, L = 8, 2.0
    x, y, z = O.by_cell_coords(n, L)
    u = 0.01 * np.cos(x) * np.cos(y) * np.cos(z)
    Q = O.by_state(B, n, L, u, x, y, z)
    A, _, psib = O.by_points(B, x, y, z)
    psi = psib + u.ravel()
    s = psib - 1.0
    np.testing.assert_allclose(Q[I.IDX["phi"]], psi ** -2, rtol=1e-14)
    np.testing.assert_allclose(Q[I.IDX["alpha"]], 0.5 * ((1 - s) / (1 + s) + 1), rtol=1e-14)
    for k, f in enumerate(("Axx", "Axy", "Axz", "Ayy", "Ayz", "Azz")):
        np.testing.assert_allclose(Q[I.IDX[f]], psi ** -6 * A[:, k], rtol=1e-13, atol=1e-16)
    for f in ("gxx", "gyy", "gzz"):
        assert (Q[I.IDX[f]] == 1.0).all()
    for f in ("gxy", "betax", "K", "Theta", "Ghatx", "bx"):
        assert (Q[I.IDX[f]] == 0.0).all()


def _ghost_centres(n, L):
    """Centres (6, n, n) of the ghost cells of a box, in the ghost-array
    order: face 2d (index -1 along axis d) / 2d+1 (index n), then the two
    other cell indices, the lower axis fastest."""
    h = 2.0 * L / n
    X = np.empty((3, 6, n, n))
    ib, ia = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    for d in range(3):
        a, b = [e for e in range(3) if e != d]
        for side in range(2):
            X[d, 2 * d + side] = -L + ((n if side else -1) + 0.5) * h
            X[a, 2 * d + side] = -L + (ia + 0.5) * h
            X[b, 2 * d + side] = -L + (ib + 0.5) * h
    return X


def test_box_ghosts_take_the_parent_at_the_ghost_centres():
    """Nested boxes: the fixed ghost values of a box are the parent's u
    interpolated at the box's ghost-cell centres, in the documented face and
    index order; with a parent that holds a cubic, exactly that cubic. The
    first guess is the same interpolation at the box's cells."""
    def f(x, y, z):
        return 0.3 + x - 0.5 * y ** 2 + 0.2 * x * y * z + z ** 3 / 7.0 - 0.1 * x ** 2 * y
    np_, Lp, n, L = 12, 3.0, 6, 1.2
    up = f(*O.by_cell_coords(np_, Lp))
    gb = O.by_box_ghosts(n, L, np_, Lp, up)
    X = _ghost_centres(n, L)
    np.testing.assert_allclose(gb, f(X[0], X[1], X[2]), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(O.by_cells_from(n, L, np_, Lp, up), f(*O.by_cell_coords(n, L)), rtol=1e-12,
                               atol=1e-12)


def test_fixed_ghosts_enter_the_discrete_operator():
    """With no curvature source the residual is the 7-point Laplacian, exact
    for a quadratic: a box holding q at its cells and ghosts has residual
    Lap q = 4 at every cell, faces and corners included (the fall-off rule
    would not give it there)."""
    B = O.make_punctures([0.5], [(5.1, 0.3, 0.2)])     # no momentum or spin: Abar = 0
    n, L = 6, 1.2

    def q(x, y, z):
        return x ** 2 + 2 * y ** 2 - z ** 2 + x * y - 0.3 * z + 1.0
    u = q(*O.by_cell_coords(n, L))
    X = _ghost_centres(n, L)
    res, mx = O.by_residual_box(B, n, L, u, q(X[0], X[1], X[2]))
    np.testing.assert_allclose(res, 4.0, rtol=0, atol=1e-11)
    res0, _ = O.by_residual(B, n, L, u)
    assert np.abs(res0 - 4.0).max() > 1.0


def test_box_solve_reproduces_the_parent_on_coinciding_cells():
    """A box whose cells and ghost cells are cells of the parent (the same
    spacing) has the parent's solution restricted to it as its discrete
    solution: solved from zero with ghosts from the parent, it returns that
    restriction (so the ghost order, the fixed-ghost derivative and the box
    geometry all agree)."""
    B = O.make_punctures([0.4, 0.35], [(1.1, 0.0, 0.0), (-1.1, 0.0, 0.0)], [(0, 0.2, 0.05), (0, -0.2, 0)],
                         [(0, 0, 0.1), (0, 0, 0)])
    np_, Lp, n, L = 24, 6.0, 12, 3.0
    up, k, r = O.by_solve(B, np_, Lp, tol=1e-12, check=20, omega=1.8)
    assert k > 0
    gb = O.by_box_ghosts(n, L, np_, Lp, up)
    u, k2, r2 = O.by_solve_box(B, n, L, gb, tol=1e-12, check=20, omega=1.7)
    assert k2 > 0 and r2 < 1e-12
    np.testing.assert_allclose(u, up[6:18, 6:18, 6:18], rtol=0, atol=1e-11)
    # starting from the parent's interpolation, it is already solved
    u0 = O.by_cells_from(n, L, np_, Lp, up)
    assert O.by_residual_box(B, n, L, u0, gb)[1] < 1e-11
