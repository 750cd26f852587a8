"""Parity of the GPU puncture initial-data solve (include/ccz4_id.h) with the
Bowen-York oracle: curvature and Brill-Lindquist factor per cell, the
red-black sweeps, the residual, a full solve, and nested boxes (fixed
ghosts from a parent, their sweeps and solve, assembly from the finest
box)."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available()


def _pair(masses, centres, momenta, spins):
    from paper_2406_11626_gb300 import initial_data as ID
    return (ID.make_punctures(masses, centres, momenta, spins),
            O.make_punctures(masses, centres, momenta, spins))


BINARY = ([0.45, 0.55], [(-1.3, 0.05, 0.0), (1.3, -0.05, 0.02)], [(0.0, -0.15, 0.02), (0.01, 0.15, 0.0)],
          [(0.0, 0.0, 0.2), (0.05, 0.0, 0.1)])


@pytest.mark.parametrize("n,L,omega", [(16, 4.0, 1.0), (15, 3.5, 1.0), (16, 4.0, 1.7), (2, 4.0, 1.0), (3, 3.5, 1.3)])
def test_sweeps_and_residual_match_the_oracle(n, L, omega):
    """Odd and even n (the colour mapping of odd rows), plain and
    over-relaxed; grids with no interior cell (n = 2) and a single one
    (n = 3), where the boundary-shell threads do all or nearly all of the
    work; 40 sweeps from a non-zero guess, then the residual of every cell."""
    from paper_2406_11626_gb300 import initial_data as ID
    gB, oB = _pair(*BINARY)
    s = ID.Solver(n, L)
    s.set_punctures(gB)
    x, y, z = O.by_cell_coords(n, L)
    u0 = 0.01 * np.exp(-(x * x + y * y + z * z) / 4.0)
    s.set_u(u0)
    s.set_relaxation(omega)
    s.sweeps(40)
    gu = s.get_u()
    ou = O.by_sweeps(oB, n, L, u0, 40, omega)
    assert np.abs(gu - ou).max() < 1e-13 * max(np.abs(ou).max(), 1e-3)
    r, res = s.residual(cells=True)
    ores, orm = O.by_residual(oB, n, L, ou)
    assert np.abs(res - ores).max() < 1e-9 * max(np.abs(ores).max(), 1.0)
    assert abs(r - orm) <= 1e-9 * max(orm, 1.0)


@pytest.mark.parametrize("omega", [1.0, 1.75])
def test_solve_matches_the_oracle_solve(omega):
    from paper_2406_11626_gb300 import initial_data as ID
    n, L = 20, 4.0
    gB, oB = _pair(*BINARY)
    s = ID.Solver(n, L)
    s.set_punctures(gB)
    s.set_relaxation(omega)
    k, r = s.solve(tol=1e-10, check=10)
    ou, ok, orr = O.by_solve(oB, n, L, tol=1e-10, check=10, omega=omega)
    assert k > 0 and r < 1e-10 and ok > 0
    assert abs(k - ok) <= 10
    assert np.abs(s.get_u() - ou).max() < 1e-10


def test_trivial_source_converges_immediately():
    from paper_2406_11626_gb300 import initial_data as ID
    s = ID.Solver(12, 3.0)
    s.set_punctures(ID.make_punctures([0.5, 0.5], [(1.1, 0, 0), (-1.1, 0, 0)]))
    k, r = s.solve(tol=1e-12, check=5)
    assert k == 0 and r == 0.0


def test_invalid_solver_arguments_are_rejected():
    from paper_2406_11626_gb300 import ccz4 as C
    from paper_2406_11626_gb300 import initial_data as ID
    for n, L in ((1, 1.0), (2000, 1.0), (16, 0.0)):
        with pytest.raises(C.CCZ4Error):
            ID.Solver(n, L)
    s = ID.Solver(8, 1.0)
    with pytest.raises(C.CCZ4Error):
        s.solve(tol=0.0)
    for w in (0.0, 2.0, -1.0):
        with pytest.raises(C.CCZ4Error):
            s.set_relaxation(w)


def test_assembled_state_matches_the_oracle_on_a_mesh():
    """The CCZ4 state of solved data on every point of a three-level mesh
    and its Sommerfeld shell equals the oracle's assembly from the same u."""
    from paper_2406_11626_gb300 import ccz4 as C
    from paper_2406_11626_gb300 import initial_data as ID
    from paper_2406_11626_gb300 import inputs as I
    gB, oB = _pair(*BINARY)
    n, L = 24, 6.0
    s = ID.Solver(n, L)
    s.set_punctures(gB)
    s.solve(tol=1e-10, check=20)
    u = s.get_u()
    p, np_ = 6, (4, 4, 4)
    lev, ijk = I.refined_mesh(np_, [((1, 1, 1), (3, 3, 3)), ((5, 5, 5), (7, 7, 7))])
    origin, dx = (-4.0, -4.0, -4.0), 2.0 / 6.0
    g = C.Grid(p, np_, ijk, origin, dx, "sommerfeld", level=lev)
    s.assemble(gB, g, "U")
    U, G = g.download("U")
    x, y, z = I.mesh_point_coords(p, lev, ijk, origin, dx)
    want = O.by_state(oB, n, L, u, x, y, z).reshape(U.shape)
    assert np.abs(U - want).max() < 1e-12 * np.abs(want).max()
    gx, gy, gz = I.ghost_positions(tuple(v * p for v in np_), origin, dx)
    wantG = O.by_state(oB, n, L, u, gx, gy, gz)
    assert np.abs(G - wantG).max() < 1e-12 * np.abs(wantG).max()


def _boxes(n, L, nb, Lb):
    """A parent solver with smooth non-zero u and a box nested in it, both
    with the binary's punctures; returns (parent, box, parent u, oracle
    punctures)."""
    from paper_2406_11626_gb300 import initial_data as ID
    gB, oB = _pair(*BINARY)
    s = ID.Solver(n, L)
    s.set_punctures(gB)
    x, y, z = O.by_cell_coords(n, L)
    up = 0.02 * np.exp(-(x * x + 2 * y * y + z * z) / 5.0) + 0.003 * x * y
    s.set_u(up)
    b = ID.Solver(nb, Lb)
    b.set_punctures(gB)
    return s, b, up, oB


@pytest.mark.parametrize("nb,Lb,omega", [(12, 2.0, 1.0), (11, 2.3, 1.6)])
def test_nested_box_ghosts_guess_sweeps_and_residual_match_the_oracle(nb, Lb, omega):
    """A box nested in a parent: its first guess and fixed ghosts (the
    parent's u interpolated), 30 sweeps with fixed ghosts and the residual
    of every cell against the oracle's nested-box functions."""
    n, L = 16, 4.0
    s, b, up, oB = _boxes(n, L, nb, Lb)
    b.set_parent(s, init_u=True)
    u0 = O.by_cells_from(nb, Lb, n, L, up)
    assert np.abs(b.get_u() - u0).max() < 1e-15
    gb = O.by_box_ghosts(nb, Lb, n, L, up)
    b.set_relaxation(omega)
    b.sweeps(30)
    ou = O.by_sweeps_box(oB, nb, Lb, u0, gb, 30, omega)
    assert np.abs(b.get_u() - ou).max() < 1e-13 * max(np.abs(ou).max(), 1e-3)
    r, res = b.residual(cells=True)
    ores, orm = O.by_residual_box(oB, nb, Lb, ou, gb)
    assert np.abs(res - ores).max() < 1e-9 * max(np.abs(ores).max(), 1.0)
    assert abs(r - orm) <= 1e-9 * max(orm, 1.0)
    # the ghosts were taken at the call: a later change of the parent does not reach the box
    s.set_u(np.zeros((n, n, n)))
    r2, _ = b.residual(cells=True)
    assert r2 == r
    # back to the fall-off rule
    b.set_parent(None)
    orf = O.by_residual(oB, nb, Lb, b.get_u())[1]
    assert abs(b.residual() - orf) <= 1e-9 * max(orf, 1.0)


def test_nested_solve_reproduces_the_parent_on_coinciding_cells():
    """A box whose cells and ghost cells are cells of the parent has the
    parent's solution, restricted, as its solution: solved from zero with
    fixed ghosts from the solved parent, it returns it; from the parent's
    interpolation it starts solved."""
    from paper_2406_11626_gb300 import initial_data as ID
    gB, _ = _pair(*BINARY)
    s = ID.Solver(24, 6.0)
    s.set_punctures(gB)
    s.set_relaxation(1.8)
    k, r = s.solve(tol=1e-12, check=20)
    assert k > 0
    b = ID.Solver(12, 3.0)
    b.set_punctures(gB)
    b.set_parent(s, init_u=False)
    b.set_relaxation(ID.box_omega(12))
    kb, rb = b.solve(tol=1e-12, check=20)
    assert kb > 0 and rb < 1e-12
    assert np.abs(b.get_u() - s.get_u()[6:18, 6:18, 6:18]).max() < 1e-11
    b.set_parent(s, init_u=True)
    assert b.solve(tol=1e-11, check=20)[0] == 0


def test_nested_assembly_takes_each_point_from_the_finest_box():
    """The outermost solver's state everywhere, then the box's where its
    stencil is centred (every |x_d| < L - 3h/2): each point of a two-level
    mesh and its Sommerfeld shell equals the oracle's assembly from the u
    that covers it."""
    from paper_2406_11626_gb300 import ccz4 as C
    from paper_2406_11626_gb300 import initial_data as ID
    from paper_2406_11626_gb300 import inputs as I
    s, b, up, oB = _boxes(16, 4.0, 16, 2.0)
    gB = ID.make_punctures(*BINARY)
    b.set_parent(s, init_u=True)
    b.set_relaxation(1.5)
    b.sweeps(5)
    ub = b.get_u()
    p, np_ = 6, (4, 4, 4)
    lev, ijk = I.refined_mesh(np_, [((1, 1, 1), (3, 3, 3))])
    origin, dx = (-3.5, -3.5, -3.5), 1.75 / 6.0
    g = C.Grid(p, np_, ijk, origin, dx, "sommerfeld", level=lev)
    ID.assemble_nested([s, b], gB, g, "U")
    U, G = g.download("U")
    x, y, z = I.mesh_point_coords(p, lev, ijk, origin, dx)
    lim = 2.0 - 1.5 * (4.0 / 16)
    inside = ((np.abs(x) < lim) & (np.abs(y) < lim) & (np.abs(z) < lim)).ravel()
    assert inside.any() and (~inside).any()
    want = np.where(inside[None, :], O.by_state(oB, 16, 2.0, ub, x, y, z), O.by_state(oB, 16, 4.0, up, x, y, z))
    assert np.abs(U - want.reshape(U.shape)).max() < 1e-12 * np.abs(want).max()
    gx, gy, gz = I.ghost_positions(tuple(v * p for v in np_), origin, dx)
    wantG = O.by_state(oB, 16, 4.0, up, gx, gy, gz)
    assert np.abs(G - wantG).max() < 1e-12 * np.abs(wantG).max()


def test_nested_box_arguments_are_checked():
    from paper_2406_11626_gb300 import ccz4 as C
    from paper_2406_11626_gb300 import initial_data as ID
    s, b, _, _ = _boxes(16, 4.0, 16, 3.9)      # ghost centres at 3.9 + 0.24 > 4
    with pytest.raises(C.CCZ4Error):
        b.set_parent(s)
    with pytest.raises(C.CCZ4Error):
        s.set_parent(s)
    ok = ID.Solver(16, 3.5)
    ok.set_punctures(ID.make_punctures(*BINARY))
    ok.set_parent(s)
