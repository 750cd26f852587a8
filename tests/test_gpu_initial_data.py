"""Parity of the GPU puncture initial-data solve (include/ccz4_id.h) with the
Bowen-York oracle: curvature and Brill-Lindquist factor per cell, the
red-black sweeps, the residual, and a full solve."""
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
