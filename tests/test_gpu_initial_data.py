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


@pytest.mark.parametrize("n,L", [(16, 4.0), (15, 3.5)])
def test_sweeps_and_residual_match_the_oracle(n, L):
    """Odd and even n (the colour mapping of odd rows); 40 sweeps from a
    non-zero guess, then the residual of every cell."""
    from paper_2406_11626_gb300 import initial_data as ID
    gB, oB = _pair(*BINARY)
    s = ID.Solver(n, L)
    s.set_punctures(gB)
    x, y, z = O.by_cell_coords(n, L)
    u0 = 0.01 * np.exp(-(x * x + y * y + z * z) / 4.0)
    s.set_u(u0)
    s.sweeps(40)
    gu = s.get_u()
    ou = O.by_sweeps(oB, n, L, u0, 40)
    assert np.abs(gu - ou).max() < 1e-13 * max(np.abs(ou).max(), 1e-3)
    r, res = s.residual(cells=True)
    ores, orm = O.by_residual(oB, n, L, ou)
    assert np.abs(res - ores).max() < 1e-9 * max(np.abs(ores).max(), 1.0)
    assert abs(r - orm) <= 1e-9 * max(orm, 1.0)


def test_solve_matches_the_oracle_solve():
    from paper_2406_11626_gb300 import initial_data as ID
    n, L = 20, 4.0
    gB, oB = _pair(*BINARY)
    s = ID.Solver(n, L)
    s.set_punctures(gB)
    k, r = s.solve(tol=1e-10, check=10)
    ou, ok, orr = O.by_solve(oB, n, L, tol=1e-10, check=10)
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
