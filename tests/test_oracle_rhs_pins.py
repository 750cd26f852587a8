"""Pins of the oracle's CCZ4 right-hand side and constraint monitors against
what the paper and the mathematics fix: flat space, the paper's closed-form
gauge wave, exact Minkowski data in moving coordinates, the Brill-Lindquist
puncture, and rotation covariance."""
import numpy as np
import pytest

import exact_minkowski as EM
import oracle as O
from paper_2406_11626_gb300 import inputs as I

GW = dict(I.GAUGE_WAVE_PARAMS)
PUNC = dict(I.PUNCTURE_PARAMS)


@pytest.mark.parametrize("bc", ["periodic", "copy", "sommerfeld"])
@pytest.mark.parametrize("gauge", [("harmonic", "zero"), ("1+log", "gamma-driver")])
def test_flat_space_rhs_is_exactly_zero(bc, gauge):
    g = O.Grid(5, (2, 2, 2), I.patch_ijk((2, 2, 2), 1), (-1.0, -1.0, -1.0), 0.2, bc)
    U = I.flat(g.ushape[1:])
    G = I.flat((g.n_ghost,))
    P = O.make_params(**dict(PUNC, slicing=gauge[0], shift=gauge[1]))
    rU, rG = g.rhs(P, U, G, G)
    assert np.all(rU == 0.0) and np.all(rG == 0.0)
    H, M, out = g.constraints(U, G)
    assert np.all(H == 0.0) and np.all(M == 0.0)


def test_flat_space_with_constant_shift_and_b_is_static():
    """Constant beta and b = 0 in flat space: every derivative vanishes, and
    the Gamma-driver returns d_t beta = f b = 0."""
    g = O.Grid(4, (2, 1, 1), I.patch_ijk((2, 1, 1)), (0, 0, 0), 0.25, "periodic")
    U = I.flat(g.ushape[1:])
    U[I.IDX["betax"]] = 0.25   # dyadic values: the KO sum of a constant is then exactly 0
    U[I.IDX["betaz"]] = -0.5
    rU, _ = g.rhs(O.make_params(**PUNC), U)
    assert np.all(rU == 0.0)


def _thin_gauge_wave(N, p=8):
    np_ = (N // p, 1, 1)
    h = 1.0 / N
    g = O.Grid(p, np_, I.patch_ijk(np_), (-0.5, -0.5, -0.5), h, "periodic")
    x, _, _ = I.point_coords(p, g.ijk, g.origin, h)
    return g, x


def test_gauge_wave_rhs_matches_exact_time_derivative_at_4th_order():
    """Sec. "Gauge Wave": the printed closed form is an exact solution with
    harmonic slicing and zero shift; the discrete right-hand side at the exact
    data must approach its time derivative as dx^4."""
    P = O.make_params(**GW)
    errs = []
    for N in (16, 32):
        g, x = _thin_gauge_wave(N)
        rU, _ = g.rhs(P, I.gauge_wave(x))
        errs.append(np.abs(rU - I.gauge_wave_dt(x)).reshape(I.NV, -1).max(axis=1))
    for v in range(I.NV):
        if errs[0][v] > 1e-10:
            assert errs[0][v] / errs[1][v] > 12.0, I.FIELDS[v]
        else:
            assert errs[1][v] < 1e-10, I.FIELDS[v]
    assert errs[1].max() < 1e-3


def test_gauge_wave_constraints_vanish_at_4th_order():
    out = []
    for N in (16, 32):
        g, x = _thin_gauge_wave(N)
        out.append(g.constraints(I.gauge_wave(x))[2])
    assert out[0][0] / out[1][0] > 12.0 and out[0][1] / out[1][1] > 12.0
    assert out[1][4] == 0.0


def _wobbly(N, seed=3, p=8):
    np_ = (N // p,) * 3
    h = 1.0 / N
    g = O.Grid(p, np_, I.patch_ijk(np_, 5), (0.0, 0.0, 0.0), h, "periodic")
    x, y, z = I.point_coords(p, g.ijk, g.origin, h)
    modes = EM.make_modes(seed)
    return g, EM.ccz4_state(modes, 0.0, x, y, z), EM.ccz4_state_dt(modes, 0.0, x, y, z)


@pytest.mark.slow
def test_minkowski_in_moving_coordinates_rhs_at_4th_order():
    """Flat spacetime in time-dependent coordinates: non-zero lapse, shift,
    extrinsic and intrinsic curvature. For every field whose equation holds
    in any gauge (all but alpha, beta, b) the discrete right-hand side at the
    exact data approaches the exact time derivative as dx^4."""
    P = O.make_params(**PUNC)
    errs = []
    for N in (16, 32):
        g, U, D = _wobbly(N)
        assert np.abs(U[I.IDX["betax"]:I.IDX["betaz"] + 1]).max() > 0.1
        assert np.abs(U[I.IDX["K"]]).max() > 0.5
        rU, _ = g.rhs(P, U)
        errs.append(np.abs(rU - D).reshape(I.NV, -1).max(axis=1))
    for v in EM.PHYSICAL:
        assert errs[0][v] / errs[1][v] > 10.0, I.FIELDS[v]
        assert errs[1][v] < 3e-2, I.FIELDS[v]


@pytest.mark.slow
def test_minkowski_in_moving_coordinates_constraints_vanish():
    outs = []
    for N in (16, 32):
        g, U, _ = _wobbly(N, seed=4)
        outs.append(g.constraints(U)[2])
    assert outs[0][0] / outs[1][0] > 10.0
    assert outs[0][1] / outs[1][1] > 10.0


def test_puncture_hamiltonian_constraint_converges_away_from_the_puncture():
    """Sec. "Single Schwarzschild Black Hole": phi = (1 + M/2r)^-2 with
    K_ij = 0 and conformal flatness solves the Hamiltonian constraint exactly;
    the discrete H must vanish as dx^4 away from r = 0."""
    maxes = []
    for N in (32, 64):
        p = 8
        np_ = (N // p,) * 3
        h = 8.0 / N
        g = O.Grid(p, np_, I.patch_ijk(np_, 2), (-4.0, -4.0, -4.0), h, "copy")
        x, y, z = I.point_coords(p, g.ijk, g.origin, h)
        U = I.brill_lindquist(x, y, z)
        r = np.sqrt(x ** 2 + y ** 2 + z ** 2).ravel()
        pts = np.nonzero((r > 2.0) & (r < 3.0))[0]
        c = g.constraints_points(U, None, pts)
        maxes.append(np.abs(c).max(axis=0))
    assert maxes[0][0] / maxes[1][0] > 12.0
    assert maxes[1][1:].max() < 1e-12   # M vanishes identically (K = A~ = 0)


def _rotate_state(Q, R, N):
    """Apply the rigid rotation R (a signed permutation) about the centre of a
    periodic cube of N^3 cell-centred points to a global field array
    Q[v, z, y, x]: scalars move, vectors and tensors rotate."""
    out = np.empty_like(Q)
    idx = np.indices((N, N, N))           # (z, y, x)
    pos = np.stack([idx[2], idx[1], idx[0]]) - (N - 1) / 2.0
    newpos = np.einsum("ij,j...->i...", R, pos)
    ni = np.rint(newpos + (N - 1) / 2.0).astype(int)
    vec = [("betax", 3), ("Ghatx", 3), ("bx", 3)]
    sym = [("gxx", 6), ("Axx", 6)]
    S = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))
    comp = Q.copy()
    for name, n in vec:
        b = I.IDX[name]
        comp[b:b + 3] = np.einsum("ij,j...->i...", R, Q[b:b + 3])
    for name, n in sym:
        b = I.IDX[name]
        T = np.empty((3, 3) + Q.shape[1:])
        for s, (i, j) in enumerate(S):
            T[i, j] = T[j, i] = Q[b + s]
        T2 = np.einsum("ia,jb,ab...->ij...", R, R, T)
        for s, (i, j) in enumerate(S):
            comp[b + s] = T2[i, j]
    out[:, ni[2], ni[1], ni[0]] = comp
    return out


def _to_global(U, g):
    p = g.p
    N = g.np[0] * p
    out = np.empty((I.NV, N, N, N))
    for n, (a, b, c) in enumerate(g.ijk):
        out[:, c * p:(c + 1) * p, b * p:(b + 1) * p, a * p:(a + 1) * p] = U[:, n]
    return out


def _from_global(Qg, g):
    p = g.p
    U = np.empty(g.ushape)
    for n, (a, b, c) in enumerate(g.ijk):
        U[:, n] = Qg[:, c * p:(c + 1) * p, b * p:(b + 1) * p, a * p:(a + 1) * p]
    return U


@pytest.mark.parametrize("R", [np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]]),
                               np.array([[1, 0, 0], [0, 0, -1], [0, 1, 0]]),
                               np.array([[0, 0, 1], [1, 0, 0], [0, 1, 0]])])
def test_rhs_and_constraints_are_rotation_covariant(R):
    """The equations are tensorial and the stencils are the same along every
    axis, so rotating the data by a lattice rotation rotates the right-hand
    side and the constraints (up to rounding)."""
    N, p = 12, 6
    g = O.Grid(p, (2, 2, 2), I.patch_ijk((2, 2, 2), 7), (0, 0, 0), 1.0 / N, "periodic")
    x, y, z = I.point_coords(p, g.ijk, g.origin, 1.0 / N)
    U = I.smooth_perturbation(x, y, z, seed=11, amp=0.05)
    P = O.make_params(**PUNC)
    rU, _ = g.rhs(P, U)
    Ur = _from_global(_rotate_state(_to_global(U, g), R, N), g)
    rUr, _ = g.rhs(P, Ur)
    expect = _from_global(_rotate_state(_to_global(rU, g), R, N), g)
    scale = np.abs(rU).max()
    np.testing.assert_allclose(rUr, expect, rtol=0, atol=1e-12 * scale)
    H, M, _ = g.constraints(U)
    Hr, Mr, _ = g.constraints(Ur)
    Hg = _to_global(np.broadcast_to(H, (I.NV,) + H.shape), g)
    Hexp = _from_global(_rotate_state(Hg, R, N), g)[0]
    np.testing.assert_allclose(Hr, Hexp, rtol=0, atol=1e-12 * np.abs(H).max())
