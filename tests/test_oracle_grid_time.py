"""Pins of the oracle's grid, halo fill, boundary cells, time stepping and
algebraic enforcement."""
import numpy as np
import pytest

import oracle as O
from paper_2406_11626_gb300 import inputs as I


def _global_reference(U, g, bc):
    """Brute-force halo'd global array [v, z, y, x] over [-3, N+3)^3 built
    from the plain definitions of each boundary kind (not from the oracle)."""
    p, npv = g.p, g.np
    N = [n * p for n in npv]
    inner = np.empty((I.NV, N[2], N[1], N[0]))
    for n, (a, b, c) in enumerate(g.ijk):
        inner[:, c * p:(c + 1) * p, b * p:(b + 1) * p, a * p:(a + 1) * p] = U[:, n]
    zs, ys, xs = (np.arange(-3, n + 3) for n in (N[2], N[1], N[0]))
    if bc == "periodic":
        return inner[:, zs[:, None, None] % N[2], ys[None, :, None] % N[1], xs[None, None, :] % N[0]]
    if bc == "copy":
        return inner[:, np.clip(zs, 0, N[2] - 1)[:, None, None], np.clip(ys, 0, N[1] - 1)[None, :, None],
                     np.clip(xs, 0, N[0] - 1)[None, None, :]]
    raise ValueError(bc)


@pytest.mark.parametrize("bc", ["periodic", "copy", "sommerfeld"])
@pytest.mark.parametrize("p,npv", [(6, (2, 3, 1)), (9, (2, 2, 2)), (4, (1, 1, 3)), (2, (3, 2, 2))])
def test_halo_fill_matches_the_global_definition(bc, p, npv):
    """Every tile value (faces, edges and corners of the width-3 halo) equals
    the value the boundary kind defines at that global point. Small patches
    (p < 3) make halos reach through several neighbours."""
    ijk = I.patch_ijk(npv, permute_seed=3)
    g = O.Grid(p, npv, ijk, (0, 0, 0), 0.1, bc)
    rng = np.random.default_rng(0)
    U = rng.standard_normal(g.ushape)
    G = rng.standard_normal(g.gshape)
    tiles = g.fill_tiles(U, G)
    N = [n * p for n in npv]
    if bc == "sommerfeld":
        ref = np.full((I.NV, N[2] + 6, N[1] + 6, N[0] + 6), np.nan)
        ref[:, 3:N[2] + 3, 3:N[1] + 3, 3:N[0] + 3] = _global_reference(U, g, "periodic")[:, 3:-3, 3:-3, 3:-3]
        gc = I.ghost_cells(N)
        np.testing.assert_array_equal(g.ghost_coords(), gc)
        ref[:, gc[:, 2] + 3, gc[:, 1] + 3, gc[:, 0] + 3] = G
    else:
        ref = _global_reference(U, g, bc)
    T = p + 6
    for n, (a, b, c) in enumerate(ijk):
        exp = ref[:, c * p:c * p + T, b * p:b * p + T, a * p:a * p + T]
        np.testing.assert_array_equal(tiles[:, n], exp)


def test_patch_decomposition_is_bitwise_invariant():
    """One 27^3 patch and 27 patches of 9^3 (shuffled) carry the same points:
    right-hand side, RK4 step and constraints agree bit for bit."""
    cfg = I.gauge_wave_config()
    P = O.make_params(**cfg.params)
    g1 = O.Grid(27, (1, 1, 1), I.patch_ijk((1, 1, 1)), cfg.origin, cfg.dx, "periodic")
    ijk = I.patch_ijk((3, 3, 3), permute_seed=9)
    g27 = O.Grid(9, (3, 3, 3), ijk, cfg.origin, cfg.dx, "periodic")
    x, y, z = I.point_coords(9, ijk, cfg.origin, cfg.dx)
    U27 = I.smooth_perturbation(x, y, z, seed=1, amp=0.02, base=I.gauge_wave(x))
    U1 = np.empty(g1.ushape)
    for n, (a, b, c) in enumerate(ijk):
        U1[:, 0, c * 9:(c + 1) * 9, b * 9:(b + 1) * 9, a * 9:(a + 1) * 9] = U27[:, n]

    def back(A1):
        out = np.empty(g27.ushape)
        for n, (a, b, c) in enumerate(ijk):
            out[:, n] = A1[:, 0, c * 9:(c + 1) * 9, b * 9:(b + 1) * 9, a * 9:(a + 1) * 9]
        return out

    r1, _ = g1.rhs(P, U1)
    r27, _ = g27.rhs(P, U27)
    np.testing.assert_array_equal(back(r1), r27)
    s1, _ = g1.rk4_step(P, cfg.dt, U1)
    s27, _ = g27.rk4_step(P, cfg.dt, U27)
    np.testing.assert_array_equal(back(s1), s27)
    H1, M1, o1 = g1.constraints(U1)
    H27, M27, o27 = g27.constraints(U27)
    np.testing.assert_array_equal(back(np.broadcast_to(H1, (I.NV,) + H1.shape))[0], H27)


def test_enforcement_restores_unit_determinant_and_zero_trace():
    g = O.Grid(4, (2, 1, 1), I.patch_ijk((2, 1, 1)), (0, 0, 0), 0.1, "periodic")
    rng = np.random.default_rng(5)
    U = I.flat(g.ushape[1:]) + rng.uniform(-0.1, 0.1, size=g.ushape)
    E = g.enforce(U)
    S = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))
    gm = np.empty((3, 3) + g.ushape[1:])
    A = np.empty_like(gm)
    for s, (i, j) in enumerate(S):
        gm[i, j] = gm[j, i] = E[s]
        A[i, j] = A[j, i] = E[11 + s]
    gm = np.moveaxis(gm, (0, 1), (-2, -1))
    A = np.moveaxis(A, (0, 1), (-2, -1))
    np.testing.assert_allclose(np.linalg.det(gm), 1.0, rtol=0, atol=1e-14)
    tr = np.einsum("...ij,...ij->...", np.linalg.inv(gm), A)
    np.testing.assert_allclose(tr, 0.0, rtol=0, atol=1e-15)
    # untouched fields, idempotence, and a conformal rescaling of g~ only
    others = [v for v in range(I.NV) if not (v < 6 or 11 <= v < 17)]
    np.testing.assert_array_equal(E[others], U[others])
    np.testing.assert_allclose(g.enforce(E), E, rtol=0, atol=2e-15)
    ratio = E[:6] / U[:6]
    np.testing.assert_allclose(ratio, np.broadcast_to(ratio[0], ratio.shape), rtol=1e-13)


def test_sommerfeld_ghost_rhs_for_an_outgoing_spherical_wave():
    """Q = Q0 + f(r - t) / r solves d_t Q + d_r Q = -(Q - Q0) / r exactly
    (speed 1). With the paper's one-sided difference the ghost right-hand side
    approaches the exact d_t Q at first order in dx."""
    errs = []
    for N in (16, 32):
        p = 8
        npv = (N // p,) * 3
        h = 8.0 / N
        g = O.Grid(p, npv, I.patch_ijk(npv), (-4.0, -4.0, -4.0), h, "sommerfeld")
        x, y, z = I.point_coords(p, g.ijk, g.origin, h)
        gx, gy, gz = I.ghost_positions((N, N, N), g.origin, h)

        def field(xx, yy, zz, t=0.0):
            r = np.sqrt(xx ** 2 + yy ** 2 + zz ** 2)
            Q = I.flat(r.shape)
            Q[I.IDX["K"]] = np.sin(r - t) / r
            Q[I.IDX["Theta"]] = 0.5 + np.exp(-(r - t - 4.0) ** 2) / r
            return Q

        U = field(x, y, z)
        G = field(gx, gy, gz)
        Gini = I.flat(G.shape[1:])
        Gini[I.IDX["Theta"]] = 0.5
        _, rG = g.rhs(O.make_params(**I.PUNCTURE_PARAMS), U, G, Gini)
        rg = np.sqrt(gx ** 2 + gy ** 2 + gz ** 2)
        exact_K = -np.cos(rg) / rg
        s = rg - 4.0
        exact_T = 2 * s * np.exp(-s ** 2) / rg
        errs.append((np.abs(rG[I.IDX["K"]] - exact_K).max(), np.abs(rG[I.IDX["Theta"]] - exact_T).max()))
    for k in range(2):
        assert 1.6 < errs[0][k] / errs[1][k] < 2.6


@pytest.mark.slow
def test_rk4_is_fourth_order_in_time():
    """Classic RK4 at fixed dx: halving dt divides the time error by ~16
    (first and second order schemes would give 2 and 4)."""
    cfg = I.gauge_wave_config()
    p = 4
    npv = (4, 1, 1)
    h = 1.0 / 16
    g = O.Grid(p, npv, I.patch_ijk(npv), (-0.5, -0.5, -0.5), h, "periodic")
    x, _, _ = I.point_coords(p, g.ijk, g.origin, h)
    P = O.make_params(**cfg.params)
    T = 0.4

    def run(nsteps):
        U = I.gauge_wave(x)
        for _ in range(nsteps):
            U, _ = g.rk4_step(P, T / nsteps, U)
        return U

    ref = run(128)
    e = [np.abs(run(n) - ref).max() for n in (8, 16)]
    assert 13.0 < e[0] / e[1] < 19.0


@pytest.mark.slow
def test_evolved_gauge_wave_converges_at_4th_order():
    """Sec. "Gauge Wave" (convergence study): RK4, CFL 0.1, KO 0.1 -- the
    evolved state approaches the exact travelling wave as dx^4, and so does
    the L2 norm of the Hamiltonian constraint."""
    cfg = I.gauge_wave_config()
    P = O.make_params(**cfg.params)
    T = 0.2
    errs, l2h = [], []
    for N in (16, 32):
        p = 4
        npv = (N // p, 1, 1)
        h = 1.0 / N
        g = O.Grid(p, npv, I.patch_ijk(npv), (-0.5, -0.5, -0.5), h, "periodic")
        x, _, _ = I.point_coords(p, g.ijk, g.origin, h)
        U = I.gauge_wave(x)
        n = int(round(T / (0.1 * h)))
        for _ in range(n):
            U, _ = g.rk4_step(P, T / n, U)
        errs.append(np.abs(U - I.gauge_wave(x, T)).max())
        l2h.append(g.constraints(U)[2][0])
    assert errs[0] / errs[1] > 12.0
    assert l2h[0] / l2h[1] > 12.0
