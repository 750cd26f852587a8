"""Pins of the oracle's first-order formulation (appendix "Formulation for
the kernel FD4 Solver", Eq. first-order-variables; the auxiliary equations
NR_foccz4_A_k, NR_foccz4_B^i_j, the D_kij equation, NR_foccz4_P_i; Alg.
fd4-fo) and of the second-order formulation with reconstruction (Alg.
fd4-so). None of them restates the oracle's formulas:

- flat space is static in both, exactly;
- on polynomial data of degree <= 4 (where FD4 first derivatives, their
  composition and the second-derivative stencils are all exact) the
  primaries' right-hand side without red terms equals that of the
  independently pinned second-order oracle, both with the auxiliary
  variables given exactly and with them reconstructed by the oracle;
- the reconstruction reproduces exact derivatives of such data;
- on the gauge wave (an exact solution, harmonic slicing) every one of the
  58 right-hand sides converges at fourth order to the exact time
  derivative, with and without the red terms (which vanish on solutions);
- on Minkowski space in moving coordinates (lapse, shift, K and the curvature
  of the slices all non-trivial) the equations that hold for any gauge, the
  physical primaries and the D_kij and P_k equations, converge the same way;
- the linear response about flat space of each auxiliary equation to one
  Fourier mode is a hand-derived constant times the mode or its FD4
  derivative (slicing, g'(alpha), Gamma-driver f, the mu terms, the shift
  terms of D, every red term);
- the evolved gauge wave converges at fourth order to the exact solution in
  both formulations.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2406_11626_gb300 import inputs as I

import exact_minkowski as EM

NV, NVF = I.NV, I.NV_FO
F = {n: i for i, n in enumerate(I.FO_FIELDS)}


def _flat_fo(shape):
    U = np.zeros((NVF,) + tuple(shape))
    U[:NV] = I.flat(shape)
    return U


@pytest.mark.parametrize("bc", ["periodic", "sommerfeld"])
@pytest.mark.parametrize("gauge", [("harmonic", "zero"), ("1+log", "gamma-driver")])
@pytest.mark.parametrize("red", [True, False])
def test_flat_space_is_exactly_static(bc, gauge, red):
    cfg = I.single_puncture_config(p=4, n_side=2, half_width=1.0)
    g = O.Grid(cfg.p, cfg.np, cfg.ijk(), cfg.origin, cfg.dx, bc)
    U = _flat_fo(g.fo_ushape[1:])
    G = _flat_fo((g.n_ghost,))
    P = O.make_params(slicing=gauge[0], shift=gauge[1], mu=0.35)
    rU, rG = g.fo_rhs(P, U, G, G, red=red)
    assert not rU.any() and not rG.any()


# ---- polynomial data: the first-order primaries agree with the second-order oracle ----------------------------

def _poly(seed, x, y, z, amp):
    """(value, gradient) of a random polynomial of total degree <= 4."""
    rng = np.random.default_rng(seed)
    val = np.zeros_like(x)
    grad = np.zeros((3,) + x.shape)
    for a in range(5):
        for b in range(5 - a):
            for c in range(5 - a - b):
                if a + b + c == 0:
                    continue
                w = rng.uniform(-amp, amp)
                val += w * x ** a * y ** b * z ** c
                if a:
                    grad[0] += w * a * x ** (a - 1) * y ** b * z ** c
                if b:
                    grad[1] += w * b * x ** a * y ** (b - 1) * z ** c
                if c:
                    grad[2] += w * c * x ** a * y ** b * z ** (c - 1)
    return val, grad


def _poly_state(seed, x, y, z, amp=2e-2):
    Q = I.flat(x.shape)
    dQ = np.zeros((3,) + Q.shape)
    for v in range(NV):
        val, grad = _poly(seed * 100 + v, x, y, z, amp)
        Q[v] += val
        dQ[:, v] = grad
    return Q, dQ


def _poly_setup():
    p, n = 6, 3
    ijk = I.patch_ijk((n, n, n), permute_seed=1)
    h = 1.0 / (n * p)
    g = O.Grid(p, (n, n, n), ijk, (-0.5, -0.5, -0.5), h, "periodic")
    x, y, z = I.point_coords(p, ijk, g.origin, h)
    # points whose stencils (reach 3, and 2 + 2 for derivatives of reconstructed values) do not wrap
    gi = [np.rint((c - g.origin[d]) / h - 0.5).astype(int) for d, c in enumerate((x, y, z))]
    inner = np.ones(x.shape, dtype=bool)
    for d in range(3):
        inner &= (gi[d] >= 4) & (gi[d] < n * p - 4)
    return g, x, y, z, inner


@pytest.mark.parametrize("gauge", [("harmonic", "zero"), ("1+log", "gamma-driver")])
@pytest.mark.parametrize("reconstructed", [False, True])
def test_primaries_without_red_terms_equal_the_second_order_oracle_on_polynomials(gauge, reconstructed):
    g, x, y, z, inner = _poly_setup()
    Q, dQ = _poly_state(3, x, y, z)
    U = I.fo_state(Q, dQ)
    if reconstructed:
        U = g.fo_reconstruct(U)
    P = O.make_params(slicing=gauge[0], shift=gauge[1], kappa1=0.3, kappa2=0.7, kappa3=0.45, e=1.7, c=1.3,
                      tau=0.8, f=0.6, eta=2.3, s=0.5, mu=0.35)
    rfo, _ = g.fo_rhs(P, U, red=False)
    rso, _ = g.rhs(P, Q)
    for v in range(NV):
        a, b = rfo[v][inner], rso[v][inner]
        assert np.abs(a - b).max() <= 1e-9 * max(np.abs(b).max(), 1.0), I.FIELDS[v]


def test_reconstruction_gives_exact_derivatives_of_polynomials():
    g, x, y, z, inner = _poly_setup()
    Q, dQ = _poly_state(5, x, y, z)
    U = g.fo_reconstruct(I.fo_state(Q, np.zeros_like(dQ)))
    want = I.fo_state(Q, dQ)
    assert np.array_equal(U[:NV], want[:NV])
    for v in range(NV, NVF):
        assert np.abs(U[v][inner] - want[v][inner]).max() < 1e-11, I.FO_FIELDS[v]


# ---- exact solutions: fourth-order convergence of every right-hand side ---------------------------------------

def _fo_gauge_wave_dt(x, t, eps=1e-3):
    f = [I.fo_gauge_wave(x, t + s * eps) for s in (-2, -1, 1, 2)]
    return (f[0] - 8.0 * f[1] + 8.0 * f[2] - f[3]) / (12.0 * eps)


def _thin_grid(nx, p=9):
    np_ = (nx, 1, 1)
    h = 1.0 / (nx * p)
    return O.Grid(p, np_, I.patch_ijk(np_), (-0.5, -0.5, -0.5), h, "periodic"), h


@pytest.mark.parametrize("red", [True, False])
def test_gauge_wave_rhs_converges_at_fourth_order_for_all_58(red):
    P = O.make_params(**I.GAUGE_WAVE_PARAMS)
    errs = []
    for nx in (3, 6):
        g, h = _thin_grid(nx)
        x, _, _ = I.point_coords(g.p, g.ijk, g.origin, h)
        rU, _ = g.fo_rhs(P, I.fo_gauge_wave(x), red=red)
        ex = _fo_gauge_wave_dt(x, 0.0)
        errs.append(np.abs(rU - ex).reshape(NVF, -1).max(axis=1))
    moving = [v for v in range(NVF) if errs[0][v] > 1e-9]
    # the fields the wave moves: every primary of the wave and A_x, D_x.., P_x
    assert {F[n] for n in ("gxx", "gyy", "alpha", "phi", "Axx", "K", "Ghatx", "Ax", "Dxxx", "Dxyy", "Px")} <= set(moving)
    for v in range(NVF):
        if v in moving:
            assert errs[0][v] / errs[1][v] > 12.0, (I.FO_FIELDS[v], errs[0][v], errs[1][v])
        else:
            assert errs[1][v] < 1e-9, I.FO_FIELDS[v]


def _minkowski_fo(modes, t, x, y, z, eps=1e-3):
    """58 variables of Minkowski space in moving coordinates: the auxiliary
    variables from fourth-order central differences in space of the exact
    primaries (their error, ~1e-10, is far below the truncation errors
    measured here)."""
    Q = EM.ccz4_state(modes, t, x, y, z)
    dQ = np.zeros((3,) + Q.shape)
    for k in range(3):
        f = []
        for s in (-2, -1, 1, 2):
            d = [x, y, z]
            d[k] = d[k] + s * eps
            f.append(EM.ccz4_state(modes, t, *d))
        dQ[k] = (f[0] - 8.0 * f[1] + 8.0 * f[2] - f[3]) / (12.0 * eps)
    return I.fo_state(Q, dQ)


def test_minkowski_in_moving_coordinates_gauge_free_equations_converge():
    modes = EM.make_modes(2, amp=0.02)
    P = O.make_params(slicing="harmonic", shift="gamma-driver", kappa1=0.0, kappa2=0.0, kappa3=0.0, tau=1.0,
                      ko_eps=0.0, mu=0.35)
    # equations that hold for any lapse and shift: the physical primaries, D_kij and P_k
    check = list(EM.PHYSICAL) + list(range(I.FO_D, I.FO_D + 18)) + list(range(I.FO_P, I.FO_P + 3))
    errs = []
    for n in (2, 4):
        p = 8
        ijk = I.patch_ijk((n, n, n))
        h = 1.0 / (n * p)
        g = O.Grid(p, (n, n, n), ijk, (-0.5, -0.5, -0.5), h, "periodic")
        x, y, z = I.point_coords(p, ijk, g.origin, h)
        U = _minkowski_fo(modes, 0.0, x, y, z)
        rU, _ = g.fo_rhs(P, U, red=True)
        et = 2e-3
        f = [_minkowski_fo(modes, s * et, x, y, z) for s in (-2, -1, 1, 2)]
        ex = (f[0] - 8.0 * f[1] + 8.0 * f[2] - f[3]) / (12.0 * et)
        errs.append(np.abs(rU - ex).reshape(NVF, -1).max(axis=1))
    algebraic = [F[n] for n in ("gxx", "gxy", "gxz", "gyy", "gyz", "gzz", "phi")]
    for v in check:
        if v in algebraic:
            # no derivative enters the first-order g~ and phi equations: exact to the data's accuracy
            assert errs[0][v] < 1e-8 and errs[1][v] < 1e-8, (I.FO_FIELDS[v], errs[0][v], errs[1][v])
        else:
            assert errs[0][v] / errs[1][v] > 10.0, (I.FO_FIELDS[v], errs[0][v], errs[1][v])


# ---- linearisation about flat space: hand-derived responses of the auxiliary equations ------------------------

PARAMS = dict(kappa1=0.3, kappa2=0.7, kappa3=0.45, e=1.7, c=1.3, tau=0.8, mu=0.35, f=0.6, eta=2.3, s=0.5,
              K0=0.0, ko_eps=0.1, shift="gamma-driver")
N, P_EDGE, M = 16, 8, 2
EPS = 1e-6


def _lin_grid():
    np_ = (N // P_EDGE, 1, 1)
    h = 1.0 / N
    g = O.Grid(P_EDGE, np_, I.patch_ijk(np_), (-0.5, -0.5, -0.5), h, "periodic")
    x, _, _ = I.point_coords(P_EDGE, g.ijk, g.origin, h)
    return g, x, h


def _symbols(h):
    th = 2.0 * math.pi * M * h
    s1 = (8.0 * math.sin(th) - math.sin(2.0 * th)) / (6.0 * h)
    ko = PARAMS["ko_eps"] / (64.0 * h) * (2.0 * math.cos(3 * th) - 12.0 * math.cos(2 * th) + 30.0 * math.cos(th) - 20.0)
    return s1, ko


def _lin_response(g, x, P, field, red, background=None):
    kx = 2.0 * math.pi * M * x
    out = []
    for sgn in (1.0, -1.0):
        U = _flat_fo(g.fo_ushape[1:])
        for name, val in (background or {}).items():
            U[F[name]] = val
        U[F[field]] += sgn * EPS * np.sin(kx)
        out.append(g.fo_rhs(P, U, red=red)[0])
    return (out[0] - out[1]) / (2.0 * EPS), np.sin(kx), np.cos(kx)


def _fo_table(field, slicing, red, s1, ko):
    """{field: (a, b)}: that right-hand side responds as a sin + b cos."""
    p = PARAMS
    ga = 2.0 if slicing == "1+log" else 1.0     # alpha^2 g(alpha) at alpha = 1
    gg = 2.0 if slicing == "1+log" else 1.0     # alpha g(alpha) at alpha = 1
    mu, s = p["mu"], p["s"]
    r = 1.0 if red else 0.0
    table = {
        # d_k K: the slicing term of A_k, (1/3) phi alpha d_k K of P_k, -4/3 alpha d K of Gamma-hat and b
        "K": {"alpha": (-ga, 0), "phi": (1.0 / 3.0, 0), "K": (ko, 0), "Ghatx": (0, -4 * s1 / 3),
              "bx": (0, -4 * s1 / 3), "Ax": (0, -ga * s1), "Px": (0, s1 / 3)},
        # d_k Theta: -2c times the slicing term of A_k
        "Theta": {"alpha": (2 * p["c"] * ga, 0), "K": (-3 * p["kappa1"] * (1 + p["kappa2"]), 0),
                  "Theta": (-p["kappa1"] * (2 + p["kappa2"]) + ko, 0), "Ghatx": (0, 2 * s1), "bx": (0, 2 * s1),
                  "Ax": (0, 2 * p["c"] * ga * s1)},
        # A_x: -d_(i A_j) in K and (trace-free) in A~
        "Ax": {"Ax": (ko, 0), "K": (0, -s1), "Axx": (0, -2 * s1 / 3), "Ayy": (0, s1 / 3), "Azz": (0, s1 / 3)},
        # P_x: the conformal-factor part of the Ricci tensor, (1/phi)(d_(i P_j) + delta_ij tr)
        "Px": {"Px": (ko, 0), "K": (0, 4 * s1), "Theta": (0, 2 * p["e"] ** 2 * s1), "Axx": (0, 2 * s1 / 3),
               "Ayy": (0, -s1 / 3), "Azz": (0, -s1 / 3)},
        # P_y (curl of P along x): the mu term of B_x^y
        "Py": {"Py": (ko, 0), "K": (0, 0), "Byx": (0, mu * s1 * r), "Bxy": (0, -mu * s1 * r),
               "Axy": (0, s1 / 2)},
        # B_x^x: Lie derivative of g~ and phi, d_(k B_l) in Gamma-hat, P_x and D
        "Bxx": {"gxx": (4.0 / 3.0, 0), "gyy": (-2.0 / 3.0, 0), "gzz": (-2.0 / 3.0, 0), "phi": (-1.0 / 3.0, 0),
                "Bxx": (ko, 0), "Ghatx": (0, (1 + s / 3) * s1), "bx": (0, (1 + s / 3) * s1), "Px": (0, -s1 / 3),
                "Dxxx": (0, 2 * s * s1 / 3), "Dxyy": (0, -s * s1 / 3), "Dxzz": (0, -s * s1 / 3)},
        # b^y: the Gamma-driver term f d_k b^i of B, f b of beta, -eta b
        "by": {"betay": (p["f"], 0), "by": (-p["eta"] + ko, 0), "Bxy": (0, p["f"] * s1)},
        # D_xxx: the g~ Laplacian of the Ricci tensor, and Z through G~^x = D_xxx
        "Dxxx": {"Dxxx": (ko, 0), "K": (0, -s1), "Theta": (0, -p["e"] ** 2 * s1 / 2), "Axx": (0, -2 * s1 / 3),
                 "Ayy": (0, s1 / 3), "Azz": (0, s1 / 3), "Ghatx": (p["kappa1"], 0), "bx": (p["kappa1"], 0)},
        # D_yxx (curl of D along x): the second mu term of B_y^x, and Z through G~^y = -D_yxx
        "Dyxx": {"Dyxx": (ko, 0), "Byx": (0, -mu * s1 * r), "Ghaty": (-p["kappa1"], 0), "by": (-p["kappa1"], 0)},
        # A~_xx: -alpha d_k A~_ij of D, and every red term (2 alpha d tr A~ of Gamma-hat, -alpha g d tr A~ of A,
        # alpha/3 g~_ij d tr A~ of D, alpha phi/3 d tr A~ of P)
        "Axx": {"gxx": (-4.0 / 3.0, 0), "gyy": (2.0 / 3.0, 0), "gzz": (2.0 / 3.0, 0), "Axx": (ko, 0),
                "Dxxx": (0, -s1 + r * s1 / 3), "Dxyy": (0, r * s1 / 3), "Dxzz": (0, r * s1 / 3),
                "Ghatx": (0, 2 * s1 * r), "bx": (0, 2 * s1 * r), "Ax": (0, -gg * s1 * r), "Px": (0, s1 / 3 * r)},
    }
    return table[field]


FO_MODES = ["K", "Theta", "Ax", "Px", "Py", "Bxx", "by", "Dxxx", "Dyxx", "Axx"]


@pytest.mark.parametrize("field", FO_MODES)
@pytest.mark.parametrize("slicing", ["1+log", "harmonic"])
@pytest.mark.parametrize("red", [True, False])
def test_linear_response_of_the_auxiliary_equations(field, slicing, red):
    g, x, h = _lin_grid()
    s1, ko = _symbols(h)
    P = O.make_params(**PARAMS, slicing=slicing)
    resp, sn, cs = _lin_response(g, x, P, field, red)
    exp = _fo_table(field, slicing, red, s1, ko)
    for v in range(NVF):
        a, b = exp.get(I.FO_FIELDS[v], (0.0, 0.0))
        want = a * sn + b * cs
        assert np.abs(resp[v] - want).max() <= 1e-7 * max(1.0, abs(a), abs(b)), (I.FO_FIELDS[v], field)


@pytest.mark.parametrize("slicing,coef", [("1+log", 2.0), ("harmonic", 4.0)])
def test_slicing_derivative_term_of_A(slicing, coef):
    """On alpha = 2, K = 0.1 (flat otherwise) a mode in A_x grows as
    -(2 alpha g + alpha^2 g') K A_x: 2 for 1+log (g = 2/alpha, g' = -2/alpha^2),
    2 alpha = 4 for harmonic slicing."""
    g, x, h = _lin_grid()
    _, ko = _symbols(h)
    P = O.make_params(**PARAMS, slicing=slicing)
    Kb = 0.1
    resp, sn, _ = _lin_response(g, x, P, "Ax", True, background={"alpha": 2.0, "K": Kb})
    assert np.abs(resp[F["Ax"]] - (-coef * Kb + ko) * sn).max() < 1e-7


# ---- evolution: the gauge wave converges at fourth order in both formulations ---------------------------------

@pytest.mark.slow
@pytest.mark.parametrize("variant", ["fo", "so-recon"])
def test_evolved_gauge_wave_converges_at_fourth_order(variant):
    P = O.make_params(**I.GAUGE_WAVE_PARAMS)
    T = 0.1
    errs = []
    for nx in (3, 6):
        g, h = _thin_grid(nx)
        x, _, _ = I.point_coords(g.p, g.ijk, g.origin, h)
        U = I.fo_gauge_wave(x)
        steps = int(round(T / (0.5 * h)))
        dt = T / steps
        for _ in range(steps):
            U, _ = g.fo_rk4_step(P, dt, U, variant=variant)
        ex = I.fo_gauge_wave(x, T)
        errs.append(np.abs(U[:NV] - ex[:NV]).max())
    assert errs[0] / errs[1] > 12.0, errs
