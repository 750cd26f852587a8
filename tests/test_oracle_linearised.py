"""Pin of the gauge and damping terms of the oracle's CCZ4 right-hand side
by its linearisation about flat space (Sec. "CCZ4 formulation", the
second-order system with the red terms removed).

A single Fourier mode eps*sin(k x) in one field of flat space (g~ = delta,
alpha = phi = 1, everything else 0) makes every other term of the evolution
equations quadratic in eps, so the linear response of each right-hand side
is a constant times the mode or times one of its FD4 derivatives. The
constants below are read off the printed equations by hand: the 1+log or
harmonic slicing, the Gamma-driver (f, eta, s), the Theta and Z damping
(kappa1, kappa2, c, e), the relaxation of det g~ (tau), the Lie-derivative,
Ricci and conformal-factor parts. On a periodic
grid the FD4 stencils act on the mode exactly as their Fourier symbols
(textbook): d1 sin = s1 cos with s1 = (8 sin(kh) - sin(2kh)) / (6h), d2 sin
= -s2 sin with s2 = (30 - 32 cos(kh) + 2 cos(2kh)) / (12 h^2), and the
dissipation adds ko * sin to the perturbed field itself with ko = eps_KO/(64h)
(2 cos 3kh - 12 cos 2kh + 30 cos kh - 20). The response is taken as the
central difference (rhs(+eps) - rhs(-eps)) / (2 eps), exact up to O(eps^2).

Nothing here restates the oracle's code: a dropped term, a wrong sign, a
wrong coefficient or a parameter in the wrong equation changes one of the
entries (every parameter enters with a distinct, non-default value)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2406_11626_gb300 import inputs as I

# every parameter distinct from the others and from its default
PARAMS = dict(kappa1=0.3, kappa2=0.7, kappa3=0.45, e=1.7, c=1.3, tau=0.8, mu=0.2, f=0.6, eta=2.3, s=0.5,
              K0=0.0, ko_eps=0.1, shift="gamma-driver")
N, P_EDGE, M = 16, 8, 2          # 16 points along x in two patches; mode number 2 on [-1/2, 1/2)
EPS = 1e-6


def _grid():
    np_ = (N // P_EDGE, 1, 1)
    h = 1.0 / N
    g = O.Grid(P_EDGE, np_, I.patch_ijk(np_), (-0.5, -0.5, -0.5), h, "periodic")
    x, _, _ = I.point_coords(P_EDGE, g.ijk, g.origin, h)
    return g, x, h


def _symbols(h):
    th = 2.0 * math.pi * M * h
    s1 = (8.0 * math.sin(th) - math.sin(2.0 * th)) / (6.0 * h)
    s2 = (30.0 - 32.0 * math.cos(th) + 2.0 * math.cos(2.0 * th)) / (12.0 * h * h)
    ko = PARAMS["ko_eps"] / (64.0 * h) * (2.0 * math.cos(3 * th) - 12.0 * math.cos(2 * th) + 30.0 * math.cos(th) - 20.0)
    return s1, s2, ko


def _response(g, x, P, field):
    kx = 2.0 * math.pi * M * x
    out = []
    for sgn in (1.0, -1.0):
        U = I.flat(g.ushape[1:])
        U[I.IDX[field]] += sgn * EPS * np.sin(kx)
        out.append(g.rhs(P, U)[0])
    return (out[0] - out[1]) / (2.0 * EPS), np.sin(kx), np.cos(kx)


def _expected(field, slicing, s1, s2, ko):
    """{field: (a, b)}: the response of that right-hand side is a sin + b cos."""
    p = PARAMS
    ga = 2.0 if slicing == "1+log" else 1.0   # alpha^2 g(alpha) at alpha = 1
    k1, k2 = p["kappa1"], p["kappa2"]
    table = {
        # lapse: -grad grad alpha in K (trace) and in A~ (trace-free part)
        "alpha": {"alpha": (ko, 0), "K": (s2, 0), "Axx": (2 * s2 / 3, 0), "Ayy": (-s2 / 3, 0), "Azz": (-s2 / 3, 0)},
        # K: slicing, volume factor of phi, -4/3 alpha d_i K in Gamma-hat and b
        "K": {"alpha": (-ga, 0), "phi": (1.0 / 3.0, 0), "K": (ko, 0), "Ghatx": (0, -4 * s1 / 3),
              "bx": (0, -4 * s1 / 3)},
        # Theta: c-terms of the slicing, kappa1 damping in K and Theta, 2 alpha d_i Theta in Gamma-hat
        "Theta": {"alpha": (2 * p["c"] * ga, 0), "K": (-3 * k1 * (1 + k2), 0), "Theta": (-k1 * (2 + k2) + ko, 0),
                  "Ghatx": (0, 2 * s1), "bx": (0, 2 * s1)},
        # longitudinal shift: Lie derivative of g~ and phi, d_k d_k beta + s/3 d_i d_k beta^k
        "betax": {"gxx": (0, 4 * s1 / 3), "gyy": (0, -2 * s1 / 3), "gzz": (0, -2 * s1 / 3), "phi": (0, -s1 / 3),
                  "betax": (ko, 0), "Ghatx": (-(1 + p["s"] / 3) * s2, 0), "bx": (-(1 + p["s"] / 3) * s2, 0)},
        # transverse shift
        "betay": {"gxy": (0, s1), "betay": (ko, 0), "Ghaty": (-s2, 0), "by": (-s2, 0)},
        # Gamma-driver: d_t beta = f b, d_t b = ... - eta b
        "by": {"betay": (p["f"], 0), "by": (-p["eta"] + ko, 0)},
        # transverse Gamma-hat: Z damping, g~_k(i d_j) Gamma-hat^k in the Ricci tensor
        "Ghaty": {"Ghaty": (-k1 + ko, 0), "Axy": (0, s1 / 2), "by": (-k1, 0)},
        # longitudinal Gamma-hat: also the trace R + 2 nabla_k Z^k in K and Theta
        "Ghatx": {"Ghatx": (-k1 + ko, 0), "Axx": (0, 2 * s1 / 3), "Ayy": (0, -s1 / 3), "Azz": (0, -s1 / 3),
                  "K": (0, s1), "Theta": (0, 0.5 * p["e"] ** 2 * s1), "bx": (-k1, 0)},
        # transverse metric: -1/2 g~^kl d_k d_l g~_ij, and Z_i = -G~_i / 2 damped by kappa1
        "gxy": {"gxy": (ko, 0), "Axy": (s2 / 2, 0), "Ghaty": (0, k1 * s1), "by": (0, k1 * s1)},
        # diagonal metric: det g~ - 1 = eps sin relaxed on the time scale tau in every diagonal
        # component; R_xx + 2 nabla_(x Z_x) = -1/2 d_x d_x g~_xx, its trace in K and Theta, its
        # trace-free part in A~; G~^x = 1/2 d_x g~_xx feeds the Z damping
        "gxx": {"gxx": (-1.0 / p["tau"] + ko, 0), "gyy": (-1.0 / p["tau"], 0), "gzz": (-1.0 / p["tau"], 0),
                "Axx": (s2 / 3, 0), "Ayy": (-s2 / 6, 0), "Azz": (-s2 / 6, 0), "K": (s2 / 2, 0),
                "Theta": (0.25 * p["e"] ** 2 * s2, 0), "Ghatx": (0, k1 * s1 / 2), "bx": (0, k1 * s1 / 2)},
        # conformal factor: (1/phi)(nabla~_i nabla~_j phi + g~_ij g~^kl nabla~_k nabla~_l phi), trace 4 d^2 phi
        "phi": {"phi": (ko, 0), "K": (-4 * s2, 0), "Theta": (-2 * p["e"] ** 2 * s2, 0), "Axx": (-2 * s2 / 3, 0),
                "Ayy": (s2 / 3, 0), "Azz": (s2 / 3, 0)},
    }
    return table[field]


@pytest.mark.parametrize("slicing", ["1+log", "harmonic"])
@pytest.mark.parametrize("field", ["alpha", "K", "Theta", "betax", "betay", "by", "Ghaty", "Ghatx", "gxy", "gxx",
                                   "phi"])
def test_linear_response_about_flat_space(field, slicing):
    g, x, h = _grid()
    P = O.make_params(**dict(PARAMS, slicing=slicing))
    r, S, C = _response(g, x, P, field)
    s1, s2, ko = _symbols(h)
    want = _expected(field, slicing, s1, s2, ko)
    scale = max(s2, 1.0)
    for v, name in enumerate(I.FIELDS):
        a, b = want.get(name, (0.0, 0.0))
        err = np.abs(r[v] - (a * S + b * C)).max()
        assert err <= 1e-7 * scale, (field, name, err, a, b)


def test_zero_shift_freezes_beta_and_b():
    """With the zero-shift option the evolution equations of beta and b are
    switched off: their right-hand sides keep only the numerical dissipation
    of their own perturbation; the other responses are unchanged."""
    g, x, h = _grid()
    s1, s2, ko = _symbols(h)
    P = O.make_params(**dict(PARAMS, slicing="1+log", shift="zero"))
    for field in ("by", "K", "Ghaty", "betax"):
        r, S, C = _response(g, x, P, field)
        for name in ("betax", "betay", "betaz", "bx", "by", "bz"):
            want = ko * S if name == field else 0.0 * S
            assert np.abs(r[I.IDX[name]] - want).max() <= 1e-7 * s2, (field, name)
    r, S, C = _response(g, x, P, "Ghaty")
    assert np.abs(r[I.IDX["Axy"]] - 0.5 * s1 * C).max() <= 1e-7 * s2


def test_bilinear_response_pins_kappa3_and_shift_advection():
    """The kappa3 terms 2 kappa3 (2/3 g~^ij Z_j B_k^k - g~^jk Z_j B_k^i) are
    products of Z and d beta, so they show in the mixed second-order response
    to a longitudinal Gamma-hat mode (Z_x = Gamma-hat^x / 2) and a shift mode
    of another wavenumber: d_t Gamma-hat^x gains beta d_x Gamma-hat^x
    (advection) - kappa3/3 Gamma-hat^x d_x beta^x; in d_t b^x the advection
    cancels (d_t b - beta d b = d_t Gamma-hat - beta d Gamma-hat - eta b) and
    only the kappa3 part stays; no other right-hand side has a product of
    the two. Mixed central difference in (eps1, eps2)."""
    g, x, h = _grid()
    P = O.make_params(**dict(PARAMS, slicing="1+log"))
    k = 2.0 * math.pi * M
    e1 = e2 = 1e-4
    r = {}
    for a in (1.0, -1.0):
        for b in (1.0, -1.0):
            U = I.flat(g.ushape[1:])
            U[I.IDX["Ghatx"]] += a * e1 * np.sin(k * x)
            U[I.IDX["betax"]] += b * e2 * np.sin(2 * k * x)
            r[a, b] = g.rhs(P, U)[0]
    mixed = (r[1, 1] - r[1, -1] - r[-1, 1] + r[-1, -1]) / (4.0 * e1 * e2)

    def d1(kk):  # FD4 symbol of d/dx on sin(kk x)
        return (8.0 * math.sin(kk * h) - math.sin(2 * kk * h)) / (6.0 * h)

    adv = np.sin(2 * k * x) * d1(k) * np.cos(k * x)                 # beta^x d_x Gamma-hat^x
    k3 = -PARAMS["kappa3"] / 3.0 * np.sin(k * x) * d1(2 * k) * np.cos(2 * k * x)
    want = {"Ghatx": adv + k3, "bx": k3}
    scale = d1(2 * k)
    for v, name in enumerate(I.FIELDS):
        err = np.abs(mixed[v] - want.get(name, 0.0)).max()
        assert err <= 1e-6 * scale, (name, err)
