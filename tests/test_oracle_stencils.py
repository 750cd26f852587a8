"""Pins of the oracle's FD4 stencils (Eqs. exa_fd4_central_difference and
exa_fd4_ko) against exact calculus on polynomials and closed-form
truncation errors."""
import numpy as np
import pytest

import oracle as O
from paper_2406_11626_gb300 import inputs as I

P_EDGE = 15
H = 0.1


def _grid():
    return O.Grid(P_EDGE, (1, 1, 1), I.patch_ijk((1, 1, 1)), (0.0, 0.0, 0.0), H, "copy")


def _centre_index():
    c = P_EDGE // 2
    return (c * P_EDGE + c) * P_EDGE + c


def _coords():
    return I.point_coords(P_EDGE, I.patch_ijk((1, 1, 1)), (0.0, 0.0, 0.0), H)


def _poly_fields(seed, deg=4):
    """25 random polynomials of degree <= deg in each coordinate separately,
    with their exact first and second derivatives at the centre point."""
    rng = np.random.default_rng(seed)
    x, y, z = _coords()
    c = P_EDGE // 2
    xc = yc = zc = (c + 0.5) * H
    U = np.zeros((I.NV,) + x.shape)
    d1 = np.zeros((I.NV, 3))
    d2 = np.zeros((I.NV, 3, 3))
    for v in range(I.NV):
        coef = rng.uniform(-1, 1, size=(deg + 1,) * 3)
        for a in range(deg + 1):
            for b in range(deg + 1):
                for cc in range(deg + 1):
                    w = coef[a, b, cc]
                    U[v] += w * x ** a * y ** b * z ** cc
                    e = [a, b, cc]
                    p = [xc, yc, zc]

                    def mono(ex):
                        if min(ex) < 0:
                            return 0.0
                        return p[0] ** ex[0] * p[1] ** ex[1] * p[2] ** ex[2]

                    for k in range(3):
                        ek = list(e)
                        ek[k] -= 1
                        d1[v, k] += w * e[k] * mono(ek)
                        for l in range(3):
                            el = list(ek)
                            el[l] -= 1
                            fac = e[k] * (e[l] - (1 if k == l else 0))
                            d2[v, k, l] += w * fac * mono(el)
    return U, d1, d2


def test_stencils_exact_on_degree4_polynomials():
    g = _grid()
    for seed in range(3):
        U, d1x, d2x = _poly_fields(seed)
        d1, d2, ko = g.point_derivs(U, None, _centre_index(), ko_eps=0.7)
        scale = max(1.0, np.abs(d2x).max())
        np.testing.assert_allclose(d1, d1x, rtol=0, atol=1e-11 * scale)
        np.testing.assert_allclose(d2, d2x, rtol=0, atol=1e-9 * scale)
        np.testing.assert_allclose(ko, 0.0, rtol=0, atol=1e-9 * scale)


def test_stencil_truncation_errors_closed_form():
    """D1(x^5) = 5x^4 - 4h^4; D2(x^6) = 30x^4 - 8h^4; the mixed stencil is the
    product of first-derivative stencils; KO(x^6) = eps/(64h) * 720 h^6 (the
    sixth difference of x^6), and KO is the sum over the three directions."""
    g = _grid()
    x, y, z = _coords()
    xc = (P_EDGE // 2 + 0.5) * H
    U = I.flat(x.shape)
    U[0] = x ** 5
    U[1] = x ** 6
    U[2] = x ** 5 * y
    U[3] = x ** 6 + y ** 6 + z ** 6
    eps = 0.3
    d1, d2, ko = g.point_derivs(U, None, _centre_index(), ko_eps=eps)
    assert d1[0, 0] - 5 * xc ** 4 == pytest.approx(-4 * H ** 4, rel=1e-6)
    assert d2[1, 0, 0] - 30 * xc ** 4 == pytest.approx(-8 * H ** 4, rel=1e-5)
    assert d2[2, 0, 1] - 5 * xc ** 4 == pytest.approx(-4 * H ** 4, rel=1e-6)
    assert d2[2, 1, 0] == pytest.approx(d2[2, 0, 1], rel=1e-13)
    assert ko[1] == pytest.approx(eps / (64 * H) * 720 * H ** 6, rel=1e-6)
    assert ko[3] == pytest.approx(3 * eps / (64 * H) * 720 * H ** 6, rel=1e-6)
    assert ko[0] == pytest.approx(0.0, abs=1e-10)


def test_ko_is_dissipative_on_the_nyquist_mode():
    """On Q = (-1)^i the sixth difference is -64 (-1)^i, so KO = -eps/h Q: the
    highest mode is damped at rate eps/h (the sign the paper prints)."""
    g = _grid()
    x, y, z = _coords()
    U = I.flat(x.shape)
    i = np.rint(x / H - 0.5).astype(int)
    U[5] = (-1.0) ** i
    d1, d2, ko = g.point_derivs(U, None, _centre_index(), ko_eps=0.25)
    q = U[5].ravel()[_centre_index()]
    assert ko[5] == pytest.approx(-0.25 / H * q, rel=1e-12)
