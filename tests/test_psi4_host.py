"""Host side of the psi_4 extraction: the spin-weight -2 harmonics against
their published closed forms for l = 2 and, for spin weight 0, against the
ordinary spherical harmonics; the sphere quadrature (orthonormality of the
harmonics, exactly); and the recovery of known modes from a field on the
sphere."""
import math

import numpy as np
import pytest

from paper_2406_11626_gb300 import psi4 as P


def _angles(n=200, seed=0):
    rng = np.random.default_rng(seed)
    return np.arccos(rng.uniform(-1, 1, n)), rng.uniform(0, 2 * np.pi, n)


def test_spin_minus_two_harmonics_have_their_closed_forms():
    th, ph = _angles()
    c, s = np.cos(th), np.sin(th)
    want = {2: math.sqrt(5 / (64 * math.pi)) * (1 + c) ** 2 * np.exp(2j * ph),
            1: math.sqrt(5 / (16 * math.pi)) * s * (1 + c) * np.exp(1j * ph),
            0: math.sqrt(15 / (32 * math.pi)) * s ** 2,
            -1: math.sqrt(5 / (16 * math.pi)) * s * (1 - c) * np.exp(-1j * ph),
            -2: math.sqrt(5 / (64 * math.pi)) * (1 - c) ** 2 * np.exp(-2j * ph)}
    for m, w in want.items():
        np.testing.assert_allclose(P.swsh(-2, 2, m, th, ph), w, rtol=1e-13, atol=1e-15)


def test_spin_zero_is_the_ordinary_harmonic():
    sp = pytest.importorskip("scipy.special")
    th, ph = _angles(seed=1)
    for l in range(0, 5):
        for m in range(-l, l + 1):
            if hasattr(sp, "sph_harm_y"):
                y = sp.sph_harm_y(l, m, th, ph)
            else:
                y = sp.sph_harm(m, l, ph, th)
            np.testing.assert_allclose(P.swsh(0, l, m, th, ph), y, rtol=1e-12, atol=1e-14)


def test_quadrature_makes_the_harmonics_orthonormal():
    pos, th, ph, w = P.sphere(2.0, n_theta=12, n_phi=24)
    assert abs(w.sum() - 4 * np.pi) < 1e-12
    np.testing.assert_allclose(np.linalg.norm(pos, axis=1), 2.0, rtol=1e-14)
    Y = {(l, m): P.swsh(-2, l, m, th, ph) for l in range(2, 6) for m in range(-l, l + 1)}
    for a, ya in Y.items():
        for b, yb in Y.items():
            ip = np.sum(w * ya * np.conj(yb))
            assert abs(ip - (1.0 if a == b else 0.0)) < 1e-12, (a, b, ip)


def test_modes_of_a_known_superposition_are_recovered():
    _, th, ph, w = P.sphere(1.0, n_theta=16, n_phi=32)
    coef = {(2, 2): 0.3 - 0.1j, (2, -2): 0.3 + 0.1j, (3, 1): -0.05j, (4, 0): 0.02}
    f = sum(c * P.swsh(-2, l, m, th, ph) for (l, m), c in coef.items())
    got = P.modes(f, th, ph, w, lmax=5)
    for k, v in got.items():
        assert abs(v - coef.get(k, 0.0)) < 1e-13, (k, v)
