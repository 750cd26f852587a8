"""Gravitational-wave extraction with psi_4 (Sec. "Gravitational waves",
appendix "psi_4 in ExaGRyPE"): psi_4 on the grid (the C-ABI kernel
ccz4_psi4), sampled on a sphere by static particle tracers, and its modes
psi_4^lm = integral of the conjugate spin-weight -2 harmonic times psi_4
over the sphere.

The paper integrates over a spherical t-design (Womersley's point sets,
t = 43, N = 948: equal weights 4 pi / N). Those sets are data files that are
not available here; this module uses the product rule of Gauss-Legendre
nodes in cos(theta) and equally spaced phi, which is exact for the same
kind of integrand (spherical polynomials up to a degree set by the node
counts: 2 n_theta - 1 in cos(theta), n_phi - 1 in the azimuthal order), with
its own weights in place of 4 pi / N. Host logic (numpy) around the
library's kernels; the harmonics are the Wigner-d form of the spin-weighted
spherical harmonics in the convention where
_{-2}Y_22 = sqrt(5 / (64 pi)) (1 + cos theta)^2 exp(2 i phi)."""
import math

import numpy as np


def sphere(radius, n_theta=24, n_phi=48, centre=(0.0, 0.0, 0.0)):
    """Quadrature points on a sphere: positions (N, 3), their theta and phi,
    and weights with sum 4 pi (Gauss-Legendre in cos(theta) times the
    trapezoid rule in phi; no point on the poles)."""
    x, w = np.polynomial.legendre.leggauss(int(n_theta))
    th = np.arccos(x)
    ph = 2.0 * np.pi * np.arange(int(n_phi)) / n_phi
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    W = np.repeat(w, n_phi).reshape(TH.shape) * (2.0 * np.pi / n_phi)
    c = np.asarray(centre, float)
    pos = np.stack([c[0] + radius * np.sin(TH) * np.cos(PH), c[1] + radius * np.sin(TH) * np.sin(PH),
                    c[2] + radius * np.cos(TH)], axis=-1)
    return pos.reshape(-1, 3), TH.ravel(), PH.ravel(), W.ravel()


def swsh(s, l, m, theta, phi):
    """Spin-weighted spherical harmonic _sY_lm(theta, phi):
    (-1)^s sqrt((2l+1)/(4 pi)) d^l_{m,-s}(theta) exp(i m phi), with the
    Wigner small-d function written as its finite sum over k."""
    if l < abs(s) or abs(m) > l:
        raise ValueError("need l >= |s| and |m| <= l")
    theta = np.asarray(theta, float)
    phi = np.asarray(phi, float)
    a = -s  # d^l_{m, a}
    c, sn = np.cos(theta / 2.0), np.sin(theta / 2.0)
    f = math.factorial
    pre = math.sqrt(f(l + m) * f(l - m) * f(l + a) * f(l - a))
    d = np.zeros_like(theta)
    for k in range(max(0, m - a), min(l + m, l - a) + 1):
        coef = (-1) ** k * pre / (f(l + m - k) * f(l - a - k) * f(k) * f(k + a - m))
        d = d + coef * c ** (2 * l + m - a - 2 * k) * sn ** (2 * k + a - m)
    return (-1) ** s * math.sqrt((2 * l + 1) / (4.0 * math.pi)) * d * np.exp(1j * m * phi)


def modes(values, theta, phi, weights, lmax=4, s=-2):
    """psi^lm = sum_q w_q conj(_sY_lm(theta_q, phi_q)) values_q for
    |s| <= l <= lmax, |m| <= l: the quadrature of the paper's mode integral."""
    values = np.asarray(values)
    out = {}
    for l in range(abs(s), lmax + 1):
        for m in range(-l, l + 1):
            out[(l, m)] = complex(np.sum(weights * np.conj(swsh(s, l, m, theta, phi)) * values))
    return out


def sample(grid, positions, buf="RHS"):
    """psi_4 = field 0 + i field 1 of state buffer buf (as ccz4_psi4 writes
    it) at the positions, by static tracers (trilinear projection)."""
    from .ccz4 import Tracers
    tr = Tracers(grid, positions, vel_field=-1)
    tr.step(buf, 0.0)
    _, val = tr.read()
    tr.close()
    return val[:, 0] + 1j * val[:, 1]


def extract(grid, radius, in_buf="U", scratch="RHS", centre=(0.0, 0.0, 0.0), lmax=4, n_theta=24, n_phi=48):
    """The psi_4 modes on a sphere of the given radius around `centre` (the
    tetrad's centre too): psi_4 of in_buf into the scratch state buffer,
    sampled on the quadrature points, integrated against the spin-weight -2
    harmonics. Returns ({(l, m): complex}, psi_4 at the points)."""
    grid.psi4(in_buf, scratch, centre)
    pos, th, ph, w = sphere(radius, n_theta, n_phi, centre)
    vals = sample(grid, pos, scratch)
    return modes(vals, th, ph, w, lmax), vals
