"""Exact CCZ4 data of Minkowski space in time-dependent "wobbly" coordinates.

Flat spacetime written in coordinates x^mu related to inertial ones X^A by
X^A = x^A + xi^A(x), with xi a few smooth Fourier modes periodic on the unit
cube. It is an exact vacuum solution, so in any such coordinates:
  - the constraints H and M vanish;
  - the time derivative of every non-gauge CCZ4 variable (g~, phi, A~, K,
    Theta, Gamma-hat) is what the evolution equations must return, since the
    equations hold for any lapse and shift once Z = 0;
  - lapse, shift, extrinsic curvature and the intrinsic curvature of the
    slices are all non-trivial, which exercises the shift, Ricci and K terms
    that the gauge wave leaves at zero.
The 3+1 quantities follow from the 4-metric g = J^T eta J by textbook ADM
relations; the time derivative is taken by a fourth-order central difference
in t of these exact values (its error, ~1e-12, is far below the spatial
discretisation errors these tests measure).

Test infrastructure only: independent of the oracle and of the CUDA path.
"""
import numpy as np

from paper_2406_11626_gb300.inputs import NV, IDX

_SYM = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))


def make_modes(seed, amp=0.02, n=2, time_dep=True):
    """Per component A = 0..3 (t, x, y, z): n modes (amplitude, omega, k[3], phase)."""
    rng = np.random.default_rng(seed)
    modes = []
    for A in range(4):
        for _ in range(n):
            k = rng.integers(-1, 2, size=3)
            if not k.any():
                k[rng.integers(0, 3)] = 1
            w = rng.uniform(-2.0, 2.0) if time_dep else 0.0
            modes.append((A, rng.uniform(-amp, amp), w, k.astype(np.float64), rng.uniform(0, 2 * np.pi)))
    return modes


def _jac(modes, t, x, y, z):
    """J[..., A, mu] = delta + d_mu xi^A and dJ[..., lam, A, mu] = d_lam d_mu xi^A."""
    shp = np.shape(x)
    J = np.zeros(shp + (4, 4))
    dJ = np.zeros(shp + (4, 4, 4))
    for A in range(4):
        J[..., A, A] = 1.0
    for A, a, w, k, ph in modes:
        c = np.array([w, 2 * np.pi * k[0], 2 * np.pi * k[1], 2 * np.pi * k[2]])
        th = w * t + c[1] * x + c[2] * y + c[3] * z + ph
        cs, sn = np.cos(th), np.sin(th)
        for mu in range(4):
            J[..., A, mu] += a * c[mu] * cs
            for lam in range(4):
                dJ[..., lam, A, mu] += -a * c[lam] * c[mu] * sn
    return J, dJ


def ccz4_state(modes, t, x, y, z):
    """All 25 CCZ4 variables at time t on the given points (b^i = 0)."""
    eta = np.diag([-1.0, 1.0, 1.0, 1.0])
    J, dJ = _jac(modes, t, x, y, z)
    g4 = np.einsum("...am,ab,...bn->...mn", J, eta, J)
    dg4 = (np.einsum("...lam,ab,...bn->...lmn", dJ, eta, J)
           + np.einsum("...am,ab,...lbn->...lmn", J, eta, dJ))
    gam = g4[..., 1:, 1:]
    ig = np.linalg.inv(gam)
    beta_l = g4[..., 0, 1:]
    beta_u = np.einsum("...ij,...j->...i", ig, beta_l)
    alpha = np.sqrt(np.einsum("...i,...i->...", beta_l, beta_u) - g4[..., 0, 0])
    dgam = dg4[..., 1:, 1:, 1:]         # [k, i, j] spatial derivatives of gamma_ij
    dtgam = dg4[..., 0, 1:, 1:]
    dbeta_l = dg4[..., 1:, 0, 1:]       # [k, j] = d_k beta_j
    # chr_[k, i, j] = 1/2 g^kl (d_i g_jl + d_j g_il - d_l g_ij), dgam[a, b, c] = d_a g_bc
    T = (np.einsum("...ijl->...lij", dgam) + np.einsum("...jil->...lij", dgam) - dgam)
    chr_ = 0.5 * np.einsum("...kl,...lij->...kij", ig, T)
    Db = dbeta_l - np.einsum("...kij,...k->...ij", chr_, beta_l)   # D_i beta_j
    Kij = -(dtgam - Db - np.swapaxes(Db, -1, -2)) / (2.0 * alpha[..., None, None])
    det = np.linalg.det(gam)
    phi = det ** (-1.0 / 6.0)
    gt = phi[..., None, None] ** 2 * gam
    Ktr = np.einsum("...ij,...ij->...", ig, Kij)
    At = phi[..., None, None] ** 2 * (Kij - Ktr[..., None, None] * gam / 3.0)
    igt = ig / phi[..., None, None] ** 2
    trd = np.einsum("...ab,...kab->...k", ig, dgam)
    dgt = phi[..., None, None, None] ** 2 * (dgam - gam[..., None, :, :] * trd[..., :, None, None] / 3.0)
    # G~^i = g~^jk G~^i_jk, G~^i_jk = 1/2 g~^il (d_j g~_kl + d_k g~_jl - d_l g~_jk)
    Gl = 0.5 * (np.einsum("...jkl->...ljk", dgt) + np.einsum("...kjl->...ljk", dgt) - dgt)
    # Gl[l, j, k] = 1/2 (d_j g~_kl + d_k g~_jl - d_l g~_jk)
    Gam = np.einsum("...il,...ljk->...ijk", igt, Gl)
    Gc = np.einsum("...jk,...ijk->...i", igt, Gam)
    Q = np.zeros((NV,) + np.shape(x))
    for s, (i, j) in enumerate(_SYM):
        Q[IDX["gxx"] + s] = gt[..., i, j]
        Q[IDX["Axx"] + s] = At[..., i, j]
    Q[IDX["alpha"]] = alpha
    for i in range(3):
        Q[IDX["betax"] + i] = beta_u[..., i]
        Q[IDX["Ghatx"] + i] = Gc[..., i]
    Q[IDX["phi"]] = phi
    Q[IDX["K"]] = Ktr
    return Q


def ccz4_state_dt(modes, t, x, y, z, eps=2e-3):
    """Fourth-order central difference in t of ``ccz4_state``."""
    f = [ccz4_state(modes, t + s * eps, x, y, z) for s in (-2, -1, 1, 2)]
    return (f[0] - 8.0 * f[1] + 8.0 * f[2] - f[3]) / (12.0 * eps)


# fields whose evolution equations hold for any gauge once Z = 0
PHYSICAL = [IDX[n] for n in ("gxx", "gxy", "gxz", "gyy", "gyz", "gzz", "phi", "Axx", "Axy", "Axz",
                             "Ayy", "Ayz", "Azz", "K", "Theta", "Ghatx", "Ghaty", "Ghatz")]
