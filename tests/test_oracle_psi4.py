"""Pins of the oracle's psi_4 (appendix "psi_4 in ExaGRyPE"): against the
Weyl tensor itself, computed by brute force from an exact vacuum 4-metric
(a boosted Schwarzschild black hole in Kerr-Schild form, centred off the
tetrad's origin) and contracted with the appendix's null tetrad, converging
at fourth order; and against closed forms on flat metrics that excite the
terms that spacetime leaves out (Theta, Z, a K_ij that varies in space)."""
import numpy as np
import pytest

import oracle as O
import weyl_reference as W
from paper_2406_11626_gb300 import inputs as I

SYM = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]


def _grid(n_side, half=1.0, p=6):
    cfg = I.single_puncture_config(p=p, n_side=n_side, half_width=half)
    og = O.Grid(cfg.p, cfg.np, cfg.ijk(), cfg.origin, cfg.dx, cfg.bc)
    x, y, z = I.point_coords(cfg.p, cfg.ijk(), cfg.origin, cfg.dx)
    g = I.ghost_positions(cfg.N, cfg.origin, cfg.dx)
    return cfg, og, (x, y, z), g


def test_psi4_is_the_weyl_tensor_on_the_tetrad_at_fourth_order():
    st = W.BoostedKS(M=1.0, c0=(3.0, 0.5, -0.2), vel=(0.0, 0.3, 0.0))
    rng = np.random.default_rng(0)
    errs = []
    for n_side in (3, 6):
        cfg, og, (x, y, z), (gx, gy, gz) = _grid(n_side)
        U = W.ccz4_state(st, x, y, z)
        G = W.ccz4_state(st, gx, gy, gz)
        ps = og.psi4(U, G)
        # the same physical points at both resolutions: the coarse grid's cell
        # centres are not fine centres, so sample each grid near fixed spots
        sel = rng.choice(x.size, 40, replace=False)
        pts = np.stack([x.ravel()[sel], y.ravel()[sel], z.ravel()[sel]], 1)
        ref, ric = W.psi4(st, pts)
        assert ric < 1e-8                      # the reference is vacuum to its differencing error
        got = ps[0].ravel()[sel] + 1j * ps[1].ravel()[sel]
        errs.append(np.abs(got - ref).max() / np.abs(ref).max())
        assert np.abs(ref).max() > 0.05        # the tetrad is not aligned with the hole: psi_4 is large
    assert errs[0] < 2e-4 and errs[1] < 1.5e-5 and errs[0] / errs[1] > 8.0, errs


def _flat_state(shape, At=None, K=0.0, Theta=0.0, Gh=None):
    U = np.zeros((I.NV,) + shape)
    for c, (i, j) in enumerate(SYM):
        U[I.IDX["gxx"] + c] = 1.0 if i == j else 0.0
        if At is not None:
            U[I.IDX["Axx"] + c] = At[c]
    U[I.IDX["alpha"]] = 1.0
    U[I.IDX["phi"]] = 1.0
    U[I.IDX["K"]] = K
    U[I.IDX["Theta"]] = Theta
    if Gh is not None:
        for i in range(3):
            U[I.IDX["Ghatx"] + i] = Gh[i]
    return U


def _flat_psi4(E, B, x, y, z):
    """(E - i B)_ij mbar^i mbar^j for flat metric fields E, B (3, 3, ...)
    with the appendix's triad at (x, y, z) from the origin."""
    X = np.stack([x, y, z])
    v = np.stack([-y, x, np.zeros_like(x)])
    v = v / np.sqrt((v * v).sum(0))
    u = X - (X * v).sum(0) * v
    u = u / np.sqrt((u * u).sum(0))
    w = np.cross(v, u, axis=0)
    m = (w - 1j * v) / np.sqrt(2.0)
    return np.einsum('ij...,i...,j...->...', E - 1j * B, m, m)


def _tf(X):
    tr = X[0, 0] + X[1, 1] + X[2, 2]
    return X - np.eye(3)[:, :, None, None, None, None] * tr / 3.0


def test_theta_and_extrinsic_curvature_terms_on_a_flat_metric():
    """Constant A~, K and Theta on the flat metric: E = (-K K + K (K - Theta))^TF,
    B = 0 (no gradients)."""
    cfg, og, (x, y, z), (gx, gy, gz) = _grid(3)
    A = np.array([0.3, -0.1, 0.05, -0.2, 0.15, -0.1])
    K, Th = 0.4, 0.25
    U = _flat_state(x.shape, At=A, K=K, Theta=Th)
    G = _flat_state(gx.shape, At=A, K=K, Theta=Th)
    ps = og.psi4(U, G)
    Kij = np.zeros((3, 3))
    for c, (i, j) in enumerate(SYM):
        Kij[i, j] = Kij[j, i] = A[c]
    Kij += np.eye(3) * K / 3.0
    E0 = -Kij @ Kij + Kij * (K - Th)
    E0 = E0 - np.eye(3) * np.trace(E0) / 3.0
    E = np.broadcast_to(E0[:, :, None, None, None, None], (3, 3) + x.shape)
    want = _flat_psi4(E, np.zeros_like(E), x, y, z)
    np.testing.assert_allclose(ps[0] + 1j * ps[1], want, rtol=0, atol=1e-12)


def test_z_term_on_a_flat_metric():
    """Gamma-hat^i = f^i(x) on the flat metric: Z_i = f_i / 2, E = (d_(i Z_j))^TF,
    B = 0. f is cubic, so the FD4 derivatives are exact."""
    cfg, og, (x, y, z), (gx, gy, gz) = _grid(3)

    def f(x, y, z):
        return np.stack([0.2 * y * y - 0.1 * x * z, 0.3 * x * y + 0.05 * z ** 3, -0.2 * x + 0.1 * y * z])

    def df(x, y, z):   # df[i][j] = d_j f^i
        o = np.zeros_like(x)
        return np.array([[-0.1 * z, 0.4 * y, -0.1 * x],
                         [0.3 * y, 0.3 * x, 0.15 * z * z],
                         [-0.2 + o, 0.1 * z, 0.1 * y]])
    U = _flat_state(x.shape, Gh=f(x, y, z))
    G = _flat_state(gx.shape, Gh=f(gx, gy, gz))
    ps = og.psi4(U, G)
    d = df(x, y, z)
    DZ = 0.25 * (d + np.swapaxes(d, 0, 1))
    want = _flat_psi4(_tf(DZ), np.zeros_like(DZ), x, y, z)
    np.testing.assert_allclose(ps[0] + 1j * ps[1], want, rtol=0, atol=1e-11)


def test_magnetic_part_of_a_linearly_varying_curvature():
    """A~_ij linear in position on the flat metric (K = Theta = 0):
    D_m K_jn = d_m A~_jn, B_ij = 1/2 (eps_mni d_m K_jn + eps_mnj d_m K_in)^TF and
    E = (-K K)^TF (K K = 0 trace term, K = 0)."""
    cfg, og, (x, y, z), (gx, gy, gz) = _grid(3)
    rng = np.random.default_rng(3)
    c0 = rng.uniform(-0.2, 0.2, 6)
    c1 = rng.uniform(-0.3, 0.3, (6, 3))

    def A(x, y, z):
        return np.stack([c0[c] + c1[c, 0] * x + c1[c, 1] * y + c1[c, 2] * z for c in range(6)])
    U = _flat_state(x.shape, At=A(x, y, z))
    G = _flat_state(gx.shape, At=A(gx, gy, gz))
    ps = og.psi4(U, G)
    Km = np.zeros((3, 3) + x.shape)
    dK = np.zeros((3, 3, 3))   # dK[m, j, n] = d_m K_jn
    a = A(x, y, z)
    for c, (i, j) in enumerate(SYM):
        Km[i, j] = Km[j, i] = a[c]
        for m in range(3):
            dK[m, i, j] = dK[m, j, i] = c1[c, m]
    eps = np.zeros((3, 3, 3))
    for i in range(3):
        for j in range(3):
            for k in range(3):
                eps[i, j, k] = (i - j) * (j - k) * (k - i) / 2.0
    B0 = 0.5 * (np.einsum('mni,mjn->ij', eps, dK) + np.einsum('mnj,min->ij', eps, dK))
    B0 = B0 - np.eye(3) * np.trace(B0) / 3.0
    B = np.broadcast_to(B0[:, :, None, None, None, None], (3, 3) + x.shape)
    E = -np.einsum('im...,mj...->ij...', Km, Km)
    want = _flat_psi4(_tf(E), B, x, y, z)
    np.testing.assert_allclose(ps[0] + 1j * ps[1], want, rtol=0, atol=1e-12)


def test_a_schwarzschild_hole_at_the_centre_has_no_psi4():
    """Brill-Lindquist data of one hole at the tetrad's centre: psi_4 = 0
    (the radial tetrad is aligned with the principal null directions); away
    from the puncture the discrete value falls at fourth order."""
    errs = []
    for n_side in (4, 8):
        cfg, og, (x, y, z), _ = _grid(n_side, half=4.0)
        U, G = I.initial_state(cfg)
        ps = og.psi4(U, G)
        r = np.sqrt(x * x + y * y + z * z)
        far = (r > 2.0) & (r < 3.0)
        errs.append(np.abs(ps[:, far]).max())
    assert errs[0] / errs[1] > 8.0, errs     # 11.6 measured; second order would give 4
