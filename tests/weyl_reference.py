"""Test support: a boosted Schwarzschild black hole in Kerr-Schild form (an
exact vacuum spacetime), its 3+1 data turned into CCZ4 variables, and psi_4
by brute force: the 4D Riemann tensor (= Weyl tensor in vacuum) from
finite differences of the closed-form 4-metric, contracted with the null
tetrad of the psi_4 appendix. Independent of the oracle's 3+1 expression of
psi_4 through E_ij and B_ij."""
import numpy as np

# sixth-order central difference weights for the first derivative at offsets -3..3
W1 = np.array([-1.0, 9.0, -45.0, 0.0, 45.0, -9.0, 1.0]) / 60.0
OFF = np.arange(-3, 4)


class BoostedKS:
    """g_ab = eta_ab + 2 (M / R) l_a l_b, with R and l_a = (1, n) evaluated
    in the rest frame of a black hole of mass M at rest at c0 (at t = 0)
    moving with velocity vel (a 3-vector, |vel| < 1) in the lab frame."""

    def __init__(self, M=1.0, c0=(3.0, 0.5, -0.2), vel=(0.0, 0.3, 0.0)):
        self.M = float(M)
        self.c0 = np.asarray(c0, float)
        v = np.asarray(vel, float)
        g = 1.0 / np.sqrt(1.0 - v @ v)
        # Lorentz boost Lam[nu][mu] = d X^nu / d x^mu (rest frame X from lab x)
        L = np.eye(4)
        L[0, 0] = g
        L[0, 1:] = -g * v
        L[1:, 0] = -g * v
        vv = v @ v
        L[1:, 1:] += (g - 1.0) * np.outer(v, v) / vv if vv > 0 else 0.0
        self.L = L

    def metric(self, t, x, y, z):
        """g_ab with shape (..., 4, 4) at arrays of lab coordinates."""
        t, x, y, z = np.broadcast_arrays(*(np.asarray(a, float) for a in (t, x, y, z)))
        xl = np.stack([t, x - self.c0[0], y - self.c0[1], z - self.c0[2]], axis=-1)
        X = xl @ self.L.T                       # rest-frame coordinates
        R = np.sqrt(X[..., 1] ** 2 + X[..., 2] ** 2 + X[..., 3] ** 2)
        lr = np.concatenate([np.ones(R.shape + (1,)), X[..., 1:] / R[..., None]], axis=-1)
        l = lr @ self.L                         # l_mu = l_nu dX^nu/dx^mu
        g = np.zeros(R.shape + (4, 4))
        g[..., 0, 0] = -1.0
        g[..., 1, 1] = g[..., 2, 2] = g[..., 3, 3] = 1.0
        return g + 2.0 * (self.M / R)[..., None, None] * l[..., :, None] * l[..., None, :]


def _d(f, X, a, h):
    """d f / d x^a at points X (..., 4) by the sixth-order central difference."""
    out = 0.0
    for w, o in zip(W1, OFF):
        if w == 0.0:
            continue
        Y = X.copy()
        Y[..., a] += o * h
        out = out + w * f(Y)
    return out / h


def three_plus_one(st, X, h=1e-3):
    """gamma_ij, K_ij, alpha, beta^i at 4-points X (..., 4) (t, x, y, z):
    K_ij = -(d_t gamma_ij - D_i beta_j - D_j beta_i) / (2 alpha)."""
    f = lambda Y: st.metric(Y[..., 0], Y[..., 1], Y[..., 2], Y[..., 3])
    g = f(X)
    dg = np.stack([_d(f, X, a, h) for a in range(4)], axis=-3)   # (..., a, 4, 4)
    gam = g[..., 1:, 1:]
    igam = np.linalg.inv(gam)
    bl = g[..., 0, 1:]
    bu = np.einsum('...ij,...j->...i', igam, bl)
    alpha = np.sqrt(np.einsum('...i,...i->...', bl, bu) - g[..., 0, 0])
    # spatial Christoffel symbols of gamma
    dgam = dg[..., 1:, 1:, 1:]                                     # (..., k, i, j) = d_k gamma_ij
    Gl = 0.5 * (np.swapaxes(dgam, -3, -2) + np.swapaxes(np.swapaxes(dgam, -3, -2), -2, -1) - dgam)
    # Gl[..., i, j, k]? build explicitly: Gamma_kij = 1/2 (d_i g_jk + d_j g_ik - d_k g_ij)
    Gl = 0.5 * (np.einsum('...ijk->...kij', dgam) + np.einsum('...jik->...kij', dgam) - dgam)
    Gam = np.einsum('...kl,...lij->...kij', igam, Gl)
    dbl = dg[..., 1:, 0, 1:]                                        # d_i beta_j
    Db = dbl - np.einsum('...kij,...k->...ij', Gam, bl)
    K = -(dg[..., 0, 1:, 1:] - Db - np.swapaxes(Db, -1, -2)) / (2.0 * alpha[..., None, None])
    return gam, K, alpha, bu


def ccz4_state(st, x, y, z, h=1e-3):
    """The 25 CCZ4 fields (field order of the oracle) of the t = 0 slice at
    points (x, y, z): phi = det(gamma)^(-1/6), g~ = phi^2 gamma,
    A~ = phi^2 (K_ij - gamma_ij K / 3), K = gamma^ij K_ij, Gamma-hat^i =
    G~^i (the contracted Christoffel symbol of g~), Theta = b = 0."""
    shp = np.shape(x)
    X = np.stack(np.broadcast_arrays(np.zeros(shp), x, y, z), axis=-1).reshape(-1, 4)
    gam, K, alpha, bu = three_plus_one(st, X, h)
    igam = np.linalg.inv(gam)
    det = np.linalg.det(gam)
    phi = det ** (-1.0 / 6.0)
    gt = phi[:, None, None] ** 2 * gam
    trK = np.einsum('...ij,...ij->...', igam, K)
    At = phi[:, None, None] ** 2 * (K - gam * trK[:, None, None] / 3.0)

    def gtil(Y):
        gg = st.metric(Y[..., 0], Y[..., 1], Y[..., 2], Y[..., 3])[..., 1:, 1:]
        return np.linalg.det(gg)[..., None, None] ** (-1.0 / 3.0) * gg
    dgt = np.stack([_d(gtil, X, a, h) for a in (1, 2, 3)], axis=-3)  # d_k g~_ij
    igt = np.linalg.inv(gt)
    Gl = 0.5 * (np.einsum('...ijk->...kij', dgt) + np.einsum('...jik->...kij', dgt) - dgt)
    Gam = np.einsum('...kl,...lij->...kij', igt, Gl)
    Gc = np.einsum('...ij,...kij->...k', igt, Gam)
    Q = np.zeros((25, X.shape[0]))
    sym = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    for c, (i, j) in enumerate(sym):
        Q[c] = gt[:, i, j]
        Q[11 + c] = At[:, i, j]
    Q[6] = alpha
    Q[7:10] = bu.T
    Q[10] = phi
    Q[17] = trK
    Q[19:22] = Gc.T
    return Q.reshape((25,) + shp)


def psi4(st, points, centre=(0.0, 0.0, 0.0), h=2e-3):
    """psi_4 = C_abcd k^a mbar^b k^c mbar^d at t = 0 and the given points
    (n, 3), with C the 4D Riemann tensor of the vacuum metric (second
    derivatives of g by nested sixth-order differences), k = (n - u)/sqrt 2,
    mbar = (w - i v)/sqrt 2, n the unit normal of the slice and (v, u, w)
    the Gram-Schmidt triad of the appendix. Also returns the largest
    component of the 4D Ricci tensor (zero in vacuum, up to the
    differencing error)."""
    f = lambda Y: st.metric(Y[..., 0], Y[..., 1], Y[..., 2], Y[..., 3])
    out = np.empty(len(points), complex)
    ric_max = 0.0
    for q, p in enumerate(np.asarray(points, float)):
        X = np.array([0.0, p[0], p[1], p[2]])
        g = f(X)
        ig = np.linalg.inv(g)
        dg = np.stack([_d(f, X[None], a, h)[0] for a in range(4)])          # dg[a] = d_a g
        ddg = np.empty((4, 4, 4, 4))
        for a in range(4):
            for b in range(a, 4):
                dab = _d(lambda Y: _d(f, Y, b, h), X[None], a, h)[0]
                ddg[a, b] = dab
                ddg[b, a] = dab
        # Gamma^a_bc and its derivatives
        Gl = 0.5 * (np.einsum('bca->abc', dg) + np.einsum('cba->abc', dg) - dg)  # Gamma_abc
        # Gl[a,b,c] = 1/2 (d_b g_ac + d_c g_ab - d_a g_bc)
        Gl = np.empty((4, 4, 4))
        for a in range(4):
            for b in range(4):
                for c in range(4):
                    Gl[a, b, c] = 0.5 * (dg[b][a, c] + dg[c][a, b] - dg[a][b, c])
        Gam = np.einsum('ad,dbc->abc', ig, Gl)
        dGl = np.empty((4, 4, 4, 4))  # dGl[e, a, b, c] = d_e Gamma_abc
        for e in range(4):
            for a in range(4):
                for b in range(4):
                    for c in range(4):
                        dGl[e, a, b, c] = 0.5 * (ddg[e, b][a, c] + ddg[e, c][a, b] - ddg[e, a][b, c])
        dig = -np.einsum('ab,ebc,cd->ead', ig, dg, ig)
        dGam = np.einsum('ead,dbc->eabc', dig, Gl) + np.einsum('ad,edbc->eabc', ig, dGl)
        # R^a_bcd = d_c Gamma^a_db - d_d Gamma^a_cb + Gamma^a_ce Gamma^e_db - Gamma^a_de Gamma^e_cb
        Rup = (np.einsum('cadb->abcd', dGam) - np.einsum('dacb->abcd', dGam) +
               np.einsum('ace,edb->abcd', Gam, Gam) - np.einsum('ade,ecb->abcd', Gam, Gam))
        Rd = np.einsum('ae,ebcd->abcd', g, Rup)
        ric = np.einsum('abad->bd', Rup)
        ric_max = max(ric_max, np.abs(ric).max())
        # 3+1 quantities and the tetrad
        gam = g[1:, 1:]
        igam = np.linalg.inv(gam)
        bl = g[0, 1:]
        bu = igam @ bl
        alpha = np.sqrt(bl @ bu - g[0, 0])
        x = p - np.asarray(centre, float)
        sdet = np.sqrt(np.linalg.det(gam))
        dot = lambda a, b: a @ gam @ b
        v = np.array([-x[1], x[0], 0.0])
        v = v / np.sqrt(dot(v, v))
        u = x.copy()
        u = u - dot(v, u) * v
        u = u / np.sqrt(dot(u, u))
        eps = np.zeros((3, 3, 3))
        for i in range(3):
            for j in range(3):
                for k in range(3):
                    eps[i, j, k] = (i - j) * (j - k) * (k - i) / 2.0
        w = igam @ (sdet * np.einsum('jkl,k,l->j', eps, v, u))
        w = w - dot(v, w) * v - dot(u, w) * u
        w = w / np.sqrt(dot(w, w))
        n4 = np.concatenate([[1.0 / alpha], -bu / alpha])
        u4 = np.concatenate([[0.0], u])
        k4 = (n4 - u4) / np.sqrt(2.0)
        mb4 = np.concatenate([[0.0], w - 1j * v]) / np.sqrt(2.0)
        out[q] = np.einsum('abcd,a,b,c,d->', Rd, k4, mb4, k4, mb4)
    return out, ric_max
