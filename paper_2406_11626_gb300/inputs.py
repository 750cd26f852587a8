"""Seeded synthetic inputs for the CCZ4 hot path: grids, initial data, configs.

This module holds no step of the method itself (no halo fill, stencil,
right-hand side, time step or constraint): it only produces the arrays that
the CUDA path and the CPU oracle both take as input. Everything is NumPy,
FP64, and deterministic given its arguments.

Conventions shared by every caller:
  - fields in the order of ``FIELDS`` (the 25 primary variables of the
    second-order formulation);
  - interior state as an array of shape (25, n_patches, p, p, p), x fastest;
  - cell-centred sample points x = origin + (i + 1/2) dx (the paper samples
    the patch volumes at their centres);
  - patches listed by integer coordinates ``ijk`` (n_patches, 3) in any order;
  - Sommerfeld ghost cells: every cell within 3 points of the domain and
    outside it, in lexicographic (z, y, x) order of the global coordinates.
"""
from dataclasses import dataclass, field

import numpy as np

FIELDS = ("gxx", "gxy", "gxz", "gyy", "gyz", "gzz", "alpha", "betax", "betay", "betaz", "phi",
          "Axx", "Axy", "Axz", "Ayy", "Ayz", "Azz", "K", "Theta", "Ghatx", "Ghaty", "Ghatz",
          "bx", "by", "bz")
NV = len(FIELDS)
HALO = 3
IDX = {n: i for i, n in enumerate(FIELDS)}
# diagonal conformal-metric components (flat space has 1 there, 0 elsewhere)
_FLAT_ONES = (IDX["gxx"], IDX["gyy"], IDX["gzz"], IDX["alpha"], IDX["phi"])


def patch_ijk(np_, permute_seed=None):
    """Integer coordinates of every patch slot of an np[0] x np[1] x np[2] block,
    lexicographic (z slowest), optionally shuffled by a seeded permutation."""
    a, b, c = (int(v) for v in np_)
    zz, yy, xx = np.meshgrid(np.arange(c), np.arange(b), np.arange(a), indexing="ij")
    ijk = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1).astype(np.int32)
    if permute_seed is not None:
        ijk = ijk[np.random.default_rng(permute_seed).permutation(len(ijk))]
    return np.ascontiguousarray(ijk)


def point_coords(p, ijk, origin, dx):
    """Coordinates (x, y, z) of all interior points, each (n_patches, p, p, p)."""
    ijk = np.asarray(ijk).reshape(-1, 3)
    l = np.arange(p)
    out = []
    for d in range(3):
        shape = [1, 1, 1]
        shape[2 - d] = p
        loc = l.reshape(shape)
        g = ijk[:, d].reshape(-1, 1, 1, 1) * p + loc
        out.append(origin[d] + (g + 0.5) * dx)
    return tuple(np.broadcast_to(o, (len(ijk), p, p, p)).copy() for o in out)


def level_spacing(dx, n_levels):
    """Grid spacing of each level of a ratio-3 mesh: divided by 3.0 once per level."""
    out = [float(dx)]
    for _ in range(1, n_levels):
        out.append(out[-1] / 3.0)
    return out


def refined_mesh(np_, boxes, permute_seed=None):
    """A statically refined mesh: level 0 covers the np_ slots; boxes[l-1] =
    ((lo_x, lo_y, lo_z), (hi_x, hi_y, hi_z)) lists, in slot units of level
    l-1 with hi exclusive, the level l-1 patches that get their 27 children
    on level l. Returns (level, ijk) with the levels in order."""
    level = []
    ijk = []
    base = patch_ijk(np_, permute_seed)
    level += [0] * len(base)
    ijk += [tuple(r) for r in base]
    parents = set(map(tuple, base))
    for l, (lo, hi) in enumerate(boxes, start=1):
        kids = []
        for (a, b, c) in sorted(parents, key=lambda t: (t[2], t[1], t[0])):
            if all(lo[d] <= (a, b, c)[d] < hi[d] for d in range(3)):
                for k in range(3):
                    for j in range(3):
                        for i in range(3):
                            kids.append((3 * a + i, 3 * b + j, 3 * c + k))
        kids.sort(key=lambda t: (t[2], t[1], t[0]))
        level += [l] * len(kids)
        ijk += kids
        parents = set(kids)
    return np.asarray(level, dtype=np.int32), np.asarray(ijk, dtype=np.int32).reshape(-1, 3)


def mesh_point_coords(p, level, ijk, origin, dx):
    """Coordinates of all interior points of a refined mesh, each
    (n_patches, p, p, p); patch n uses the spacing of its level."""
    level = np.asarray(level)
    ijk = np.asarray(ijk).reshape(-1, 3)
    hs = level_spacing(dx, int(level.max()) + 1)
    out = [np.empty((len(ijk), p, p, p)) for _ in range(3)]
    for l, h in enumerate(hs):
        sel = np.nonzero(level == l)[0]
        if len(sel) == 0:
            continue
        xyz = point_coords(p, ijk[sel], origin, h)
        for d in range(3):
            out[d][sel] = xyz[d]
    return tuple(out)


def ghost_cells(N):
    """Global integer coordinates (n_ghost, 3) of the ghost shell of an
    N[0] x N[1] x N[2] point domain, in lexicographic (z, y, x) order."""
    zs, ys, xs = (np.arange(-HALO, n + HALO) for n in (N[2], N[1], N[0]))
    zz, yy, xx = np.meshgrid(zs, ys, xs, indexing="ij")
    out = ((xx < 0) | (xx >= N[0]) | (yy < 0) | (yy >= N[1]) | (zz < 0) | (zz >= N[2]))
    return np.stack([xx[out], yy[out], zz[out]], axis=1).astype(np.int32)


def ghost_positions(N, origin, dx):
    c = ghost_cells(N)
    return tuple(origin[d] + (c[:, d] + 0.5) * dx for d in range(3))


def flat(shape):
    """Minkowski space in Cartesian coordinates: g~ = delta, alpha = phi = 1."""
    Q = np.zeros((NV,) + tuple(shape))
    for i in _FLAT_ONES:
        Q[i] = 1.0
    return Q


def gauge_wave(x, t=0.0, A=0.1, k=2.0):
    """Gauge-wave spacetime, Sec. "Gauge Wave" of the paper: H = 1 - A sin(k pi (x - t)),
    alpha = sqrt(H), beta = 0, phi = H^(-1/6), K_xx = -(k pi A / 2) cos / sqrt(H),
    K = K_xx / H. The conformal quantities follow from those printed values:
    g~_xx = H^(2/3), g~_yy = g~_zz = H^(-1/3), A~ = phi^2 (K_ij - K gamma_ij / 3),
    Gamma-hat^x = G~^x = -d_x g~^xx = -d_x H^(-2/3), Theta = b = 0."""
    x = np.asarray(x, dtype=np.float64)
    s = np.sin(k * np.pi * (x - t))
    c = np.cos(k * np.pi * (x - t))
    H = 1.0 - A * s
    Q = np.zeros((NV,) + x.shape)
    Q[IDX["gxx"]] = H ** (2.0 / 3.0)
    Q[IDX["gyy"]] = H ** (-1.0 / 3.0)
    Q[IDX["gzz"]] = H ** (-1.0 / 3.0)
    Q[IDX["alpha"]] = np.sqrt(H)
    Q[IDX["phi"]] = H ** (-1.0 / 6.0)
    Kxx = -(k * np.pi * A / 2.0) * c / np.sqrt(H)
    Q[IDX["K"]] = Kxx / H
    Q[IDX["Axx"]] = H ** (-1.0 / 3.0) * (2.0 / 3.0) * Kxx
    Q[IDX["Ayy"]] = H ** (-1.0 / 3.0) * (-1.0 / 3.0) * Kxx / H
    Q[IDX["Azz"]] = Q[IDX["Ayy"]]
    dH = -A * k * np.pi * c
    Q[IDX["Ghatx"]] = (2.0 / 3.0) * H ** (-5.0 / 3.0) * dH
    return Q


def gauge_wave_dt(x, t=0.0, A=0.1, k=2.0):
    """Exact time derivative of every field of ``gauge_wave`` (the wave
    depends on x - t only, so d_t = -d_x, taken here in closed form)."""
    x = np.asarray(x, dtype=np.float64)
    s = np.sin(k * np.pi * (x - t))
    c = np.cos(k * np.pi * (x - t))
    w = k * np.pi
    H = 1.0 - A * s
    Ht = A * w * c            # d_t H
    ct = w * s                # d_t cos(w (x - t))
    D = np.zeros((NV,) + x.shape)
    D[IDX["gxx"]] = (2.0 / 3.0) * H ** (-1.0 / 3.0) * Ht
    D[IDX["gyy"]] = (-1.0 / 3.0) * H ** (-4.0 / 3.0) * Ht
    D[IDX["gzz"]] = D[IDX["gyy"]]
    D[IDX["alpha"]] = 0.5 * H ** (-0.5) * Ht
    D[IDX["phi"]] = (-1.0 / 6.0) * H ** (-7.0 / 6.0) * Ht
    a = -(w * A / 2.0)
    Kxx = a * c * H ** (-0.5)
    Kxx_t = a * (ct * H ** (-0.5) - 0.5 * c * H ** (-1.5) * Ht)
    D[IDX["K"]] = Kxx_t / H - Kxx * Ht / H ** 2
    D[IDX["Axx"]] = (2.0 / 3.0) * ((-1.0 / 3.0) * H ** (-4.0 / 3.0) * Ht * Kxx + H ** (-1.0 / 3.0) * Kxx_t)
    D[IDX["Ayy"]] = (-1.0 / 3.0) * ((-4.0 / 3.0) * H ** (-7.0 / 3.0) * Ht * Kxx + H ** (-4.0 / 3.0) * Kxx_t)
    D[IDX["Azz"]] = D[IDX["Ayy"]]
    dH = -A * w * c
    dH_t = -A * w * ct
    D[IDX["Ghatx"]] = (2.0 / 3.0) * ((-5.0 / 3.0) * H ** (-8.0 / 3.0) * Ht * dH + H ** (-5.0 / 3.0) * dH_t)
    return D


def brill_lindquist(x, y, z, masses=(1.0,), centres=((0.0, 0.0, 0.0),)):
    """Puncture data with K_ij = 0, conformal flatness and zero shift
    (Sec. "Single Schwarzschild Black Hole"): phi = psi^(-2) with
    psi = 1 + sum_n m_n / (2 r_n), and the averaged lapse
    alpha = ((1 - sum m_n / 2 r_n) / (1 + sum m_n / 2 r_n) + 1) / 2 of the
    single- and binary-black-hole sections."""
    x, y, z = (np.asarray(v, dtype=np.float64) for v in (x, y, z))
    s = np.zeros_like(x)
    for m, c in zip(masses, centres):
        r = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2)
        s = s + m / (2.0 * r)
    Q = flat(x.shape)
    Q[IDX["phi"]] = (1.0 + s) ** (-2.0)
    Q[IDX["alpha"]] = 0.5 * ((1.0 - s) / (1.0 + s) + 1.0)
    return Q


# ---- the 58 variables of the first-order formulation ---------------------------
# The 25 primaries, then A_k = d_k alpha (25..27), B_k^i = d_k beta^i
# (28 + 3k + i), D_kij = 1/2 d_k g~_ij (37 + 6k + pair) and P_k = d_k phi
# (55..57) (Eq. auxiliary-variables of the paper).
NV_FO = 58
FO_A, FO_B, FO_D, FO_P = 25, 28, 37, 55
FO_FIELDS = FIELDS + tuple("A" + "xyz"[k] for k in range(3)) + tuple(
    "B" + "xyz"[k] + "xyz"[i] for k in range(3) for i in range(3)) + tuple(
    "D" + "xyz"[k] + p for k in range(3) for p in ("xx", "xy", "xz", "yy", "yz", "zz")) + tuple(
    "P" + "xyz"[k] for k in range(3))


def fo_state(Q, dQ):
    """58 variables from the 25 primaries Q (25, ...) and their spatial
    derivatives dQ (3, 25, ...), dQ[k, v] = d_k Q_v."""
    out = np.zeros((NV_FO,) + Q.shape[1:])
    out[:NV] = Q
    for k in range(3):
        out[FO_A + k] = dQ[k, IDX["alpha"]]
        out[FO_P + k] = dQ[k, IDX["phi"]]
        for i in range(3):
            out[FO_B + 3 * k + i] = dQ[k, IDX["betax"] + i]
        for c in range(6):
            out[FO_D + 6 * k + c] = 0.5 * dQ[k, IDX["gxx"] + c]
    return out


def fo_gauge_wave(x, t=0.0, A=0.1, k=2.0):
    """The gauge wave's 58 variables: every field is a function of x - t,
    so d_x = -d_t, taken from the closed-form gauge_wave_dt."""
    Q = gauge_wave(x, t, A, k)
    dQ = np.zeros((3,) + Q.shape)
    dQ[0] = -gauge_wave_dt(x, t, A, k)
    return fo_state(Q, dQ)


def fo_brill_lindquist(x, y, z, masses=(1.0,), centres=((0.0, 0.0, 0.0),)):
    """Brill-Lindquist data with its auxiliary variables in closed form:
    psi = 1 + s, s = sum m/(2 r), phi = psi^-2, the averaged lapse
    ((1 - s)/(1 + s) + 1)/2 = 1/psi, so P_k = -2 psi^-3 d_k s and
    A_k = -psi^-2 d_k s with d_k s = -sum m (x_k - c_k)/(2 r^3); B = D = 0."""
    x, y, z = (np.asarray(v, dtype=np.float64) for v in (x, y, z))
    Q = brill_lindquist(x, y, z, masses, centres)
    s = np.zeros_like(x)
    ds = np.zeros((3,) + x.shape)
    for m, c in zip(masses, centres):
        d = (x - c[0], y - c[1], z - c[2])
        r = np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
        s = s + m / (2.0 * r)
        for k in range(3):
            ds[k] = ds[k] - m * d[k] / (2.0 * r ** 3)
    psi = 1.0 + s
    dQ = np.zeros((3,) + Q.shape)
    for k in range(3):
        dQ[k, IDX["phi"]] = -2.0 * psi ** -3 * ds[k]
        dQ[k, IDX["alpha"]] = -(psi ** -2) * ds[k]
    return fo_state(Q, dQ)


def fo_initial_state(cfg):
    """(U, G) of the 58 variables at t = 0 for the gauge-wave and
    single-puncture configurations (single level)."""
    x, y, z = point_coords(cfg.p, cfg.ijk(), cfg.origin, cfg.dx)
    if cfg.name == "gauge_wave":
        U = fo_gauge_wave(x, 0.0, cfg.extra["A"], cfg.extra["k"])
        G = np.zeros((NV_FO, 0))
        if cfg.bc == "sommerfeld":
            gx, _, _ = ghost_positions(cfg.N, cfg.origin, cfg.dx)
            G = fo_gauge_wave(gx, 0.0, cfg.extra["A"], cfg.extra["k"])
    elif cfg.name == "single_puncture":
        U = fo_brill_lindquist(x, y, z, (cfg.extra["M"],))
        G = np.zeros((NV_FO, 0))
        if cfg.bc == "sommerfeld":
            G = fo_brill_lindquist(*ghost_positions(cfg.N, cfg.origin, cfg.dx), (cfg.extra["M"],))
    else:
        raise ValueError(cfg.name)
    return np.ascontiguousarray(U), np.ascontiguousarray(G)


def smooth_perturbation(x, y, z, seed, amp=1e-2, box=1.0, modes=3, base=None):
    """Flat space (or ``base``) plus, in every one of the 25 fields, a sum of
    ``modes`` seeded Fourier modes exp-periodic on a cube of side ``box``
    (integer wave vectors in -2..2), each of amplitude up to ``amp``."""
    rng = np.random.default_rng(seed)
    x, y, z = (np.asarray(v, dtype=np.float64) for v in (x, y, z))
    Q = flat(x.shape) if base is None else np.array(base, dtype=np.float64, copy=True)
    for v in range(NV):
        for _ in range(modes):
            kv = rng.integers(-2, 3, size=3)
            if not kv.any():
                kv[0] = 1
            ph = rng.uniform(0.0, 2.0 * np.pi)
            a = rng.uniform(-amp, amp)
            Q[v] += a * np.sin(2.0 * np.pi * (kv[0] * x + kv[1] * y + kv[2] * z) / box + ph)
    return Q


def random_noise(shape, seed, amp=1e-3):
    """Flat space plus independent uniform noise in every value (non-smooth:
    exercises every stencil weight and every algebraic term)."""
    rng = np.random.default_rng(seed)
    return flat(shape) + rng.uniform(-amp, amp, size=(NV,) + tuple(shape))


@dataclass
class Config:
    """A workload: one uniform level of p^3 patches, its physics and time step."""
    name: str
    p: int
    np: tuple
    origin: tuple
    dx: float
    bc: str
    params: dict
    dt: float
    steps: int
    permute_seed: object = None
    extra: dict = field(default_factory=dict)

    @property
    def N(self):
        return tuple(n * self.p for n in self.np)

    @property
    def n_patches(self):
        return int(np.prod(self.np))

    @property
    def n_points(self):
        return self.n_patches * self.p ** 3

    def ijk(self):
        return patch_ijk(self.np, self.permute_seed)


GAUGE_WAVE_PARAMS = dict(kappa1=1.0, kappa2=0.0, kappa3=0.0, e=1.0, c=1.0, tau=1.0, mu=0.2,
                         f=0.75, eta=2.0, s=1.0, K0=0.0, ko_eps=0.1, slicing="harmonic", shift="zero")
PUNCTURE_PARAMS = dict(kappa1=0.1, kappa2=0.0, kappa3=0.5, e=1.0, c=1.0, tau=1.0, mu=0.2,
                       f=0.75, eta=2.0, s=1.0, K0=0.0, ko_eps=0.1, slicing="1+log",
                       shift="gamma-driver")


def gauge_wave_config(p=9, np_=(3, 3, 3), steps=10, cfl=0.1, permute_seed=None):
    """Periodic [-0.5, 0.5]^3 gauge wave, A = 0.1, wavelength 1 along x,
    harmonic slicing, zero shift, classic RK4 with dt = cfl * dx."""
    N = np_[0] * p
    dx = 1.0 / N
    return Config("gauge_wave", p, tuple(np_), (-0.5, -0.5, -0.5), dx, "periodic",
                  dict(GAUGE_WAVE_PARAMS), cfl * dx, steps, permute_seed, dict(A=0.1, k=2.0))


def single_puncture_config(p=9, n_side=16, half_width=8.0, steps=200, cfl=0.1, permute_seed=None):
    """M = 1 Brill-Lindquist puncture at the origin, [-8, 8]^3 as 16^3 patches
    of 9^3 points (144^3 points, dx = 1/9), 1+log slicing, Gamma-driver shift
    with eta = 2, Kreiss-Oliger 0.1, Sommerfeld outer boundary, RK4."""
    N = n_side * p
    dx = 2.0 * half_width / N
    return Config("single_puncture", p, (n_side,) * 3, (-half_width,) * 3, dx, "sommerfeld",
                  dict(PUNCTURE_PARAMS), cfl * dx, steps, permute_seed, dict(M=1.0))


@dataclass
class MeshConfig(Config):
    """A workload on a statically refined mesh: Config's level-0 grid plus
    the level and slot (in units of its level) of every patch."""
    level: np.ndarray = None
    mesh_ijk: np.ndarray = None

    @property
    def n_patches(self):
        return len(self.level)

    @property
    def n_levels(self):
        return int(self.level.max()) + 1

    def ijk(self):
        return self.mesh_ijk


def multilevel_puncture_config(p=9, n_side=16, half_width=8.0, boxes=None, steps=20, cfl=0.1):
    """The single-puncture physics on ratio-3 static levels around the
    puncture. Default: [-8, 8]^3 as 16^3 level-0 patches of 9^3 (dx = 1/9),
    the central 4^3 of them refined into 12^3 level-1 patches, whose central
    4^3 are refined into 12^3 level-2 patches (dx = 1/81): 7552 patches,
    5.5M points. One global dt = cfl * (finest dx)."""
    if boxes is None:
        c0 = n_side // 2
        c1 = 3 * c0
        boxes = [((c0 - 2,) * 3, (c0 + 2,) * 3), ((c1 - 2,) * 3, (c1 + 2,) * 3)]
    level, ijk = refined_mesh((n_side,) * 3, boxes)
    N = n_side * p
    dx = 2.0 * half_width / N
    h = level_spacing(dx, int(level.max()) + 1)
    return MeshConfig("single_puncture", p, (n_side,) * 3, (-half_width,) * 3, dx, "sommerfeld",
                      dict(PUNCTURE_PARAMS), cfl * h[-1], steps, None, dict(M=1.0), level, ijk)


BINARY_PARAMS = dict(PUNCTURE_PARAMS, eta=1.0)


BINARY_ID_BOXES = ((208, 13.0), (192, 6.0), (512, 4.0))


def binary_puncture_config(p=9, steps=500, cfl=0.1, id_n=192, id_tol=1e-10, id_omega=1.98,
                           id_boxes=BINARY_ID_BOXES):
    """Two punctures of bare mass 0.487 at x = -3 and +3 with momenta
    (0, -0.0934, 0) and (0, +0.0934, 0), no spin (Bowen-York data, u from the
    plain relaxation solve on id_n^3 cells of [-32, 32]^3 to a max residual
    of id_tol, over-relaxed by id_omega, then on the nested boxes id_boxes,
    (n, L) pairs outermost first, each with fixed ghosts from the box around
    it and solved to id_tol: by default h = 1/8 on [-13, 13]^3 (level 1),
    1/16 on [-6, 6]^3 (level 2) and 1/64 on [-4, 4]^3 (about the finest
    level's spacing, 4/243); () keeps the single solve);
    [-32, 32]^3 with four ratio-3 levels of 9^3 patches: 16^3
    level-0 patches (dx = 4/9), [-12, 12]^3 refined (5832 patches),
    [-5.33, 5.33] x [-2.67, 2.67]^2 refined (3456), [-3.56, 3.56] x
    [-0.89, 0.89]^2 refined (6912): 20296 patches, 14.8M points. 1+log,
    Gamma-driver f = 0.75, eta = 1 (the paper's binary setup), KO 0.1,
    Sommerfeld, RK4 with dt = cfl * finest dx."""
    boxes = [((5, 5, 5), (11, 11, 11)), ((20, 22, 22), (28, 26, 26)), ((64, 70, 70), (80, 74, 74))]
    level, ijk = refined_mesh((16, 16, 16), boxes)
    dx = 64.0 / (16 * p)
    h = level_spacing(dx, 4)
    return MeshConfig("binary_puncture", p, (16, 16, 16), (-32.0, -32.0, -32.0), dx, "sommerfeld",
                      dict(BINARY_PARAMS), cfl * h[-1], steps, None,
                      dict(m1=0.487, m2=0.487, d=6.0, P=0.0934, S=0.0, id_n=id_n, id_L=32.0, id_tol=id_tol,
                           id_omega=id_omega, id_boxes=tuple(id_boxes)),
                      level, ijk)


def initial_state(cfg):
    """(U, G) at t = 0 for a config; G (the Sommerfeld ghost shell) is empty
    for other boundary kinds. For Sommerfeld, G also serves as Q_ini."""
    ijk = cfg.ijk()
    if isinstance(cfg, MeshConfig):
        x, y, z = mesh_point_coords(cfg.p, cfg.level, ijk, cfg.origin, cfg.dx)
    else:
        x, y, z = point_coords(cfg.p, ijk, cfg.origin, cfg.dx)
    gx = gy = gz = None
    if cfg.bc == "sommerfeld":
        gx, gy, gz = ghost_positions(cfg.N, cfg.origin, cfg.dx)
    if cfg.name == "gauge_wave":
        U = gauge_wave(x, 0.0, cfg.extra["A"], cfg.extra["k"])
        G = np.zeros((NV, 0)) if gx is None else gauge_wave(gx, 0.0, cfg.extra["A"], cfg.extra["k"])
    elif cfg.name == "binary_puncture":
        raise ValueError("the binary puncture's data come from the initial-data solve "
                         "(initial_data.solve_config and Solver.assemble)")
    elif cfg.name == "single_puncture":
        U = brill_lindquist(x, y, z, (cfg.extra["M"],))
        G = np.zeros((NV, 0)) if gx is None else brill_lindquist(gx, gy, gz, (cfg.extra["M"],))
    else:
        raise ValueError(cfg.name)
    return np.ascontiguousarray(U), np.ascontiguousarray(G)
