"""ctypes binding of the CCZ4 oracle (plain FP64 C restatement of the paper).

TEST INFRASTRUCTURE ONLY. The test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only users of this package. The CUDA
path neither imports nor links it, and the product raises when its own CUDA
library is missing instead of falling back here.

Array layouts (NumPy, float64, C order):
  U      (25, n_patches, p, p, p)     interior points, x fastest
  G      (25, n_ghost)                evolved Sommerfeld ghost cells
  tiles  (25, n_patches, p+6, p+6, p+6)
"""
import ctypes
import os

import numpy as np

from . import build as _build

NV = 25
NV_FO = 58
HALO = 3
BC = {"periodic": 0, "copy": 1, "sommerfeld": 2}
SLICING = {"harmonic": 0, "1+log": 1}
SHIFT = {"zero": 0, "gamma-driver": 1}

_dbl_p = ctypes.POINTER(ctypes.c_double)
_lng_p = ctypes.POINTER(ctypes.c_long)
_int_p = ctypes.POINTER(ctypes.c_int)


class Params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("kappa1", "kappa2", "kappa3", "e", "c", "tau", "mu", "f", "eta", "s", "K0", "ko_eps")] + [
        ("slicing", ctypes.c_int), ("shift", ctypes.c_int), ("somm_speed", ctypes.c_double * NV)]


def make_params(kappa1=1.0, kappa2=0.0, kappa3=0.0, e=1.0, c=1.0, tau=1.0, mu=0.2, f=0.75,
                eta=2.0, s=1.0, K0=0.0, ko_eps=0.1, slicing="harmonic", shift="zero",
                somm_speed=1.0):
    p = Params()
    for k, v in dict(kappa1=kappa1, kappa2=kappa2, kappa3=kappa3, e=e, c=c, tau=tau, mu=mu, f=f,
                     eta=eta, s=s, K0=K0, ko_eps=ko_eps).items():
        setattr(p, k, float(v))
    p.slicing = SLICING[slicing] if isinstance(slicing, str) else int(slicing)
    p.shift = SHIFT[shift] if isinstance(shift, str) else int(shift)
    sp = np.broadcast_to(np.asarray(somm_speed, dtype=np.float64), (NV,))
    for i in range(NV):
        p.somm_speed[i] = float(sp[i])
    return p


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.og_grid_new.restype = ctypes.c_void_p
        L.og_grid_new.argtypes = [ctypes.c_int] * 5 + [_int_p] + [ctypes.c_double] * 4 + [ctypes.c_int]
        L.og_mesh_new.restype = ctypes.c_void_p
        L.og_mesh_new.argtypes = [ctypes.c_int] * 5 + [_int_p, _int_p] + [ctypes.c_double] * 4 + [ctypes.c_int]
        L.og_n_levels.restype = ctypes.c_int
        L.og_n_levels.argtypes = [ctypes.c_void_p]
        L.og_restrict.argtypes = [ctypes.c_void_p, _dbl_p]
        L.og_grid_free.argtypes = [ctypes.c_void_p]
        L.og_n_ghost.restype = ctypes.c_long
        L.og_n_ghost.argtypes = [ctypes.c_void_p]
        L.og_ghost_coords.argtypes = [ctypes.c_void_p, _int_p]
        L.og_fill_tiles.argtypes = [ctypes.c_void_p, _dbl_p, _dbl_p, _dbl_p]
        L.og_rhs.argtypes = [ctypes.c_void_p, ctypes.POINTER(Params), _dbl_p, _dbl_p, _dbl_p, _dbl_p, _dbl_p]
        L.og_ghost_rhs.argtypes = [ctypes.c_void_p, ctypes.POINTER(Params), _dbl_p, _dbl_p, _dbl_p, _dbl_p]
        L.og_rk4_step.argtypes = [ctypes.c_void_p, ctypes.POINTER(Params), ctypes.c_double, _dbl_p, _dbl_p, _dbl_p]
        L.og_enforce.argtypes = [ctypes.c_void_p, _dbl_p]
        L.og_constraints.argtypes = [ctypes.c_void_p, _dbl_p, _dbl_p, _dbl_p, _dbl_p, _dbl_p]
        L.og_psi4.argtypes = [ctypes.c_void_p, _dbl_p, _dbl_p, _dbl_p, _dbl_p]
        L.og_rhs_points.argtypes = [ctypes.c_void_p, ctypes.POINTER(Params), _dbl_p, _dbl_p,
                                    ctypes.c_long, _lng_p, _dbl_p]
        L.og_constraints_points.argtypes = [ctypes.c_void_p, _dbl_p, _dbl_p, ctypes.c_long, _lng_p, _dbl_p]
        L.og_point_derivs.argtypes = [ctypes.c_void_p, _dbl_p, _dbl_p, ctypes.c_long, ctypes.c_double,
                                      _dbl_p, _dbl_p, _dbl_p]
        L.og_fo_rhs.argtypes = [ctypes.c_void_p, ctypes.POINTER(Params), ctypes.c_int, _dbl_p, _dbl_p, _dbl_p,
                                _dbl_p, _dbl_p]
        L.og_fo_reconstruct.argtypes = [ctypes.c_void_p, _dbl_p, _dbl_p]
        L.og_fo_rk4_step.argtypes = [ctypes.c_void_p, ctypes.POINTER(Params), ctypes.c_int, ctypes.c_double,
                                     _dbl_p, _dbl_p, _dbl_p]
        L.og_constraints_excluding.argtypes = [ctypes.c_void_p, _dbl_p, _dbl_p, ctypes.c_int, _dbl_p,
                                               ctypes.c_double, _dbl_p]
        L.og_tracers_step.restype = ctypes.c_long
        L.og_tracers_step.argtypes = [ctypes.c_void_p, _dbl_p, _dbl_p, ctypes.c_long, _dbl_p, ctypes.c_double,
                                      ctypes.c_int, ctypes.c_double, _dbl_p]
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dbl_p)


def _f64(a, shape):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != tuple(shape):
        a = a.reshape(shape)
    return a


class Grid:
    """p^3 patches: one uniform level covering np[0] x np[1] x np[2] patch
    slots, or, with ``level``, a statically refined mesh whose level-0
    patches cover those slots and whose level-l patches (spacing dx / 3^l,
    slots in level-l units) are complete 3x3x3 child sets of level l-1
    patches."""

    def __init__(self, p, np_, ijk, origin, dx, bc="periodic", level=None):
        self.p = int(p)
        self.np = tuple(int(v) for v in np_)
        self.ijk = np.ascontiguousarray(ijk, dtype=np.int32).reshape(-1, 3)
        self.n_patches = self.ijk.shape[0]
        self.origin = tuple(float(v) for v in origin)
        self.dx = float(dx)
        self.bc = BC[bc] if isinstance(bc, str) else int(bc)
        L = lib()
        if level is None:
            self.level = np.zeros(self.n_patches, dtype=np.int32)
            self._h = L.og_grid_new(self.p, *self.np, self.n_patches, self.ijk.ctypes.data_as(_int_p),
                                    *self.origin, self.dx, self.bc)
        else:
            self.level = np.ascontiguousarray(level, dtype=np.int32).reshape(-1)
            if self.level.shape[0] != self.n_patches:
                raise ValueError("oracle: one level per patch")
            self._h = L.og_mesh_new(self.p, *self.np, self.n_patches, self.level.ctypes.data_as(_int_p),
                                    self.ijk.ctypes.data_as(_int_p), *self.origin, self.dx, self.bc)
        if not self._h:
            raise ValueError("oracle: invalid grid description")
        self.n_ghost = int(L.og_n_ghost(self._h))
        self.n_levels = int(L.og_n_levels(self._h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.og_grid_free(h)
            self._h = None

    @property
    def ushape(self):
        return (NV, self.n_patches, self.p, self.p, self.p)

    @property
    def gshape(self):
        return (NV, self.n_ghost)

    def _g(self, G):
        if self.n_ghost == 0:
            return np.zeros((NV, 1))
        return _f64(G, self.gshape)

    def ghost_coords(self):
        out = np.zeros((max(self.n_ghost, 1), 3), dtype=np.int32)
        lib().og_ghost_coords(self._h, out.ctypes.data_as(_int_p))
        return out[:self.n_ghost]

    def fill_tiles(self, U, G=None):
        U = _f64(U, self.ushape)
        G = self._g(G)
        T = self.p + 2 * HALO
        out = np.empty((NV, self.n_patches, T, T, T))
        lib().og_fill_tiles(self._h, _d(U), _d(G), _d(out))
        return out

    def rhs(self, P, U, G=None, Gini=None):
        U = _f64(U, self.ushape)
        G = self._g(G)
        Gini = self._g(Gini)
        rU = np.empty(self.ushape)
        rG = np.empty((NV, max(self.n_ghost, 1)))
        lib().og_rhs(self._h, ctypes.byref(P), _d(U), _d(G), _d(Gini), _d(rU), _d(rG))
        return rU, rG[:, :self.n_ghost]

    def ghost_rhs(self, P, U, G, Gini):
        """Right-hand side of the Sommerfeld ghost shell only, (25, n_ghost)."""
        U = _f64(U, self.ushape)
        G = self._g(G)
        Gini = self._g(Gini)
        rG = np.empty((NV, max(self.n_ghost, 1)))
        lib().og_ghost_rhs(self._h, ctypes.byref(P), _d(U), _d(G), _d(Gini), _d(rG))
        return rG[:, :self.n_ghost]

    def rk4_step(self, P, dt, U, G=None, Gini=None):
        """One RK4 step; returns new (U, G) (inputs are not modified)."""
        U = _f64(U, self.ushape).copy()
        G = self._g(G).copy()
        Gini = self._g(Gini)
        lib().og_rk4_step(self._h, ctypes.byref(P), float(dt), _d(U), _d(G), _d(Gini))
        return U, G[:, :self.n_ghost]

    def restrict(self, U):
        """Coarse points under refined patches <- mean of their 27 fine cells."""
        U = _f64(U, self.ushape).copy()
        lib().og_restrict(self._h, _d(U))
        return U

    def enforce(self, U):
        U = _f64(U, self.ushape).copy()
        lib().og_enforce(self._h, _d(U))
        return U

    def constraints(self, U, G=None):
        U = _f64(U, self.ushape)
        G = self._g(G)
        H = np.empty(self.ushape[1:])
        M = np.empty((3,) + self.ushape[1:])
        out = np.empty(5)
        lib().og_constraints(self._h, _d(U), _d(G), _d(H), _d(M), _d(out))
        return H, M, out

    def psi4(self, U, G=None, centre=(0.0, 0.0, 0.0)):
        """psi_4 at every interior point, (2, n_patches, p, p, p): real and
        imaginary parts, the tetrad centred at `centre`."""
        U = _f64(U, self.ushape)
        G = self._g(G)
        c = np.ascontiguousarray(centre, dtype=np.float64).reshape(3)
        out = np.empty((2,) + self.ushape[1:])
        lib().og_psi4(self._h, _d(U), _d(G), _d(c), _d(out))
        return out

    def constraints_excluding(self, H, M, centres, radius):
        """Norms of H and |M| over leaf points at distance >= radius from
        every centre: (L2 H, L2 |M|, max |H|, max |M|, count)."""
        H = _f64(H, self.ushape[1:])
        M = _f64(M, (3,) + self.ushape[1:])
        c = np.ascontiguousarray(centres, dtype=np.float64).reshape(-1, 3)
        out = np.empty(5)
        lib().og_constraints_excluding(self._h, _d(H), _d(M), len(c), _d(c), float(radius), _d(out))
        return out

    def rhs_points(self, P, U, G, pts):
        U = _f64(U, self.ushape)
        G = self._g(G)
        pts = np.ascontiguousarray(pts, dtype=np.int64)
        out = np.empty((len(pts), NV))
        rc = lib().og_rhs_points(self._h, ctypes.byref(P), _d(U), _d(G), len(pts),
                                 pts.ctypes.data_as(_lng_p), _d(out))
        if rc:
            raise IndexError("oracle: sample point out of range")
        return out

    def constraints_points(self, U, G, pts):
        U = _f64(U, self.ushape)
        G = self._g(G)
        pts = np.ascontiguousarray(pts, dtype=np.int64)
        out = np.empty((len(pts), 4))
        rc = lib().og_constraints_points(self._h, _d(U), _d(G), len(pts), pts.ctypes.data_as(_lng_p), _d(out))
        if rc:
            raise IndexError("oracle: sample point out of range")
        return out

    def point_derivs(self, U, G, pt, ko_eps=0.1):
        U = _f64(U, self.ushape)
        G = self._g(G)
        d1 = np.empty((NV, 3))
        d2 = np.empty((NV, 3, 3))
        ko = np.empty(NV)
        rc = lib().og_point_derivs(self._h, _d(U), _d(G), int(pt), float(ko_eps), _d(d1), _d(d2), _d(ko))
        if rc:
            raise IndexError("oracle: sample point out of range")
        return d1, d2, ko

    # -- first-order formulation (58 fields; fo_* take and return (58, ...) arrays) --
    @property
    def fo_ushape(self):
        return (NV_FO, self.n_patches, self.p, self.p, self.p)

    def _gfo(self, G):
        if self.n_ghost == 0:
            return np.zeros((NV_FO, 1))
        return _f64(G, (NV_FO, self.n_ghost))

    def fo_rhs(self, P, U, G=None, Gini=None, red=True):
        """Right-hand side of the 58 variables: red=True the first-order
        formulation, False the second-order one without the red terms."""
        U = _f64(U, self.fo_ushape)
        G, Gini = self._gfo(G), self._gfo(Gini)
        rU = np.empty(self.fo_ushape)
        rG = np.empty((NV_FO, max(self.n_ghost, 1)))
        lib().og_fo_rhs(self._h, ctypes.byref(P), int(bool(red)), _d(U), _d(G), _d(Gini), _d(rU), _d(rG))
        return rU, rG[:, :self.n_ghost]

    def fo_reconstruct(self, U, G=None):
        """Interior auxiliary variables <- FD4 derivatives of the primaries."""
        U = _f64(U, self.fo_ushape).copy()
        lib().og_fo_reconstruct(self._h, _d(U), _d(self._gfo(G)))
        return U

    def fo_rk4_step(self, P, dt, U, G=None, Gini=None, variant="fo"):
        """One RK4 step of the 58-variable state: variant "fo" (first order)
        or "so-recon" (second order with reconstruction)."""
        U = _f64(U, self.fo_ushape).copy()
        G = self._gfo(G).copy()
        Gini = self._gfo(Gini)
        v = {"fo": 0, "so-recon": 1}[variant]
        lib().og_fo_rk4_step(self._h, ctypes.byref(P), v, float(dt), _d(U), _d(G), _d(Gini))
        return U, G[:, :self.n_ghost]

    def tracers_step(self, U, G, pos, dt=0.0, vel_field=-1, vel_scale=-1.0):
        """One tracer step: returns (new positions (n, 3), projected fields
        (n, 25), number of tracers that could not be projected)."""
        U = _f64(U, self.ushape)
        G = self._g(G)
        pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3).copy()
        vals = np.empty((len(pos), NV))
        bad = lib().og_tracers_step(self._h, _d(U), _d(G), len(pos), _d(pos), float(dt), int(vel_field),
                                    float(vel_scale), _d(vals))
        return pos, vals, int(bad)


# ---------------------------------------------------------------------------
# Bowen-York puncture initial data (bowen_york.h)
# ---------------------------------------------------------------------------
MAX_PUNCTURES = 4


class Punctures(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("m", ctypes.c_double * MAX_PUNCTURES),
                ("c", (ctypes.c_double * 3) * MAX_PUNCTURES), ("P", (ctypes.c_double * 3) * MAX_PUNCTURES),
                ("S", (ctypes.c_double * 3) * MAX_PUNCTURES)]


def make_punctures(masses, centres, momenta=None, spins=None):
    B = Punctures()
    B.n = len(masses)
    if not 1 <= B.n <= MAX_PUNCTURES:
        raise ValueError("1..%d punctures" % MAX_PUNCTURES)
    for k in range(B.n):
        B.m[k] = float(masses[k])
        for d in range(3):
            B.c[k][d] = float(centres[k][d])
            B.P[k][d] = float(momenta[k][d]) if momenta is not None else 0.0
            B.S[k][d] = float(spins[k][d]) if spins is not None else 0.0
    return B


def _by_lib():
    L = lib()
    if not getattr(L, "_by_ready", False):
        bp = ctypes.POINTER(Punctures)
        L.og_by_points.argtypes = [bp, ctypes.c_long, _dbl_p, _dbl_p, _dbl_p, _dbl_p, _dbl_p, _dbl_p]
        L.og_by_residual.restype = ctypes.c_double
        L.og_by_residual.argtypes = [bp, ctypes.c_int, ctypes.c_double, _dbl_p, _dbl_p]
        L.og_by_sweeps.argtypes = [bp, ctypes.c_int, ctypes.c_double, _dbl_p, ctypes.c_int, ctypes.c_double]
        L.og_by_solve.restype = ctypes.c_int
        L.og_by_solve.argtypes = [bp, ctypes.c_int, ctypes.c_double, _dbl_p, ctypes.c_double, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_double, _dbl_p]
        L.og_by_interp.argtypes = [ctypes.c_int, ctypes.c_double, _dbl_p, ctypes.c_long, _dbl_p, _dbl_p, _dbl_p,
                                   _dbl_p]
        L.og_by_state.argtypes = [bp, ctypes.c_int, ctypes.c_double, _dbl_p, ctypes.c_long, _dbl_p, _dbl_p, _dbl_p,
                                  _dbl_p]
        L.og_by_box_ghosts.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_double, _dbl_p, _dbl_p]
        L.og_by_cells_from.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_double, _dbl_p, _dbl_p]
        L.og_by_residual_box.restype = ctypes.c_double
        L.og_by_residual_box.argtypes = [bp, ctypes.c_int, ctypes.c_double, _dbl_p, _dbl_p, _dbl_p]
        L.og_by_sweeps_box.argtypes = [bp, ctypes.c_int, ctypes.c_double, _dbl_p, _dbl_p, ctypes.c_int,
                                       ctypes.c_double]
        L.og_by_solve_box.restype = ctypes.c_int
        L.og_by_solve_box.argtypes = [bp, ctypes.c_int, ctypes.c_double, _dbl_p, _dbl_p, ctypes.c_double,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_double, _dbl_p]
        L._by_ready = True
    return L


def by_points(B, x, y, z):
    """(Abar[m, 6], Abar.Abar[m], psi_BL[m]) at the points."""
    x, y, z = (np.ascontiguousarray(v, dtype=np.float64).ravel() for v in (x, y, z))
    m = len(x)
    A = np.empty((m, 6))
    aa = np.empty(m)
    psi = np.empty(m)
    _by_lib().og_by_points(ctypes.byref(B), m, _d(x), _d(y), _d(z), _d(A), _d(aa), _d(psi))
    return A, aa, psi


def by_cell_coords(n, L):
    """Cell centres of the initial-data grid, each (n, n, n) as [z][y][x]."""
    c = -L + (np.arange(n) + 0.5) * (2.0 * L / n)
    return (np.broadcast_to(c[None, None, :], (n, n, n)), np.broadcast_to(c[None, :, None], (n, n, n)),
            np.broadcast_to(c[:, None, None], (n, n, n)))


def by_residual(B, n, L, u):
    u = _f64(u, (n, n, n))
    res = np.empty((n, n, n))
    mx = _by_lib().og_by_residual(ctypes.byref(B), int(n), float(L), _d(u), _d(res))
    return res, mx


def by_sweeps(B, n, L, u, n_sweeps, omega=1.0):
    u = _f64(u, (n, n, n)).copy()
    _by_lib().og_by_sweeps(ctypes.byref(B), int(n), float(L), _d(u), int(n_sweeps), float(omega))
    return u


def by_solve(B, n, L, u0=None, tol=1e-10, max_sweeps=1000000, check=10, omega=1.0):
    """Solves from u0 (default 0); returns (u, sweeps or -1, final residual)."""
    u = np.zeros((n, n, n)) if u0 is None else _f64(u0, (n, n, n)).copy()
    r = ctypes.c_double()
    k = _by_lib().og_by_solve(ctypes.byref(B), int(n), float(L), _d(u), float(tol), int(max_sweeps), int(check),
                              float(omega), ctypes.byref(r))
    return u, k, r.value


def by_box_ghosts(n, L, np_, Lp, up):
    """Fixed ghost values (6, n, n) of a box of n^3 cells on [-L, L]^3 from
    the parent solution up (np_^3 cells of [-Lp, Lp]^3): face 2d / 2d+1 of
    axis d, then the two other cell indices (the lower axis fastest)."""
    up = _f64(up, (np_, np_, np_))
    gb = np.empty((6, n, n))
    _by_lib().og_by_box_ghosts(int(n), float(L), int(np_), float(Lp), _d(up), _d(gb))
    return gb


def by_cells_from(n, L, np_, Lp, up):
    """The parent solution interpolated at the box's cell centres (n, n, n)."""
    up = _f64(up, (np_, np_, np_))
    u = np.empty((n, n, n))
    _by_lib().og_by_cells_from(int(n), float(L), int(np_), float(Lp), _d(up), _d(u))
    return u


def by_residual_box(B, n, L, u, gb):
    u = _f64(u, (n, n, n))
    gb = None if gb is None else _f64(gb, (6, n, n))
    res = np.empty((n, n, n))
    mx = _by_lib().og_by_residual_box(ctypes.byref(B), int(n), float(L), _d(u), _d(gb) if gb is not None else None,
                                      _d(res))
    return res, mx


def by_sweeps_box(B, n, L, u, gb, n_sweeps, omega=1.0):
    u = _f64(u, (n, n, n)).copy()
    gb = _f64(gb, (6, n, n))
    _by_lib().og_by_sweeps_box(ctypes.byref(B), int(n), float(L), _d(u), _d(gb), int(n_sweeps), float(omega))
    return u


def by_solve_box(B, n, L, gb, u0=None, tol=1e-10, max_sweeps=1000000, check=10, omega=1.0):
    """Solves a box with fixed ghosts gb from u0 (default 0); returns (u,
    sweeps or -1, final residual)."""
    u = np.zeros((n, n, n)) if u0 is None else _f64(u0, (n, n, n)).copy()
    gb = _f64(gb, (6, n, n))
    r = ctypes.c_double()
    k = _by_lib().og_by_solve_box(ctypes.byref(B), int(n), float(L), _d(u), _d(gb), float(tol), int(max_sweeps),
                                  int(check), float(omega), ctypes.byref(r))
    return u, k, r.value


def by_interp(n, L, u, x, y, z):
    """Tricubic interpolation of the solver grid u at the points."""
    u = _f64(u, (n, n, n))
    x, y, z = (np.ascontiguousarray(v, dtype=np.float64).ravel() for v in (x, y, z))
    out = np.empty(len(x))
    _by_lib().og_by_interp(int(n), float(L), _d(u), len(x), _d(x), _d(y), _d(z), _d(out))
    return out


def by_state(B, n, L, u, x, y, z):
    """The 25 CCZ4 fields (25, m) of the solved data at the points."""
    u = _f64(u, (n, n, n))
    x, y, z = (np.ascontiguousarray(v, dtype=np.float64).ravel() for v in (x, y, z))
    Q = np.empty((NV, len(x)))
    _by_lib().og_by_state(ctypes.byref(B), int(n), float(L), _d(u), len(x), _d(x), _d(y), _d(z), _d(Q))
    return Q
