"""Python binding of the CCZ4 C ABI (include/ccz4.h): argument marshalling only.

Every step of the hot path runs in the CUDA kernels of lib/libccz4_gb300.so.
If that library is missing, every call raises: there is no CPU fallback.
PyTorch is used only to pick up the current CUDA stream and, optionally, to
view device buffers as tensors.
"""
import ctypes
import os

import numpy as np

from .inputs import NV

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libccz4_gb300.so")

OK, ERR_INVALID, ERR_NOMEM, ERR_CUDA, ERR_NONFINITE, ERR_TIMEOUT, ERR_BOUNDS = range(7)
BC = {"periodic": 0, "copy": 1, "sommerfeld": 2}
SLICING = {"harmonic": 0, "1+log": 1}
SHIFT = {"zero": 0, "gamma-driver": 1}
PRECISION = {"fp64": 0, "mixed": 1}
BUF = {"U": 0, "Y0": 1, "Y1": 2, "ACC": 3, "RHS": 4, "INI": 5, "TILE": 6, "MIX": 7}
# mixed second derivatives d_x d_y, d_x d_z, d_y d_z of g~ (slots 0..17),
# alpha (18..20), beta (21..29) and phi (30..32), written by the halo fill
NMIX = 33

_dbl_p = ctypes.POINTER(ctypes.c_double)


class GridDesc(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("np", ctypes.c_int * 3), ("n_patches", ctypes.c_int),
                ("ijk", ctypes.POINTER(ctypes.c_int)), ("origin", ctypes.c_double * 3),
                ("dx", ctypes.c_double), ("bc", ctypes.c_int)]


class MeshDesc(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("np", ctypes.c_int * 3), ("n_patches", ctypes.c_int),
                ("level", ctypes.POINTER(ctypes.c_int)), ("ijk", ctypes.POINTER(ctypes.c_int)),
                ("origin", ctypes.c_double * 3), ("dx", ctypes.c_double), ("bc", ctypes.c_int)]


class Params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("kappa1", "kappa2", "kappa3", "e", "c", "tau", "mu", "f", "eta", "s", "K0", "ko_eps")] + [
        ("slicing", ctypes.c_int), ("shift", ctypes.c_int), ("somm_speed", ctypes.c_double * NV),
        ("precision", ctypes.c_int)]


class CCZ4Error(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("ccz4 error %d: %s" % (code, msg))
        self.code = code


_lib = None


def lib():
    """Loads the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("CCZ4 CUDA library not found at %s; run __graft_entry__.build() "
                          "(paper_2406_11626_gb300.build.build()) first" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp, ll_p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong)
    sig = {
        "ccz4_alloc_patches": [ctypes.POINTER(GridDesc), ctypes.POINTER(vp)],
        "ccz4_free_patches": [vp],
        "ccz4_grid_info": [vp, ll_p, ll_p, ll_p],
        "ccz4_field_ptr": [vp, ctypes.c_int, ctypes.POINTER(_dbl_p), ll_p],
        "ccz4_upload": [vp, ctypes.c_int, _dbl_p, _dbl_p, vp],
        "ccz4_download": [vp, ctypes.c_int, _dbl_p, _dbl_p, vp],
        "ccz4_fill_halos": [vp, ctypes.c_int, vp],
        "ccz4_fill_halos_for": [vp, ctypes.c_int, ctypes.POINTER(Params), vp],
        "ccz4_rhs": [vp, ctypes.POINTER(Params), ctypes.c_int, ctypes.c_int, vp],
        "ccz4_rk_stage": [vp, ctypes.POINTER(Params), ctypes.c_int, ctypes.c_double, vp],
        "ccz4_stage_buffers": [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
        "ccz4_step": [vp, ctypes.POINTER(Params), ctypes.c_double, ctypes.c_int, vp],
        "ccz4_step_graph": [vp, ctypes.POINTER(Params), ctypes.c_double, ctypes.c_int, vp],
        "ccz4_evolve_host": [vp, ctypes.POINTER(Params), ctypes.c_double, ctypes.c_int,
                             _dbl_p, _dbl_p, _dbl_p, _dbl_p, vp],
        "ccz4_enforce": [vp, ctypes.c_int, vp],
        "ccz4_constraints": [vp, ctypes.c_int, _dbl_p, _dbl_p, _dbl_p, vp],
        "ccz4_alloc_mesh": [ctypes.POINTER(MeshDesc), ctypes.POINTER(vp)],
        "ccz4_mesh_info": [vp, ctypes.POINTER(ctypes.c_int), ll_p],
        "ccz4_restrict": [vp, ctypes.c_int, vp],
        "ccz4_set_launch": [vp, ctypes.c_int],
        "ccz4_set_tuning": [vp, ctypes.c_int, ctypes.c_int],
        "ccz4_point_index": [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ll_p, vp],
        "ccz4_psi4": [vp, ctypes.c_int, ctypes.c_int, _dbl_p, vp],
        "ccz4_set_allocator": [_ALLOC_FN, _DEALLOC_FN, vp],
        "ccz4_mesh_plan": [ctypes.POINTER(MeshDesc), ll_p, ctypes.POINTER(ctypes.c_int),
                           ctypes.POINTER(ctypes.c_int)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    fo_sig = {
        "ccz4_fo_alloc": [vp, ctypes.c_int, ctypes.POINTER(vp)],
        "ccz4_fo_free": [vp],
        "ccz4_fo_upload": [vp, ctypes.c_int, _dbl_p, _dbl_p, vp],
        "ccz4_fo_download": [vp, ctypes.c_int, _dbl_p, _dbl_p, vp],
        "ccz4_fo_rhs": [vp, ctypes.POINTER(Params), ctypes.c_int, ctypes.c_int, vp],
        "ccz4_fo_reconstruct": [vp, ctypes.c_int, vp],
        "ccz4_fo_rk_stage": [vp, ctypes.POINTER(Params), ctypes.c_int, ctypes.c_double, vp],
        "ccz4_fo_step": [vp, ctypes.POINTER(Params), ctypes.c_double, ctypes.c_int, vp],
    }
    for name, args in fo_sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.ccz4_constraints_excluding.argtypes = [vp, vp, vp, ctypes.c_int, _dbl_p, ctypes.c_double, _dbl_p, vp]
    L.ccz4_constraints_excluding.restype = ctypes.c_int
    L.ccz4_tracers_new.argtypes = [vp, ctypes.c_int, _dbl_p, ctypes.c_int, ctypes.c_double, ctypes.POINTER(vp)]
    L.ccz4_tracers_step.argtypes = [vp, ctypes.c_int, ctypes.c_double, vp]
    L.ccz4_tracers_read.argtypes = [vp, _dbl_p, _dbl_p, vp]
    L.ccz4_tracers_free.argtypes = [vp]
    for f in (L.ccz4_tracers_new, L.ccz4_tracers_step, L.ccz4_tracers_read, L.ccz4_tracers_free):
        f.restype = ctypes.c_int
    L.ccz4_flops_per_point_stage.argtypes = [ctypes.POINTER(Params), _dbl_p]
    L.ccz4_flops_per_point_stage.restype = ctypes.c_int
    L.ccz4_last_error.restype = ctypes.c_char_p
    L.ccz4_last_error.argtypes = []
    _lib = L
    return L


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_DEALLOC_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_TORCH_ALLOCATOR = None   # the callbacks handed to the library, kept alive while it may call them


def use_torch_allocator(enable=True):
    """Grids created from now on take their large buffers (state buffers,
    halo tiles, mixed derivatives) from PyTorch's caching allocator on the
    current device (ccz4_set_allocator); enable=False restores cudaMalloc.
    Grids keep the allocator they were created with."""
    global _TORCH_ALLOCATOR
    if not enable:
        _check(lib().ccz4_set_allocator(_ALLOC_FN(), _DEALLOC_FN(), None))
        return
    import torch

    def alloc(ctx, nbytes, stream):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes))
        except RuntimeError:
            return None

    def dealloc(ctx, ptr, nbytes, stream):
        torch.cuda.caching_allocator_delete(int(ptr))
    cbs = (_ALLOC_FN(alloc), _DEALLOC_FN(dealloc))
    _check(lib().ccz4_set_allocator(cbs[0], cbs[1], None))
    _TORCH_ALLOCATOR = cbs


def _check(code):
    if code != OK:
        raise CCZ4Error(code, lib().ccz4_last_error().decode())


def make_params(kappa1=1.0, kappa2=0.0, kappa3=0.0, e=1.0, c=1.0, tau=1.0, mu=0.2, f=0.75,
                eta=2.0, s=1.0, K0=0.0, ko_eps=0.1, slicing="harmonic", shift="zero",
                somm_speed=1.0, precision="fp64"):
    P = Params()
    for k, v in dict(kappa1=kappa1, kappa2=kappa2, kappa3=kappa3, e=e, c=c, tau=tau, mu=mu, f=f,
                     eta=eta, s=s, K0=K0, ko_eps=ko_eps).items():
        setattr(P, k, float(v))
    P.slicing = SLICING[slicing] if isinstance(slicing, str) else int(slicing)
    P.shift = SHIFT[shift] if isinstance(shift, str) else int(shift)
    P.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    sp = np.broadcast_to(np.asarray(somm_speed, dtype=np.float64), (NV,))
    for i in range(NV):
        P.somm_speed[i] = float(sp[i])
    return P


def flops_per_point_stage(precision="fp64", P=None):
    """Algorithmic flops of one interior point-stage of the stage kernel
    (counted on the host from the kernel's own templates)."""
    if P is None:
        from .inputs import PUNCTURE_PARAMS
        P = make_params(**PUNCTURE_PARAMS, precision=precision)
    out = (ctypes.c_double * 6)()
    _check(lib().ccz4_flops_per_point_stage(ctypes.byref(P), out))
    return {"fp64": out[0], "fp32": out[1], "fp64_div_root": out[2], "conversions": out[3],
            "fp64_fma": out[4], "fp64_add_mul": out[5]}


def stage_buffers(stage):
    """(input, output) buffer ids of RK stage s."""
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(lib().ccz4_stage_buffers(int(stage), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return ctypes.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _wrap_device(ptr, shape, dtype):
    """Zero-copy torch view of device memory owned by the library."""
    import torch
    typestr = {torch.float64: "<f8", torch.float32: "<f4", torch.int32: "<i4"}[dtype]

    class _CAI:
        __cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                    "version": 3, "strides": None}
    return torch.as_tensor(_CAI(), device="cuda")


def _buf(b):
    return BUF[b] if isinstance(b, str) else int(b)


def _d(a):
    return a.ctypes.data_as(_dbl_p) if a is not None else None


def _mesh_desc(p, np_, level, ijk, origin, dx, bc):
    level = np.ascontiguousarray(level, dtype=np.int32).reshape(-1)
    ijk = np.ascontiguousarray(ijk, dtype=np.int32).reshape(-1, 3)
    d = MeshDesc()
    d.p = int(p)
    for q in range(3):
        d.np[q] = int(np_[q])
        d.origin[q] = float(origin[q])
    d.n_patches = len(ijk)
    d.level = level.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    d.ijk = ijk.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    d.dx = float(dx)
    d.bc = BC[bc] if isinstance(bc, str) else int(bc)
    return d, (level, ijk)  # keep the arrays alive with the descriptor


def mesh_plan(p, np_, level, ijk, origin, dx, bc="periodic"):
    """Host-only plan of a refined mesh (no GPU needed): returns the tile
    sources (n_patches, (p+6)^3) and the interpolation entries (n_interp, 9),
    as ccz4_mesh_plan describes them."""
    d, keep = _mesh_desc(p, np_, level, ijk, origin, dx, bc)
    n = ctypes.c_longlong()
    _check(lib().ccz4_mesh_plan(ctypes.byref(d), ctypes.byref(n), None, None))
    T3 = (int(p) + 6) ** 3
    src = np.empty((len(keep[1]), T3), dtype=np.int32)
    interp = np.empty((max(n.value, 1), 9), dtype=np.int32)
    ip = ctypes.POINTER(ctypes.c_int)
    _check(lib().ccz4_mesh_plan(ctypes.byref(d), ctypes.byref(n), src.ctypes.data_as(ip), interp.ctypes.data_as(ip)))
    return src, interp[:n.value]


class Grid:
    """p^3 patches on the current CUDA device: one uniform level, or (with
    ``level``) a statically refined mesh of ratio-3 levels whose level-l
    patches have spacing dx / 3^l and slots ijk in level-l units."""

    def __init__(self, p, np_, ijk, origin, dx, bc="periodic", level=None):
        L = lib()
        self.p = int(p)
        self.np = tuple(int(v) for v in np_)
        self.ijk = np.ascontiguousarray(ijk, dtype=np.int32).reshape(-1, 3)
        self.n_patches = len(self.ijk)
        h = ctypes.c_void_p()
        if level is None:
            d = GridDesc()
            d.p = self.p
            for q in range(3):
                d.np[q] = self.np[q]
                d.origin[q] = float(origin[q])
            d.n_patches = self.n_patches
            d.ijk = self.ijk.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
            d.dx = float(dx)
            d.bc = BC[bc] if isinstance(bc, str) else int(bc)
            _check(L.ccz4_alloc_patches(ctypes.byref(d), ctypes.byref(h)))
            self.level = np.zeros(self.n_patches, dtype=np.int32)
        else:
            d, keep = _mesh_desc(self.p, self.np, level, self.ijk, origin, dx, bc)
            _check(L.ccz4_alloc_mesh(ctypes.byref(d), ctypes.byref(h)))
            self.level = keep[0]
        self._h = h
        n, g, s = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        _check(L.ccz4_grid_info(h, ctypes.byref(n), ctypes.byref(g), ctypes.byref(s)))
        self.n_points, self.n_ghost, self.field_stride = n.value, g.value, s.value
        nl, nleaf = ctypes.c_int(), ctypes.c_longlong()
        _check(L.ccz4_mesh_info(h, ctypes.byref(nl), ctypes.byref(nleaf)))
        self.n_levels, self.n_leaf_points = nl.value, nleaf.value
        self.origin = tuple(float(v) for v in origin)
        self.dx = float(dx)

    @classmethod
    def from_config(cls, cfg):
        return cls(cfg.p, cfg.np, cfg.ijk(), cfg.origin, cfg.dx, cfg.bc, level=getattr(cfg, "level", None))

    def set_launch(self, mode):
        """'flat' (default) or 'queue' launch of the stage kernel, or 'fused'
        (9^3 patches): the fill and the stage of each RK stage of step and
        step_graph in one cooperative launch."""
        m = {"flat": 0, "queue": 1, "fused": 2}[mode] if isinstance(mode, str) else int(mode)
        _check(lib().ccz4_set_launch(self._h, m))

    def set_tuning(self, stage_shape=0, fill_shape=0):
        """Launch shapes of the flat stage kernel (0 default, 1 one resident
        block more, 2 one fewer, 3 two phases (mixed precision)) and of the halo fill (0 default, 1 512
        threads, 2 16 loads per thread, 3 128 threads); results are identical."""
        _check(lib().ccz4_set_tuning(self._h, int(stage_shape), int(fill_shape)))

    def restrict(self, buf="U", stream=None):
        """Coarse points under refined patches <- mean of their 27 fine cells."""
        _check(lib().ccz4_restrict(self._h, _buf(buf), _stream(stream)))

    def close(self):
        if getattr(self, "_h", None):
            lib().ccz4_free_patches(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- data movement ------------------------------------------------------
    def upload(self, U, G=None, buf="U", stream=None):
        U = np.ascontiguousarray(U, dtype=np.float64).reshape(NV, self.n_points)
        Gc = None
        if self.n_ghost:
            Gc = np.ascontiguousarray(G, dtype=np.float64).reshape(NV, self.n_ghost)
        _check(lib().ccz4_upload(self._h, _buf(buf), _d(U), _d(Gc), _stream(stream)))

    def download(self, buf="U", stream=None):
        if _buf(buf) == BUF["TILE"]:
            T = self.p + 6
            out = np.empty((NV, self.n_patches, T, T, T))
            _check(lib().ccz4_download(self._h, BUF["TILE"], _d(out), None, _stream(stream)))
            return out
        if _buf(buf) == BUF["MIX"]:
            out = np.empty((NMIX, self.n_points))
            _check(lib().ccz4_download(self._h, BUF["MIX"], _d(out), None, _stream(stream)))
            return out
        U = np.empty((NV, self.n_patches, self.p, self.p, self.p))
        G = np.empty((NV, self.n_ghost))
        _check(lib().ccz4_download(self._h, _buf(buf), _d(U), _d(G) if self.n_ghost else None,
                                   _stream(stream)))
        return U, G

    def device_ptr(self, buf):
        p, n = _dbl_p(), ctypes.c_longlong()
        _check(lib().ccz4_field_ptr(self._h, _buf(buf), ctypes.byref(p), ctypes.byref(n)))
        return ctypes.cast(p, ctypes.c_void_p).value, n.value

    def as_tensor(self, buf):
        """Zero-copy torch view (1-D, float64) of a device buffer."""
        import torch
        ptr, n = self.device_ptr(buf)
        return _wrap_device(ptr, (n,), torch.float64)

    # -- the hot path -----------------------------------------------------------
    def fill_halos(self, buf="U", stream=None, P=None):
        """Halo fill of a state buffer; with parameters P, as the stage kernel
        for P needs it. In the mixed path, the tiles of every field but alpha
        and phi then hold split FP32 pairs {hi, lo} (hi + lo = the FP64 value
        within 2^-48 of it; view a downloaded tile field as float32 pairs),
        and the mixed derivatives of g~ and beta are stored with FP32
        weights as FP32."""
        if P is None:
            _check(lib().ccz4_fill_halos(self._h, _buf(buf), _stream(stream)))
        else:
            _check(lib().ccz4_fill_halos_for(self._h, _buf(buf), ctypes.byref(P), _stream(stream)))

    def rhs(self, P, in_buf="U", out_buf="RHS", stream=None):
        _check(lib().ccz4_rhs(self._h, ctypes.byref(P), _buf(in_buf), _buf(out_buf), _stream(stream)))

    def rk_stage(self, P, stage, dt, stream=None, fill=True):
        """RK4 stage s; with fill=True the halo of the stage input is filled first."""
        if fill:
            self.fill_halos(stage_buffers(stage)[0], stream, P)
        _check(lib().ccz4_rk_stage(self._h, ctypes.byref(P), int(stage), float(dt), _stream(stream)))

    def step(self, P, dt, n_steps=1, stream=None):
        _check(lib().ccz4_step(self._h, ctypes.byref(P), float(dt), int(n_steps), _stream(stream)))

    def step_graph(self, P, dt, n_steps=1, stream=None):
        _check(lib().ccz4_step_graph(self._h, ctypes.byref(P), float(dt), int(n_steps), _stream(stream)))

    def evolve_host(self, P, dt, n_steps, U, G=None, U_out=None, G_out=None, stream=None):
        U = np.ascontiguousarray(U, dtype=np.float64)
        U_out = np.empty_like(U) if U_out is None else U_out
        Gc = G_o = None
        if self.n_ghost:
            Gc = np.ascontiguousarray(G, dtype=np.float64)
            G_o = np.empty_like(Gc) if G_out is None else G_out
        _check(lib().ccz4_evolve_host(self._h, ctypes.byref(P), float(dt), int(n_steps), _d(U), _d(Gc),
                                      _d(U_out), _d(G_o), _stream(stream)))
        return U_out, G_o

    def enforce(self, buf="U", stream=None):
        _check(lib().ccz4_enforce(self._h, _buf(buf), _stream(stream)))

    def constraints(self, buf="U", dev_H=None, dev_M=None, stream=None, raise_nonfinite=True):
        out = np.empty(5)
        code = lib().ccz4_constraints(self._h, _buf(buf), _d(out),
                                      ctypes.cast(dev_H, _dbl_p) if dev_H else None,
                                      ctypes.cast(dev_M, _dbl_p) if dev_M else None, _stream(stream))
        if code == ERR_NONFINITE and not raise_nonfinite:
            return out
        _check(code)
        return out

    def psi4(self, in_buf="U", out_buf="RHS", centre=(0.0, 0.0, 0.0), stream=None):
        """psi_4 of the state in in_buf into fields 0 (Re) and 1 (Im) of
        out_buf at every interior point (ccz4_psi4), the tetrad centred at
        `centre`."""
        c = np.ascontiguousarray(centre, dtype=np.float64).reshape(3)
        _check(lib().ccz4_psi4(self._h, _buf(in_buf), _buf(out_buf), _d(c), _stream(stream)))

    def point_index(self, xyz, stream=None, raise_bounds=True):
        """Index within a field of a state buffer of each lattice point
        (x, y, z) (ccz4_point_index): -1 for a point beyond the ghost shell,
        which raises CCZ4Error (ERR_BOUNDS) unless raise_bounds is False."""
        q = np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3)
        out = np.empty(len(q), dtype=np.int64)
        code = lib().ccz4_point_index(self._h, len(q), q.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                      out.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), _stream(stream))
        if code != ERR_BOUNDS or raise_bounds:
            _check(code)
        return out

    def constraints_excluding(self, dev_H, dev_M, centres, radius=1.0, stream=None):
        """Norms of the per-point H and M (device pointers, as constraints()
        writes them) over leaf points at a distance >= radius from every
        centre: (L2 H, L2 |M|, max |H|, max |M|, point count)."""
        c = np.ascontiguousarray(centres, dtype=np.float64).reshape(-1, 3)
        out = np.empty(5)
        _check(lib().ccz4_constraints_excluding(self._h, ctypes.c_void_p(dev_H), ctypes.c_void_p(dev_M), len(c),
                                                _d(c), float(radius), _d(out), _stream(stream)))
        return out


FO_VARIANT = {"fo": 0, "so-recon": 1}


class FirstOrder:
    """The 58-variable formulations on a single-level grid (ccz4_fo_* in
    include/ccz4.h): variant "fo", the first-order formulation (every
    variable evolved, red terms kept), or "so-recon", the second-order one
    whose auxiliary variables are reconstructed from FD4 derivatives of the
    primaries before every stage. Arrays are (58, n_patches, p, p, p) and
    (58, n_ghost)."""

    NV = 58

    def __init__(self, grid, variant="fo"):
        self.grid = grid   # the grid must outlive the formulation
        self.variant = variant
        h = ctypes.c_void_p()
        _check(lib().ccz4_fo_alloc(grid._h, FO_VARIANT[variant], ctypes.byref(h)))
        self._h = h

    def upload(self, U, G=None, buf="U", stream=None):
        g = self.grid
        U = np.ascontiguousarray(U, dtype=np.float64).reshape(self.NV, g.n_points)
        Gc = np.ascontiguousarray(G, dtype=np.float64).reshape(self.NV, g.n_ghost) if g.n_ghost else None
        _check(lib().ccz4_fo_upload(self._h, _buf(buf), _d(U), _d(Gc), _stream(stream)))

    def download(self, buf="U", stream=None):
        g = self.grid
        U = np.empty((self.NV, g.n_patches, g.p, g.p, g.p))
        G = np.empty((self.NV, g.n_ghost))
        _check(lib().ccz4_fo_download(self._h, _buf(buf), _d(U), _d(G) if g.n_ghost else None, _stream(stream)))
        return U, G

    def rhs(self, P, in_buf="U", out_buf="RHS", stream=None):
        _check(lib().ccz4_fo_rhs(self._h, ctypes.byref(P), _buf(in_buf), _buf(out_buf), _stream(stream)))

    def reconstruct(self, buf="U", stream=None):
        _check(lib().ccz4_fo_reconstruct(self._h, _buf(buf), _stream(stream)))

    def rk_stage(self, P, stage, dt, stream=None):
        _check(lib().ccz4_fo_rk_stage(self._h, ctypes.byref(P), int(stage), float(dt), _stream(stream)))

    def step(self, P, dt, n_steps=1, stream=None):
        _check(lib().ccz4_fo_step(self._h, ctypes.byref(P), float(dt), int(n_steps), _stream(stream)))

    def close(self):
        if getattr(self, "_h", None):
            lib().ccz4_fo_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Tracers:
    """Particle tracers on a grid (ccz4_tracers_* in include/ccz4.h): each
    step records the 25 fields at every tracer by trilinear interpolation
    and, with a velocity field, moves it by one explicit Euler step.
    Puncture trackers: ``Tracers(grid, positions, velocity="shift")``, which
    moves with the opposite shift."""

    def __init__(self, grid, pos, vel_field=-1, vel_scale=-1.0, velocity=None):
        if velocity == "shift":
            from .inputs import IDX
            vel_field, vel_scale = IDX["betax"], -1.0
        pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
        self.n = len(pos)
        self.grid = grid     # the grid must outlive the tracers
        h = ctypes.c_void_p()
        _check(lib().ccz4_tracers_new(grid._h, self.n, _d(pos), int(vel_field), float(vel_scale), ctypes.byref(h)))
        self._h = h

    def step(self, buf="U", dt=0.0, stream=None):
        _check(lib().ccz4_tracers_step(self._h, _buf(buf), float(dt), _stream(stream)))

    def read(self, stream=None, raise_bounds=True):
        """(positions (n, 3), last step's values (n, 25)); raises on a tracer
        the grid could not resolve unless raise_bounds is False."""
        pos = np.empty((self.n, 3))
        val = np.empty((self.n, NV))
        code = lib().ccz4_tracers_read(self._h, _d(pos), _d(val), _stream(stream))
        if code != ERR_BOUNDS or raise_bounds:
            _check(code)
        return pos, val

    def close(self):
        if getattr(self, "_h", None):
            lib().ccz4_tracers_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def constraints_noalloc(tiles_ptr, p, n_patches, dx, H_ptr, M_ptr, out_ptr, stream=None):
    """Constraint monitors from caller-held halo tiles, allocating nothing
    (ccz4_constraints_noalloc in include/ccz4.h): for callers that cannot
    allocate device memory. All pointers are device addresses; H_ptr and
    M_ptr may be None; out_ptr receives the 5 reduced values on the device."""
    f = lib().ccz4_constraints_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    _check(f(ctypes.c_void_p(tiles_ptr), int(p), int(n_patches), float(dx),
             ctypes.c_void_p(H_ptr) if H_ptr else None, ctypes.c_void_p(M_ptr) if M_ptr else None,
             ctypes.c_void_p(out_ptr), _stream(stream)))
