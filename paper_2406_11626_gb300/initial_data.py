"""Python binding of the puncture initial-data solve (include/ccz4_id.h):
argument marshalling only; every step runs in the CUDA kernels of the
library (no CPU fallback)."""
import ctypes
import math

import numpy as np

from .ccz4 import _check, _stream, lib as _lib

MAX_PUNCTURES = 4


class Punctures(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("m", ctypes.c_double * MAX_PUNCTURES),
                ("c", (ctypes.c_double * 3) * MAX_PUNCTURES), ("P", (ctypes.c_double * 3) * MAX_PUNCTURES),
                ("S", (ctypes.c_double * 3) * MAX_PUNCTURES)]


def make_punctures(masses, centres, momenta=None, spins=None):
    B = Punctures()
    B.n = len(masses)
    for k in range(B.n):
        B.m[k] = float(masses[k])
        for d in range(3):
            B.c[k][d] = float(centres[k][d])
            B.P[k][d] = float(momenta[k][d]) if momenta is not None else 0.0
            B.S[k][d] = float(spins[k][d]) if spins is not None else 0.0
    return B


def binary(m1, m2, d, P, S):
    """Two punctures on the x axis at -d/2 (mass m1) and +d/2 (mass m2),
    momenta (0, -P, 0) and (0, +P, 0) (a circular-orbit pattern), spins
    (0, 0, S) each."""
    return make_punctures([m1, m2], [(-0.5 * d, 0.0, 0.0), (0.5 * d, 0.0, 0.0)],
                          [(0.0, -P, 0.0), (0.0, P, 0.0)], [(0.0, 0.0, S), (0.0, 0.0, S)])


def _sig():
    L = _lib()
    if getattr(L, "_id_ready", False):
        return L
    vp = ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    sigs = {
        "ccz4_id_create": [ctypes.c_int, ctypes.c_double, ctypes.POINTER(vp)],
        "ccz4_id_free": [vp],
        "ccz4_id_set_punctures": [vp, ctypes.POINTER(Punctures), vp],
        "ccz4_id_u_ptr": [vp, ctypes.POINTER(dp)],
        "ccz4_id_sweeps": [vp, ctypes.c_int, vp],
        "ccz4_id_set_relaxation": [vp, ctypes.c_double],
        "ccz4_id_residual": [vp, dp, dp, vp],
        "ccz4_id_solve": [vp, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp, vp],
        "ccz4_id_assemble": [vp, ctypes.POINTER(Punctures), vp, ctypes.c_int, vp],
        "ccz4_id_assemble_box": [vp, ctypes.POINTER(Punctures), vp, ctypes.c_int, vp],
        "ccz4_id_set_parent": [vp, vp, ctypes.c_int, vp],
    }
    for name, args in sigs.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L._id_ready = True
    return L


class Solver:
    """The Hamiltonian-constraint solve for u on n^3 cells of [-L, L]^3."""

    def __init__(self, n, L):
        self.n, self.L = int(n), float(L)
        h = ctypes.c_void_p()
        _check(_sig().ccz4_id_create(self.n, self.L, ctypes.byref(h)))
        self._h = h
        p = ctypes.POINTER(ctypes.c_double)()
        _check(_sig().ccz4_id_u_ptr(h, ctypes.byref(p)))
        self.u_ptr = ctypes.cast(p, ctypes.c_void_p).value

    def close(self):
        if getattr(self, "_h", None):
            _sig().ccz4_id_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def u_tensor(self):
        """u as a torch tensor view of the device buffer ([n][n][n], x fastest)."""
        import torch
        from .ccz4 import _wrap_device
        return _wrap_device(self.u_ptr, (self.n,) * 3, torch.float64)

    def set_relaxation(self, omega):
        """Relaxation factor of the point update (1: Gauss-Seidel)."""
        _check(_sig().ccz4_id_set_relaxation(self._h, float(omega)))

    def set_punctures(self, B, stream=None):
        _check(_sig().ccz4_id_set_punctures(self._h, ctypes.byref(B), _stream(stream)))

    def set_u(self, u, stream=None):
        self.u_tensor().copy_(_as_tensor(u).reshape((self.n,) * 3))

    def get_u(self):
        return self.u_tensor().cpu().numpy().copy()

    def sweeps(self, k, stream=None):
        _check(_sig().ccz4_id_sweeps(self._h, int(k), _stream(stream)))

    def residual(self, stream=None, cells=False):
        r = ctypes.c_double()
        res = None
        if cells:
            import torch
            res = torch.empty((self.n,) * 3, dtype=torch.float64, device="cuda")
            ptr = ctypes.cast(ctypes.c_void_p(res.data_ptr()), ctypes.POINTER(ctypes.c_double))
        else:
            ptr = None
        _check(_sig().ccz4_id_residual(self._h, ctypes.byref(r), ptr, _stream(stream)))
        return (r.value, res.cpu().numpy()) if cells else r.value

    def solve(self, tol=1e-10, max_sweeps=1000000, check=50, stream=None):
        """Sweeps from the current u; returns (sweeps or -1, final residual)."""
        k, r = ctypes.c_int(), ctypes.c_double()
        _check(_sig().ccz4_id_solve(self._h, float(tol), int(max_sweeps), int(check), ctypes.byref(k),
                                    ctypes.byref(r), _stream(stream)))
        return k.value, r.value

    def assemble(self, B, grid, buf="U", stream=None):
        """Writes the CCZ4 state of the solved data into a state buffer of a
        ccz4.Grid (every interior point of every level and every ghost cell)."""
        from .ccz4 import _buf
        _check(_sig().ccz4_id_assemble(self._h, ctypes.byref(B), grid._h, _buf(buf), _stream(stream)))

    def assemble_box(self, B, grid, buf="U", stream=None):
        """As assemble, for the points with every |x_d| < L - 3h/2 only."""
        from .ccz4 import _buf
        _check(_sig().ccz4_id_assemble_box(self._h, ctypes.byref(B), grid._h, _buf(buf), _stream(stream)))

    def set_parent(self, parent, init_u=True, stream=None):
        """Makes this solver a box nested in `parent` (fixed ghost values from
        the parent's current u; with init_u also the first guess), or with
        parent None restores the 1/r fall-off ghosts."""
        _check(_sig().ccz4_id_set_parent(self._h, parent._h if parent is not None else None, int(bool(init_u)),
                                         _stream(stream)))


def solve_config(cfg, stream=None):
    """The solver of a binary-puncture config after its plain solve from
    u = 0 to the config's tolerance; returns (solver, punctures, sweeps)."""
    e = cfg.extra
    s = Solver(e["id_n"], e["id_L"])
    s.set_relaxation(e.get("id_omega", 1.0))
    B = binary(e["m1"], e["m2"], e["d"], e["P"], e["S"])
    s.set_punctures(B, stream)
    k, r = s.solve(tol=e["id_tol"], check=e.get("id_check", 200), stream=stream)
    if k < 0:
        raise RuntimeError("initial-data solve did not reach %g (residual %g)" % (e["id_tol"], r))
    return s, B, k


def box_omega(n):
    """Over-relaxation factor of a box with fixed ghosts: Young's optimum
    for the 7-point Laplacian on n cells per axis with Dirichlet data,
    2 / (1 + sin(pi / (n + 1)))."""
    return 2.0 / (1.0 + math.sin(math.pi / (n + 1)))


def solve_nested(cfg, stream=None, log=None):
    """The initial-data solve of a binary-puncture config on its nested
    boxes: the global solve (solve_config), then each box of
    cfg.extra["id_boxes"] ((n, L) pairs, outermost first) from its parent's
    interpolated u with fixed ghosts from it, to the same tolerance.
    Returns (solvers, punctures, sweeps per solver)."""
    s, B, k = solve_config(cfg, stream)
    solvers, sweeps = [s], [k]
    e = cfg.extra
    for n, L in e.get("id_boxes", ()):
        b = Solver(n, L)
        b.set_punctures(B, stream)
        b.set_parent(solvers[-1], init_u=True, stream=stream)
        b.set_relaxation(box_omega(n))
        kb, r = b.solve(tol=e["id_tol"], check=e.get("id_check", 200), stream=stream)
        if kb < 0:
            raise RuntimeError("initial-data box (n=%d, L=%g) did not reach %g (residual %g)"
                               % (n, L, e["id_tol"], r))
        if log:
            log("initial-data box n=%d L=%g h=%.4g: %d sweeps, residual %.2e" % (n, L, 2.0 * L / n, kb, r))
        solvers.append(b)
        sweeps.append(kb)
    return solvers, B, sweeps


def assemble_nested(solvers, B, grid, buf="U", stream=None):
    """The CCZ4 state from nested solvers: the outermost everywhere, then
    each box, coarse to fine, where its stencil is centred."""
    solvers[0].assemble(B, grid, buf, stream)
    for b in solvers[1:]:
        b.assemble_box(B, grid, buf, stream)


def _as_tensor(a):
    import torch
    if isinstance(a, torch.Tensor):
        return a.to(device="cuda", dtype=torch.float64)
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def main(argv=None):
    """Solves the puncture initial data of one binary from u = 0 and prints
    the sweeps, the residual and the time per sweep (CUDA events)."""
    import argparse
    import json
    import torch
    ap = argparse.ArgumentParser(description="Bowen-York initial data of a binary puncture on the GPU")
    ap.add_argument("--n", type=int, default=96, help="cells per axis")
    ap.add_argument("--L", type=float, default=16.0, help="half width of the grid")
    ap.add_argument("--binary", type=float, nargs=5, default=(0.487, 0.487, 6.0, 0.0934, 0.0),
                    metavar=("M1", "M2", "D", "P", "S"), help="bare masses, separation, momentum, spin")
    ap.add_argument("--omega", type=float, default=1.97, help="relaxation factor (1: Gauss-Seidel)")
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--check", type=int, default=20, help="sweeps between residual checks")
    ap.add_argument("--sweeps", type=int, default=0, help="run exactly this many sweeps instead of a solve")
    a = ap.parse_args(argv)
    s = Solver(a.n, a.L)
    s.set_relaxation(a.omega)
    s.set_punctures(binary(*a.binary))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    if a.sweeps > 0:
        s.sweeps(a.sweeps)
        k = a.sweeps
    else:
        k, _ = s.solve(tol=a.tol, check=a.check)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    out = {"n": a.n, "L": a.L, "omega": a.omega, "sweeps": k, "residual": s.residual(), "ms": ms,
           "us_per_sweep": 1e3 * ms / max(k, 1)}
    print(json.dumps(out))
    return 0 if k > 0 else 1


if __name__ == "__main__":
    raise SystemExit(main())
