"""Helpers shared by the parity tests (the GPU ones and the host evaluation
of the kernel templates): build the same seeded problem for the CUDA
library (through its C ABI) and for the CPU oracle."""
import numpy as np

import oracle as O
from paper_2406_11626_gb300 import inputs as I


def rel_err(a, b):
    """Per-field relative max-norm: ||a - b||_inf / max(||b||_inf, 1)."""
    a = np.asarray(a).reshape(I.NV, -1)
    b = np.asarray(b).reshape(I.NV, -1)
    if a.shape[1] == 0:
        return np.zeros(I.NV)
    return np.abs(a - b).max(axis=1) / np.maximum(np.abs(b).max(axis=1), 1.0)


def make_pair(p, npv, origin, dx, bc, permute_seed=None):
    from paper_2406_11626_gb300 import ccz4 as C
    ijk = I.patch_ijk(npv, permute_seed)
    return C.Grid(p, npv, ijk, origin, dx, bc), O.Grid(p, npv, ijk, origin, dx, bc), ijk


def random_state(p, npv, origin, dx, ijk, seed, bc, amp=0.02, base="flat"):
    """Smooth perturbation of flat space (or of puncture data) in every field,
    plus its Sommerfeld ghost shell, on the same points for both sides."""
    x, y, z = I.point_coords(p, ijk, origin, dx)
    box = npv[0] * p * dx
    N = tuple(n * p for n in npv)
    if base == "puncture":
        U0 = I.brill_lindquist(x, y, z)
    else:
        U0 = I.flat(x.shape)
    U = I.smooth_perturbation(x, y, z, seed, amp=amp, box=box, base=U0)
    G = np.zeros((I.NV, 0))
    if bc == "sommerfeld":
        gx, gy, gz = I.ghost_positions(N, origin, dx)
        G0 = I.brill_lindquist(gx, gy, gz) if base == "puncture" else I.flat(gx.shape)
        G = I.smooth_perturbation(gx, gy, gz, seed, amp=amp, box=box, base=G0)
    return np.ascontiguousarray(U), np.ascontiguousarray(G)


def both_params(**kw):
    from paper_2406_11626_gb300 import ccz4 as C
    return C.make_params(**kw), O.make_params(**{k: v for k, v in kw.items() if k != "precision"})


def ko_pieces(tiles, v, p):
    """From an FP64 tile of field v: the largest first second difference
    |u(x+h) + u(x-h) - 2u(x)| over the interior points and the three axes,
    and the Kreiss-Oliger sum evaluated naively in FP32 (every value
    rounded to FP32 first, the sum in FP32), shaped like the interior."""
    t = tiles[v]
    n = t.shape[0]
    inner = (slice(None),) + (slice(3, 3 + p),) * 3

    def shift(a, axis, k):
        sl = [slice(None), slice(3, 3 + p), slice(3, 3 + p), slice(3, 3 + p)]
        sl[axis] = slice(3 + k, 3 + k + p)
        return a[tuple(sl)]

    b1 = max(np.abs(shift(t, ax, 1) + shift(t, ax, -1) - 2.0 * t[inner]).max() for ax in (1, 2, 3))
    t32 = t.astype(np.float32)
    ko = np.zeros((n, p, p, p), np.float32)
    for ax in (1, 2, 3):
        s1 = shift(t32, ax, 1) + shift(t32, ax, -1)
        s2 = shift(t32, ax, 2) + shift(t32, ax, -2)
        s3 = shift(t32, ax, 3) + shift(t32, ax, -3)
        ko += s3 - np.float32(6.0) * s2 + np.float32(15.0) * s1 - np.float32(20.0) * t32[inner]
    return b1, ko


def offset_state(p, npv, origin, dx, ijk):
    """A periodic smooth perturbation of flat space with beta = 1000 + s and
    b = -500 + s (s smooth, of size 1e-3): with the zero-shift option their
    right-hand sides are pure Kreiss-Oliger dissipation, blind to the
    offsets. Returns U, G and the offsets by field name."""
    U, G = random_state(p, npv, origin, dx, ijk, seed=9, bc="periodic")
    offset = {"betax": 1000.0, "betay": 1000.0, "betaz": 1000.0, "bx": -500.0, "by": -500.0, "bz": -500.0}
    for name, c in offset.items():
        U[I.IDX[name]] = c + 0.05 * (U[I.IDX[name]] + U[I.IDX["gxx"]] - 1.0)
    return U, G, offset
