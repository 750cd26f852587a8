"""Helpers shared by the GPU parity tests: build the same seeded problem for
the CUDA library (through its C ABI) and for the CPU oracle."""
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
