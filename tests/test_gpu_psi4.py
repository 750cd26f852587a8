"""psi_4 on the GPU (ccz4_psi4 through the C ABI) against the oracle's
og_psi4, per point, on a boosted black hole's exact data (the hole outside
the grid, the tetrad centred off the grid's centre), on perturbed puncture
data of a shuffled grid and on a three-level mesh; and the extraction on a
sphere (static tracers, the quadrature of psi4.py) against the oracle's
sampling of its own psi_4, and against the brute-force Weyl tensor."""
import numpy as np
import pytest

import oracle as O
import weyl_reference as W
from paper_2406_11626_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-30)


def _ks_state(cfg, st):
    x, y, z = I.point_coords(cfg.p, cfg.ijk(), cfg.origin, cfg.dx)
    gx, gy, gz = I.ghost_positions(cfg.N, cfg.origin, cfg.dx)
    return W.ccz4_state(st, x, y, z), W.ccz4_state(st, gx, gy, gz)


def _gpu_psi4(cfg, U, G, centre, mesh=False):
    from paper_2406_11626_gb300 import ccz4 as C
    g = C.Grid.from_config(cfg)
    g.upload(U, G)
    g.psi4("U", "RHS", centre)
    R, _ = g.download("RHS")
    return g, R[:2]


@pytest.mark.parametrize("centre", [(0.0, 0.0, 0.0), (0.13, -0.21, 0.07)])
def test_psi4_matches_oracle_on_a_boosted_black_hole(centre):
    cfg = I.single_puncture_config(p=6, n_side=3, half_width=1.0, permute_seed=4)
    st = W.BoostedKS(M=1.0, c0=(3.0, 0.5, -0.2), vel=(0.0, 0.3, 0.0))
    U, G = _ks_state(cfg, st)
    _, gp = _gpu_psi4(cfg, U, G, centre)
    og = O.Grid(cfg.p, cfg.np, cfg.ijk(), cfg.origin, cfg.dx, cfg.bc)
    op = og.psi4(U, G, centre)
    assert np.abs(op).max() > 0.05
    assert _rel(gp, op) < 1e-10


def test_psi4_matches_oracle_on_perturbed_puncture_data_and_a_mesh():
    cfg = I.single_puncture_config(p=6, n_side=3, half_width=1.5, permute_seed=2)
    U, G = I.initial_state(cfg)
    x, y, z = I.point_coords(cfg.p, cfg.ijk(), cfg.origin, cfg.dx)
    U = I.smooth_perturbation(x, y, z, seed=5, amp=1e-2, box=3.0, base=U)
    _, gp = _gpu_psi4(cfg, U, G, (0.05, 0.1, -0.1))
    op = O.Grid(cfg.p, cfg.np, cfg.ijk(), cfg.origin, cfg.dx, cfg.bc).psi4(U, G, (0.05, 0.1, -0.1))
    far = np.sqrt(x * x + y * y + z * z) > 0.5        # psi_4 of the perturbed puncture is huge at the puncture
    assert _rel(gp[:, far], op[:, far]) < 1e-10
    mcfg = I.multilevel_puncture_config(p=6, n_side=4, half_width=2.0, boxes=[((1, 1, 1), (3, 3, 3))])
    x, y, z = I.mesh_point_coords(mcfg.p, mcfg.level, mcfg.ijk(), mcfg.origin, mcfg.dx)
    st = W.BoostedKS(M=1.0, c0=(4.0, 0.5, -0.2), vel=(0.2, 0.1, 0.0))
    gx, gy, gz = I.ghost_positions(mcfg.N, mcfg.origin, mcfg.dx)
    U, G = W.ccz4_state(st, x, y, z), W.ccz4_state(st, gx, gy, gz)
    _, gp = _gpu_psi4(mcfg, U, G, (0.0, 0.0, 0.0))
    og = O.Grid(mcfg.p, mcfg.np, mcfg.ijk(), mcfg.origin, mcfg.dx, mcfg.bc, level=mcfg.level)
    op = og.psi4(U, G)
    assert _rel(gp, op) < 1e-10


def test_extraction_on_a_sphere_matches_the_oracle_and_the_weyl_tensor():
    from paper_2406_11626_gb300 import psi4 as P
    cfg = I.single_puncture_config(p=6, n_side=6, half_width=1.5)
    st = W.BoostedKS(M=1.0, c0=(3.5, 0.5, -0.2), vel=(0.0, 0.3, 0.0))
    U, G = _ks_state(cfg, st)
    from paper_2406_11626_gb300 import ccz4 as C
    g = C.Grid.from_config(cfg)
    g.upload(U, G)
    nt, nphi = 8, 16
    got, vals = P.extract(g, 0.9, n_theta=nt, n_phi=nphi, lmax=4)
    # the oracle: its psi_4 in fields 0 and 1, sampled by its tracer projection
    og = O.Grid(cfg.p, cfg.np, cfg.ijk(), cfg.origin, cfg.dx, cfg.bc)
    op = og.psi4(U, G)
    S = np.zeros_like(U)
    S[0], S[1] = op[0], op[1]
    pos, th, ph, w = P.sphere(0.9, nt, nphi)
    _, ov, bad = og.tracers_step(S, np.zeros_like(G), pos, 0.0, -1, 0.0)
    assert bad == 0
    ovals = ov[:, 0] + 1j * ov[:, 1]
    assert _rel(vals, ovals) < 1e-10
    want = P.modes(ovals, th, ph, w, lmax=4)
    for k in got:
        assert abs(got[k] - want[k]) <= 1e-10 * max(abs(v) for v in want.values()), k
    # against the Weyl tensor itself at the sphere points: the trilinear
    # projection is second order, and the tetrad turns fast near the z axis
    # (v = (-y, x, 0)), so points near the poles carry the largest error
    # (measured on the oracle's sampling at this spacing, dx = 1/12: 1.6 % of
    # max |psi_4| for sin(theta) > 0.5, 5.7 % at all points, 1.3 % in the modes;
    # 0.5 %, 1.3 % and 0.35 % at dx = 1/24)
    ref, _ = W.psi4(st, pos)
    eq = np.sin(th) > 0.5
    assert _rel(vals[eq], ref[eq]) * np.abs(ref[eq]).max() / np.abs(ref).max() < 2.5e-2
    rm = P.modes(ref, th, ph, w, lmax=4)
    scale = max(abs(v) for v in rm.values())
    assert scale > 1e-3
    assert max(abs(got[k] - rm[k]) for k in rm) < 2.5e-2 * scale


def test_invalid_psi4_arguments_are_refused():
    from paper_2406_11626_gb300 import ccz4 as C
    cfg = I.single_puncture_config(p=6, n_side=2, half_width=1.0)
    g = C.Grid.from_config(cfg)
    with pytest.raises(C.CCZ4Error):
        g.psi4("U", "U")
    with pytest.raises(C.CCZ4Error):
        g.psi4("U", "TILE")
    with pytest.raises(C.CCZ4Error):
        g.psi4("U", "RHS", (np.nan, 0.0, 0.0))
