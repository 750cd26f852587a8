"""Host logic of refined meshes in the CUDA library, checked on the CPU:
ccz4_mesh_plan validates a mesh and resolves every halo'd tile point into a
state index or a coarse-to-fine interpolation entry. Gathering tiles from
that plan (weights and order as the header documents them) must reproduce
the oracle's halo fill bit for bit."""
import numpy as np
import pytest

import oracle as O
from paper_2406_11626_gb300 import ccz4 as C
from paper_2406_11626_gb300 import inputs as I

PW = np.array([[1.0, 0.0], [2.0 / 3.0, 1.0 / 3.0], [1.0 / 3.0, 2.0 / 3.0]])


def _gather(state, src, interp):
    """Tiles (NV, n_patches, T3) from a state (NV, n_points + n_ghost) and a plan."""
    out = np.empty((state.shape[0],) + src.shape)
    direct = src >= 0
    out[:, direct] = state[:, src[direct]]
    assert (src[~direct] <= -2).all()
    e = interp[-src[~direct] - 2]
    q = state[:, e[:, :8]]                      # (NV, n, 8): corners (z, y, x), x fastest
    r = e[:, 8]
    rx, ry, rz = r & 3, (r >> 2) & 3, (r >> 4) & 3

    def lerp(rr, a, b):
        # x, then y, then z; a weight of one takes the single value
        return np.where(rr != 0, PW[rr, 0] * a + PW[rr, 1] * b, a)
    t = [[lerp(rx, q[:, :, (c * 2 + b) * 2], q[:, :, (c * 2 + b) * 2 + 1]) for b in range(2)] for c in range(2)]
    u = [lerp(ry, t[c][0], t[c][1]) for c in range(2)]
    out[:, ~direct] = lerp(rz, u[0], u[1])
    return out


MESHES = [
    (6, (4, 4, 4), [((1, 1, 1), (3, 3, 3))]),
    (6, (4, 4, 4), [((1, 1, 1), (3, 3, 3)), ((5, 5, 5), (7, 7, 7))]),
    (2, (4, 4, 4), [((1, 1, 1), (3, 3, 3))]),
    (9, (3, 3, 3), [((1, 1, 1), (2, 2, 2))]),
    (3, (5, 4, 4), [((1, 1, 1), (4, 3, 3)), ((4, 4, 4), (6, 5, 5))]),
]


@pytest.mark.parametrize("mesh,bc", [(0, "periodic"), (0, "copy"), (0, "sommerfeld"), (1, "sommerfeld"),
                                     (2, "copy"), (3, "periodic"), (4, "sommerfeld")])
def test_tiles_from_the_plan_equal_the_oracle_fill(mesh, bc):
    p, np_, boxes = MESHES[mesh]
    lev, ijk = I.refined_mesh(np_, boxes, permute_seed=mesh)
    # shuffle the patch order across levels: nothing may rely on it
    perm = np.random.default_rng(mesh).permutation(len(lev))
    lev, ijk = lev[perm], ijk[perm]
    origin, dx = (-0.4, 0.3, -0.1), 0.2
    og = O.Grid(p, np_, ijk, origin, dx, bc, level=lev)
    src, interp = C.mesh_plan(p, np_, lev, ijk, origin, dx, bc)
    rng = np.random.default_rng(7)
    U = rng.standard_normal(og.ushape)
    G = rng.standard_normal((I.NV, og.n_ghost))
    state = np.concatenate([U.reshape(I.NV, -1), G], axis=1)
    tiles = _gather(state, src, interp).reshape((I.NV, len(lev)) + (p + 6,) * 3)
    np.testing.assert_array_equal(tiles, og.fill_tiles(U, G))
    if len(boxes) and mesh != 2:
        assert len(interp) > 0


def test_invalid_meshes_are_rejected_on_the_host():
    ok = I.refined_mesh((4, 4, 4), [((1, 1, 1), (3, 3, 3))])
    C.mesh_plan(6, (4, 4, 4), *ok, (0, 0, 0), 0.1, "copy")
    bad = []
    for boxes in ([((0, 1, 1), (2, 3, 3))], [((1, 1, 1), (4, 3, 3))],
                  [((1, 1, 1), (3, 3, 3)), ((3, 4, 4), (4, 5, 5))]):
        bad.append(I.refined_mesh((4, 4, 4), boxes))
    lev, ijk = ok
    keep = np.ones(len(lev), bool)
    keep[np.nonzero(lev == 1)[0][5]] = False
    bad.append((lev[keep], ijk[keep]))                 # incomplete child set
    bad.append((np.where(lev == 1, 9, lev), ijk))      # level out of range
    dup = ijk.copy()
    dup[1] = dup[0]
    bad.append((lev, dup))                             # level-0 slot twice
    orphan_l, orphan_i = lev.copy(), ijk.copy()
    orphan_i[lev == 1] += 9                            # children without parents
    bad.append((orphan_l, orphan_i))
    for lv, ij in bad:
        with pytest.raises(C.CCZ4Error) as e:
            C.mesh_plan(6, (4, 4, 4), lv, ij, (0, 0, 0), 0.1, "copy")
        assert e.value.code == C.ERR_INVALID
    with pytest.raises(C.CCZ4Error):
        C.mesh_plan(19, (4, 4, 4), *ok, (0, 0, 0), 0.1, "copy")  # p above the limit


def test_three_level_puncture_plan():
    """The three-level puncture workload plans (and its level-2 halos
    interpolate from level 1)."""
    cfg = I.multilevel_puncture_config()
    src, interp = C.mesh_plan(cfg.p, cfg.np, cfg.level, cfg.ijk(), cfg.origin, cfg.dx, cfg.bc)
    assert src.shape == (7552, 15 ** 3)
    assert len(interp) > 0
    assert (src >= -1 - len(interp)).all()
