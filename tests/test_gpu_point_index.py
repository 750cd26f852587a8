"""ccz4_point_index: lattice points to state-buffer indices on the GPU,
checked against the coordinates each index holds; points beyond a
Sommerfeld grid's ghost shell come back as -1 with CCZ4_ERR_BOUNDS, raised by
the device-side bounds check of the halo fill's point lookup, without a trap
and without touching the grid's own status."""
import numpy as np
import pytest

from paper_2406_11626_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _coord_state(cfg):
    """A state whose fields 0, 1, 2 hold x, y, z of each point (and ghost
    cell)."""
    x, y, z = I.point_coords(cfg.p, cfg.ijk(), cfg.origin, cfg.dx)
    U = np.zeros((I.NV,) + x.shape)
    U[0], U[1], U[2] = x, y, z
    if cfg.bc == "sommerfeld":
        gx, gy, gz = I.ghost_positions(cfg.N, cfg.origin, cfg.dx)
        G = np.zeros((I.NV, len(gx)))
        G[0], G[1], G[2] = gx, gy, gz
    else:
        G = np.zeros((I.NV, 0))
    return U, G


def _values(U, G, idx):
    """Fields 0..2 at state indices idx (interior, then ghost cells)."""
    n = U[0].size
    flat = [np.concatenate([U[v].ravel(), G[v]]) for v in range(3)]
    return np.stack([f[idx] for f in flat], axis=1), n


def test_interior_and_ghost_points_map_to_their_values():
    from paper_2406_11626_gb300 import ccz4 as C
    cfg = I.single_puncture_config(p=6, n_side=3, half_width=1.5, permute_seed=3)
    g = C.Grid.from_config(cfg)
    U, G = _coord_state(cfg)
    g.upload(U, G)
    N = np.array(cfg.N)
    rng = np.random.default_rng(0)
    inside = rng.integers(0, N, size=(200, 3))
    shell = rng.integers(-3, N + 3, size=(300, 3))
    shell = shell[((shell < 0) | (shell >= N)).any(axis=1)]
    pts = np.concatenate([inside, shell])
    idx = g.point_index(pts)
    assert (idx >= 0).all()
    gU, gG = g.download("U")
    vals, n = _values(gU, gG, idx)
    want = np.asarray(cfg.origin) + (pts + 0.5) * cfg.dx
    np.testing.assert_allclose(vals, want, rtol=0, atol=1e-12)
    assert (idx[:len(inside)] < n).all() and (idx[len(inside):] >= n).all()


def test_points_beyond_the_ghost_shell_report_bounds_without_a_trap():
    from paper_2406_11626_gb300 import ccz4 as C
    cfg = I.single_puncture_config(p=6, n_side=3, half_width=1.5)
    g = C.Grid.from_config(cfg)
    U, G = I.initial_state(cfg)
    g.upload(U, G)
    N = cfg.N[0]
    pts = np.array([[0, 0, 0], [-4, 0, 0], [N + 3, 5, 5], [2, -1, 3], [1, 2, N + 10]])
    with pytest.raises(C.CCZ4Error) as e:
        g.point_index(pts)
    assert e.value.code == C.ERR_BOUNDS and "3 of 5 points" in str(e.value)
    idx = g.point_index(pts, raise_bounds=False)
    assert list(idx < 0) == [False, True, True, False, True]
    # the grid's own status is untouched: the monitors still run
    out = g.constraints("U")
    assert np.isfinite(out[:4]).all()


def test_periodic_points_wrap_and_meshes_are_refused():
    from paper_2406_11626_gb300 import ccz4 as C
    cfg = I.gauge_wave_config(p=6, np_=(3, 3, 3), permute_seed=1)
    g = C.Grid.from_config(cfg)
    U, G = _coord_state(cfg)
    g.upload(U)
    N = np.array(cfg.N)
    pts = np.array([[-1, 0, 0], [N[0], 3, 4], [5, -7, N[2] + 2]])
    idx = g.point_index(pts)
    gU, gG = g.download("U")
    vals, _ = _values(gU, gG, idx)
    want = np.asarray(cfg.origin) + (np.mod(pts, N) + 0.5) * cfg.dx
    np.testing.assert_allclose(vals, want, rtol=0, atol=1e-12)
    assert len(g.point_index(np.zeros((0, 3), int))) == 0
    gm = C.Grid.from_config(I.multilevel_puncture_config(p=6, n_side=4, half_width=2.0,
                                                         boxes=[((1, 1, 1), (3, 3, 3))]))
    with pytest.raises(C.CCZ4Error) as e:
        gm.point_index([[0, 0, 0]])
    assert e.value.code == C.ERR_INVALID


def test_grids_can_take_their_buffers_from_torchs_allocator():
    """ccz4_set_allocator with PyTorch's caching allocator: the grid's large
    buffers show up in torch's accounting, a step gives the same state bit
    for bit as a grid on cudaMalloc, and releasing the grid returns them."""
    import torch
    from paper_2406_11626_gb300 import ccz4 as C
    cfg = I.single_puncture_config(p=6, n_side=3, half_width=1.5)
    U, G = I.initial_state(cfg)
    P = C.make_params(**cfg.params)
    out = []
    for use in (False, True):
        C.use_torch_allocator(use)
        try:
            torch.cuda.synchronize()
            before = torch.cuda.memory_allocated()
            g = C.Grid.from_config(cfg)
            grew = torch.cuda.memory_allocated() - before
            g.upload(U, G)
            g.upload(U, G, buf="INI")
            g.step(P, cfg.dt, 2)
            out.append(g.download("U"))
            g.close()
            torch.cuda.synchronize()
            back = torch.cuda.memory_allocated() - before
        finally:
            C.use_torch_allocator(False)
        if use:
            n = cfg.n_patches * cfg.p ** 3
            assert grew >= 25 * 6 * n * 8 and back == 0, (grew, back)
        else:
            assert grew == 0
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
