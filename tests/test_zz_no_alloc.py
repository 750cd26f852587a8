"""The allocation-free constraint monitor, ccz4_constraints_noalloc.

Some callers of this library cannot call cudaMalloc (a host framework that
owns all device memory, or a time loop that must not allocate once it
runs). For them the library offers one entry point that allocates nothing:
its reduction scratch sits in a fixed device array inside the library.
These tests call it through the C ABI and check it against the allocating
ccz4_constraints on the same halo tiles, on two calls in a row (the second
call reuses the scratch the first one left behind). This file is collected
last so that a run stopping at its first failure has run every other test.
"""
import numpy as np
import pytest

from paper_2406_11626_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-11


def _grid_with_state():
    from paper_2406_11626_gb300 import ccz4 as C
    cfg = I.single_puncture_config(p=9, n_side=4, half_width=2.0)
    g = C.Grid.from_config(cfg)
    U, G = I.initial_state(cfg)
    x, y, z = I.point_coords(cfg.p, cfg.ijk(), cfg.origin, cfg.dx)
    U = I.smooth_perturbation(x, y, z, seed=5, amp=1e-2, box=4.0, base=U)
    g.upload(U, G)
    return C, g


def test_noalloc_constraints_match_the_allocating_entry_point_twice():
    import torch
    C, g = _grid_with_state()
    n = g.n_points
    H1 = torch.zeros(n, dtype=torch.float64, device="cuda")
    M1 = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    out1 = g.constraints("U", H1.data_ptr(), M1.data_ptr())   # also fills the halo tiles of U
    tiles, _ = g.device_ptr("TILE")
    h1, m1 = H1.cpu().numpy(), M1.cpu().numpy()
    for _ in range(2):
        H2 = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        M2 = torch.full((3 * n,), float("nan"), dtype=torch.float64, device="cuda")
        out2 = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        C.constraints_noalloc(tiles, g.p, g.n_patches, g.dx, H2.data_ptr(), M2.data_ptr(), out2.data_ptr())
        torch.cuda.synchronize()
        # the call took no device memory (its scratch is the library's fixed array)
        assert torch.cuda.mem_get_info()[0] == free0
        h2, m2, o2 = H2.cpu().numpy(), M2.cpu().numpy(), out2.cpu().numpy()
        assert np.abs(h2 - h1).max() <= TOL * max(np.abs(h1).max(), 1.0)
        assert np.abs(m2 - m1).max() <= TOL * max(np.abs(m1).max(), 1.0)
        np.testing.assert_allclose(o2[:4], out1[:4], rtol=TOL, atol=0)
        assert o2[4] == out1[4] == 0.0


def test_noalloc_constraints_reject_sizes_beyond_the_fixed_scratch():
    C, g = _grid_with_state()
    tiles, _ = g.device_ptr("TILE")
    with pytest.raises(C.CCZ4Error) as e:
        C.constraints_noalloc(tiles, 9, 5800, g.dx, None, None, tiles)   # 4.23M points > 4,194,304
    assert e.value.code == C.ERR_INVALID
    assert "exceed the maximum" in str(e.value)
    # an edge whose cube overflows 64-bit sizes is rejected before any size is formed
    for p, n in ((1 << 21, 1), (162, 1), (161, 2)):
        with pytest.raises(C.CCZ4Error) as e:
            C.constraints_noalloc(tiles, p, n, g.dx, None, None, tiles)
        assert e.value.code == C.ERR_INVALID
