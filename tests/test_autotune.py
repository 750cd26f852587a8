"""The autotuner: candidate layouts, the coordinate descent over patch edge,
launch and launch shapes, the per-workload JSON cache (host logic with a
fake timer), and one small sweep on the GPU."""
import json

import pytest

from paper_2406_11626_gb300 import autotune as A


def test_layouts_match_the_target_size():
    lay = dict(A.layouts(144))
    assert lay == {6: 24, 9: 16, 12: 12, 17: 8, 18: 8}
    assert all(p <= 18 for p, _ in A.layouts(100, candidates=(6, 19, 25)))


def test_workload_configurations():
    uni = A.workload_configs("puncture144")
    assert sorted(c.p for c in uni) == [6, 9, 12, 17, 18]
    assert all(abs(c.dx - 1.0 / 9.0) < 1e-15 for c in uni)
    m3, = A.workload_configs("puncture3level")
    bi, = A.workload_configs("binary")
    assert m3.n_levels == 3 and bi.n_levels == 4 and m3.p == bi.p == 9
    U, G = A.timing_state(bi)      # closed-form data on the binary mesh, no solve needed
    assert U.shape[1] == bi.n_patches and G.shape[1] > 0
    with pytest.raises(ValueError):
        A.workload_configs("nope")


def _fake(calls):
    def fake(cfg, precision, steps, warmup, launch, stage_shape, fill_shape):
        calls.append((cfg.p, launch, stage_shape, fill_shape))
        pts = cfg.n_points
        # a cost model with a minimum at p = 12, the queue launch 1 % faster, stage shape 2 3 % faster,
        # fill shape 1 2 % faster (on the flat launch only for the stage shape)
        c = 1.0 + (cfg.p - 12) ** 2 / 50.0
        c *= 0.99 if launch == "queue" else 1.0
        c *= 0.97 if stage_shape == 2 else 1.0
        c *= 0.98 if fill_shape == 1 else 1.0
        return pts * c * 1e-9, pts
    return fake


def test_tune_descends_each_coordinate_and_caches(tmp_path):
    calls = []
    cache = str(tmp_path / "tune.json")
    r = A.tune("puncture144", timer=_fake(calls), key_extra="fake-gpu", cache=cache)
    # the queue launch wins the first coordinate, so the stage shape (a flat-launch knob) is not swept
    assert (r["p"], r["launch"], r["stage_shape"], r["fill_shape"]) == (12, "queue", 0, 1)
    # 5 edges x flat and queue, the fused launch at p = 9 only, then 3 more fill shapes
    assert len(calls) == 11 + 3
    assert sum(1 for c in calls if c[1] == "fused") == 1 and (9, "fused", 0, 0) in calls
    assert A.tune("puncture144", timer=_fake(calls), key_extra="fake-gpu", cache=cache) == r
    assert len(calls) == 14         # served from the cache
    r2 = A.tune("puncture144", timer=_fake(calls), key_extra="fake-gpu", cache=cache, launches=("flat",))
    assert (r2["p"], r2["launch"], r2["stage_shape"], r2["fill_shape"]) == (12, "flat", 2, 1)
    assert len(calls) == 14 + 5 + 3 + 3     # 5 edges, 3 more stage shapes, 3 more fill shapes
    A.tune("puncture144", timer=_fake(calls), key_extra="fake-gpu", cache=cache, refresh=True)
    assert len(calls) == 25 + 14
    assert len(json.load(open(cache))) == 2     # one entry per key


def test_tune_fused_launch_sweeps_no_shapes(tmp_path):
    calls = []

    def fake(cfg, precision, steps, warmup, launch, stage_shape, fill_shape):
        calls.append((cfg.p, launch, stage_shape, fill_shape))
        c = 0.7 if launch == "fused" else 1.0
        return cfg.n_points * c * 1e-9, cfg.n_points

    r = A.tune("puncture144", timer=fake, key_extra="fake-gpu", cache=str(tmp_path / "t.json"))
    # the fused launch wins at p = 9; it has its own shapes, so none is swept after it
    assert (r["p"], r["launch"], r["stage_shape"], r["fill_shape"]) == (9, "fused", 0, 0)
    assert len(calls) == 11


def test_compare_times_each_launch_in_turn():
    calls = []
    row = A.compare("puncture144", "mixed", ("flat", "fused"), steps=4, warmup=1, repeats=2, timer=_fake(calls))
    assert [c[1] for c in calls] == ["flat", "fused", "flat", "fused"]
    assert all(c[0] == 9 and c[2:] == (0, 0) for c in calls)
    assert row["p"] == 9 and row["points"] == 144 ** 3 and len(row["flat"]) == len(row["fused"]) == 2


def test_mesh_workloads_keep_their_patch_edge(tmp_path):
    calls = []
    for w in ("puncture3level", "binary"):
        r = A.tune(w, "mixed", timer=_fake(calls), key_extra="fake-gpu", cache=str(tmp_path / "t.json"),
                   launches=("flat",))
        assert r["p"] == 9 and r["stage_shape"] == 2 and r["fill_shape"] == 1 and r["workload"] == w
    assert {c[0] for c in calls} == {9}
    assert len(json.load(open(str(tmp_path / "t.json")))) == 2


@pytest.mark.gpu
def test_tune_on_the_gpu(tmp_path):
    import torch
    assert torch.cuda.is_available()
    r = A.tune("puncture144", n_target=36, steps=1, warmup=1, cache=str(tmp_path / "t.json"))
    assert r["p"] in A.CANDIDATES and r["launch"] in A.LAUNCHES
    assert r["stage_shape"] in A.STAGE_SHAPES and r["fill_shape"] in A.FILL_SHAPES
    assert all(v["point_stages_per_s"] > 0 for v in r["results"].values())


@pytest.mark.gpu
@pytest.mark.parametrize("stage_shape,fill_shape", [(1, 1), (2, 2), (0, 3), (3, 0)])
def test_launch_shapes_give_identical_steps(stage_shape, fill_shape):
    """Every launch shape computes the same step bit for bit (FP64 and
    mixed, single level and mesh), except the mixed path's two-phase shape:
    it evaluates the same expressions from parked stencil values, but its
    compiled FP32 algebra may round a few intermediate values differently
    (seen in the Gamma-hat^x and b^x updates of a few points), so it is held
    to 1e-8 of each field's largest value, below the mixed path's own
    distance from the FP64 path."""
    import numpy as np
    from paper_2406_11626_gb300 import ccz4 as C
    from paper_2406_11626_gb300 import inputs as I
    for cfg in (I.single_puncture_config(p=6, n_side=3, half_width=1.5),
                I.multilevel_puncture_config(p=6, n_side=4, half_width=2.0, boxes=[((1, 1, 1), (3, 3, 3))])):
        U, G = I.initial_state(cfg)
        for prec in ("fp64", "mixed"):
            out = []
            for shapes in ((0, 0), (stage_shape, fill_shape)):
                g = C.Grid.from_config(cfg)
                g.set_tuning(*shapes)
                g.upload(U, G)
                g.upload(U, G, buf="INI")
                g.step_graph(C.make_params(**cfg.params, precision=prec), cfg.dt, 2)
                out.append(g.download("U"))
                g.close()
            if prec == "mixed" and stage_shape == 3:
                for a, b in zip(out[1], out[0]):
                    scale = np.abs(b).max(axis=tuple(range(1, b.ndim)), keepdims=True)
                    assert (np.abs(a - b) <= 1e-8 * np.maximum(scale, 1e-30)).all()
            else:
                assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    g = C.Grid.from_config(I.single_puncture_config(p=6, n_side=2, half_width=1.0))
    with pytest.raises(C.CCZ4Error):
        g.set_tuning(4, 0)
