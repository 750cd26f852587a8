"""The evolution driver: its workload table and argument checks on the
host, and a short run on the GPU whose constraint reports are complete and
stay at the level of the exact gauge-wave solution."""
import pytest

from paper_2406_11626_gb300 import evolve as E


def test_workloads_build_their_configurations():
    names = {k: E.WORKLOADS[k]().name for k in ("gauge_wave", "puncture144", "mid", "binary")}
    assert names["gauge_wave"] == "gauge_wave" and names["binary"] == "binary_puncture"
    assert E.WORKLOADS["mesh-mid"]().n_patches == 2240


def test_invalid_arguments_are_rejected_before_any_work():
    with pytest.raises(ValueError):
        E.run("gauge_wave", steps=4, every=0)
    with pytest.raises(ValueError):
        E.run("gauge_wave", steps=-1, every=1)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_short_gauge_wave_run_reports_every_interval(precision):
    reps = E.run("gauge_wave", steps=6, every=4, precision=precision)
    assert [r["step"] for r in reps] == [0, 4, 6]
    assert all(r["nonfinite"] == 0 for r in reps)
    # the printed gauge wave is an exact solution: H stays at the truncation level
    assert all(r["L2_H"] < 1e-3 for r in reps)
    assert reps[-1]["time"] > 0 and reps[-1]["wall_s"] > 0


def test_puncture_positions_of_the_workloads():
    assert E.puncture_positions(E.WORKLOADS["binary"]()) == [(-3.0, 0.0, 0.0), (3.0, 0.0, 0.0)]
    assert E.puncture_positions(E.WORKLOADS["mid"]()) == [(0.0, 0.0, 0.0)]
    assert E.puncture_positions(E.WORKLOADS["gauge_wave"]()) == []


@pytest.mark.gpu
def test_puncture_tracker_follows_the_opposite_shift_on_a_mesh():
    """A short three-level run with the tracker: the single puncture at the
    origin stays there (the data are symmetric under x -> -x, y -> -y,
    z -> -z, so the projected shift vanishes there), and every report
    carries the tracker's position."""
    reps = E.run("mesh-mid", steps=4, every=2, track=True)
    assert [r["step"] for r in reps] == [0, 2, 4]
    assert all(len(r["punctures"]) == 1 for r in reps)
    assert max(abs(c) for c in reps[-1]["punctures"][0]) < 1e-12


@pytest.mark.parametrize("box,want_near,n_kids", [(((1, 1, 1), (2, 2, 2)), 27 ** 3 - 21 ** 3, 27),
                                                   (((1, 1, 1), (3, 2, 2)), 54 * 27 * 27 - 48 * 21 * 21, 54)])
def test_interface_mask_marks_the_three_points_next_to_a_refined_block(box, want_near, n_kids):
    """A block of refined patches (one parent's 27 children, or two
    parents' 54) inside a 4^3 level-0 grid of 9^3 patches: the points of the
    block within three points of its outer faces reach interpolated halo
    points (the block's point count less its core shrunk by three on every
    side); the refined parents are not leaves; level 0 has no interface."""
    import numpy as np
    from paper_2406_11626_gb300 import inputs as I
    cfg = I.multilevel_puncture_config(p=9, n_side=4, half_width=2.0, boxes=[box])
    leaf, near = E.interface_mask(cfg)
    assert near.sum() == want_near
    lev = np.asarray(cfg.level)
    assert (lev == 1).sum() == n_kids
    assert not near[lev == 0].any() and (~leaf).sum() == (n_kids // 27) * 729
    assert leaf[lev == 1].all()
    # the split of a norm: H = 1 near the interface, 0 elsewhere
    H = near.astype(float)
    out = E.interface_split(cfg, H, (leaf, near), centres=[(0.0, 0.0, 0.0)], radius=0.5)
    assert out["L2_H_cf"] == 1.0 and out["L2_H_off_cf"] == 0.0 and out["L2_H_off_cf_r1"] == 0.0
    assert out["points_cf"] + out["points_off_cf"] == leaf.sum()


def test_a_single_level_has_no_interface():
    from paper_2406_11626_gb300 import inputs as I
    leaf, near = E.interface_mask(I.single_puncture_config(p=6, n_side=3, half_width=1.5))
    assert leaf.all() and not near.any()
