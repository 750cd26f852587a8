"""The patch-edge autotuner: candidate layouts, choice and JSON cache (host
logic with a fake timer), and one small sweep on the GPU."""
import json

import pytest

from paper_2406_11626_gb300 import autotune as A


def test_layouts_match_the_target_size():
    lay = dict(A.layouts(144))
    assert lay == {6: 24, 9: 16, 12: 12, 17: 8, 18: 8}
    assert all(p <= 18 for p, _ in A.layouts(100, candidates=(6, 19, 25)))


def test_tune_picks_the_fastest_and_caches(tmp_path):
    calls = []

    def fake(p, n_side, h, precision, steps, warmup, launch):
        calls.append(p)
        pts = (p * n_side) ** 3
        # a cost model with a minimum at p = 12, the queue launch 1 % faster
        return pts * (1.0 + (p - 12) ** 2 / 50.0) * (0.99 if launch == "queue" else 1.0) * 1e-9, pts

    cache = str(tmp_path / "tune.json")
    r = A.tune(144, timer=fake, key_extra="fake-gpu", cache=cache)
    assert r["p"] == 12 and r["n_side"] == 12 and r["launch"] == "queue"
    assert sorted(calls) == [6, 6, 9, 9, 12, 12, 17, 17, 18, 18]
    r2 = A.tune(144, timer=fake, key_extra="fake-gpu", cache=cache)
    assert r2 == r and len(calls) == 10         # served from the cache
    A.tune(144, timer=fake, key_extra="fake-gpu", cache=cache, refresh=True)
    assert len(calls) == 20
    A.tune(144, timer=fake, key_extra="other-gpu", cache=cache)
    assert len(json.load(open(cache))) == 2     # one entry per key


@pytest.mark.gpu
def test_tune_on_the_gpu(tmp_path):
    import torch
    assert torch.cuda.is_available()
    r = A.tune(36, steps=1, warmup=1, cache=str(tmp_path / "t.json"))
    assert r["p"] in A.CANDIDATES and r["launch"] in A.LAUNCHES
    assert all(v["point_stages_per_s"] > 0 for v in r["results"].values())
