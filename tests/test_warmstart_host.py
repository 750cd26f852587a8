"""Host logic of the learned warm start: the learning-rate schedule, the
Sobol draws of the binary parameters and the model-problem relaxation
factor (no GPU)."""
import math

import numpy as np

from paper_2406_11626_gb300 import warmstart as W


def test_cosine_schedule_runs_from_lr_to_lr_final():
    lr, lo, steps = 1e-3, 1e-5, 101
    r = [W.lr_at(k, steps, lr, lo) for k in range(steps)]
    assert r[0] == lr and abs(r[-1] - lo) < 1e-18
    assert abs(r[50] - 0.5 * (lr + lo)) < 1e-15          # half-way: the mean
    assert all(a >= b for a, b in zip(r, r[1:]))          # non-increasing
    assert W.lr_at(7, steps, lr) == lr                    # no lr_final: constant


def test_sobol_draws_cover_the_parameter_box():
    d = W.sobol_draws(256, seed=0)
    assert d.shape == (256, 5)
    for c, (lo, hi) in enumerate(W.RANGES):
        assert d[:, c].min() >= lo and d[:, c].max() <= hi
        # a low-discrepancy set fills each axis evenly: every eighth of the range is hit
        assert len(np.unique(np.floor((d[:, c] - lo) / (hi - lo) * 8).clip(0, 7))) == 8
    assert np.array_equal(d, W.sobol_draws(256, seed=0))  # seeded


def test_optimal_omega_is_youngs_formula():
    # rho = cos(pi/n): 2 / (1 + sqrt(1 - rho^2)) = 2 / (1 + sin(pi/n))
    for n in (8, 96, 192):
        rho = math.cos(math.pi / n)
        assert abs(W.optimal_omega(n) - 2.0 / (1.0 + math.sqrt(1.0 - rho * rho))) < 1e-12
    assert 1.0 < W.optimal_omega(96) < 2.0
