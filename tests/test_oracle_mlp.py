"""Pins of the warm-start network oracle: back-propagated gradients against
central finite differences, the SiLU derivative, the first Adam step's
closed form, and a fit that the update actually reduces the loss."""
import numpy as np

from oracle import mlp as M


def _setup(seed=0, n_in=8, width=16, depth=3, batch=12):
    rng = np.random.default_rng(seed)
    theta = rng.standard_normal(M.n_params(n_in, width, depth)) * 0.3
    X = rng.standard_normal((batch, n_in))
    T = rng.standard_normal(batch)
    return theta, X, T, dict(n_in=n_in, width=width, depth=depth)


def test_layout_counts_every_parameter():
    assert M.n_params() == 8 * 128 + 128 + 3 * (128 * 128 + 128) + 128 + 1
    theta = np.arange(M.n_params(8, 4, 2), dtype=float)
    (W0, b0), (W1, b1), (W2, b2) = M.unpack(theta, 8, 4, 2)
    assert W0.shape == (4, 8) and W1.shape == (4, 4) and W2.shape == (1, 4)
    assert W0[0, 0] == 0 and b0[0] == 32 and W1[0, 0] == 36 and b2[0] == theta[-1]


def test_silu_derivative_matches_finite_differences():
    z = np.linspace(-6, 6, 101)
    h = 1e-6
    fd = (M.silu(z + h) - M.silu(z - h)) / (2 * h)
    np.testing.assert_allclose(M.silu_prime(z), fd, rtol=1e-8, atol=1e-10)
    assert M.silu(0.0) == 0.0 and abs(M.silu(30.0) - 30.0) < 1e-10


def test_gradient_matches_central_differences():
    theta, X, T, kw = _setup()
    L, g = M.gradient(theta, X, T, **kw)
    assert L == M.loss(theta, X, T, **kw)
    rng = np.random.default_rng(1)
    idx = rng.choice(len(theta), 60, replace=False)
    h = 1e-6
    for k in idx:
        e = np.zeros_like(theta)
        e[k] = h
        fd = (M.loss(theta + e, X, T, **kw) - M.loss(theta - e, X, T, **kw)) / (2 * h)
        assert abs(g[k] - fd) <= 1e-7 * max(1.0, abs(fd)), (k, g[k], fd)


def test_first_adam_step_moves_each_parameter_by_lr():
    """At step 1 the bias-corrected ratio is g / (|g| + eps): every parameter
    with a gradient well above eps moves by lr against its sign."""
    theta, X, T, kw = _setup(2)
    _, g = M.gradient(theta, X, T, **kw)
    lr = 1e-3
    t1, m, v = M.adam(theta, np.zeros_like(theta), np.zeros_like(theta), g, 1, lr)
    big = np.abs(g) > 1e-4
    np.testing.assert_allclose((theta - t1)[big], lr * np.sign(g[big]), rtol=1e-4)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_adam_reduces_the_loss_on_a_smooth_target():
    rng = np.random.default_rng(3)
    kw = dict(n_in=2, width=16, depth=2)
    theta = rng.standard_normal(M.n_params(**kw)) * 0.3
    X = rng.uniform(-1, 1, (256, 2))
    T = np.sin(2 * X[:, 0]) * X[:, 1]
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    L0 = M.loss(theta, X, T, **kw)
    for k in range(1, 401):
        _, g = M.gradient(theta, X, T, **kw)
        theta, m, v = M.adam(theta, m, v, g, k, 1e-2)
    assert M.loss(theta, X, T, **kw) < 0.1 * L0
