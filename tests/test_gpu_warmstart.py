"""The learned warm start on the GPU (include/ccz4_mlp.h): forward pass,
back-propagated gradients and Adam against the FP64 oracle, the feature
kernels, and the gain of a trained network over the plain solve from u = 0
on held-out draws (the plain solve decides both)."""
import numpy as np
import pytest

from oracle import mlp as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available()


def _net(width=128, depth=4, seed=0, max_batch=4096):
    from paper_2406_11626_gb300 import warmstart as W
    net = W.MLP(8, width, depth, max_batch)
    theta = W.init_params(8, width, depth, seed)
    net.set_params(theta)
    return net, theta.astype(np.float64)


def test_forward_matches_the_oracle():
    import torch
    net, theta = _net()
    rng = np.random.default_rng(0)
    X = rng.standard_normal((3000, 8)).astype(np.float32)
    y = net.forward(torch.as_tensor(X, device="cuda")).cpu().numpy()
    yo, _ = M.forward(theta, X.astype(np.float64))
    assert np.abs(y - yo).max() <= 2e-5 * max(np.abs(yo).max(), 1e-3)


@pytest.mark.parametrize("batch,width,depth", [(3000, 128, 4), (700, 40, 2)])
def test_gradient_matches_the_oracle(batch, width, depth):
    """Ragged batches (several 1024-row gradient chunks plus a tail) and a
    width that is not a multiple of the tiles."""
    import torch
    net, theta = _net(width, depth, seed=3)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((batch, 8)).astype(np.float32)
    T = rng.standard_normal(batch).astype(np.float32)
    loss = net.loss_grad(torch.as_tensor(X, device="cuda"), torch.as_tensor(T, device="cuda"))
    g = net.grad.cpu().numpy().astype(np.float64)
    Lo, go = M.gradient(theta, X.astype(np.float64), T.astype(np.float64), n_in=8, width=width, depth=depth)
    assert abs(float(loss.item()) - Lo) <= 1e-5 * Lo
    # per layer, relative to the layer's largest gradient entry
    k = 0
    for o, i in M.layer_shapes(8, width, depth):
        for size in (o * i, o):
            a, b = g[k:k + size], go[k:k + size]
            assert np.abs(a - b).max() <= 2e-4 * max(np.abs(b).max(), 1e-6), (k, size)
            k += size


def test_adam_steps_match_the_oracle():
    import torch
    net, theta = _net(48, 2, seed=5)
    rng = np.random.default_rng(2)
    X = torch.as_tensor(rng.standard_normal((512, 8)).astype(np.float32), device="cuda")
    T = torch.as_tensor(rng.standard_normal(512).astype(np.float32), device="cuda")
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    th = theta.copy()
    for k in (1, 2, 3):
        net.loss_grad(X, T)
        g = net.grad.cpu().numpy().astype(np.float64)
        net.adam(1e-3)
        th, m, v = M.adam(th, m, v, g, k, 1e-3)
        got = net.theta.cpu().numpy().astype(np.float64)
        assert np.abs(got - th).max() <= 1e-6 + 1e-5 * np.abs(th).max()


def test_feature_kernels_follow_the_documented_map():
    import torch
    from paper_2406_11626_gb300 import warmstart as W
    n, L = 6, 4.0
    p5 = (0.45, 0.62, 5.0, 0.13, 0.07)
    x = W.features_grid(n, L, p5).cpu().numpy()
    c = (-L + (np.arange(n) + 0.5) * 2 * L / n) / L
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
    want_par = [(p5[0] - 0.5) / 0.2, (p5[1] - 0.5) / 0.2, (p5[2] - 7) / 5, (p5[3] - 0.1) / 0.1,
                (p5[4] - 0.15) / 0.15]
    np.testing.assert_allclose(x[:, 0], xx.ravel(), rtol=1e-6)
    np.testing.assert_allclose(x[:, 1], yy.ravel(), rtol=1e-6)
    np.testing.assert_allclose(x[:, 2], zz.ravel(), rtol=1e-6)
    np.testing.assert_allclose(x[:, 3:], np.broadcast_to(want_par, (n ** 3, 5)), rtol=1e-5, atol=1e-6)
    store = torch.arange(2 * n ** 3, dtype=torch.float32, device="cuda").reshape(2, -1) * 1e-3
    draws = torch.tensor([p5, (0.3, 0.7, 2.0, 0.0, 0.3)], dtype=torch.float32, device="cuda")
    idx = torch.tensor([0, 5, n ** 3 + 7, 2 * n ** 3 - 1], dtype=torch.int64, device="cuda")
    xs, t = W.features_sample(n, L, draws, store, idx)
    np.testing.assert_allclose(t.cpu().numpy(), 10.0 * store.reshape(-1)[idx].cpu().numpy(), rtol=1e-6)
    np.testing.assert_allclose(xs[1].cpu().numpy(), x[5], rtol=1e-6)
    np.testing.assert_allclose(xs[2, 3:].cpu().numpy(), [-1.0, 1.0, -1.0, -1.0, 1.0], rtol=1e-5, atol=1e-6)
    y = torch.tensor([1.0, -2.5], dtype=torch.float32, device="cuda")
    u = torch.zeros(2, dtype=torch.float64, device="cuda")
    W.output_to_u(y, u.data_ptr())
    np.testing.assert_allclose(u.cpu().numpy(), [0.1, -0.25])


def test_training_reduces_the_loss():
    import torch
    net, _ = _net(64, 3, seed=7, max_batch=2048)
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, (2048, 8)).astype(np.float32)
    T = (np.sin(2 * X[:, 0]) * X[:, 1] + 0.5 * X[:, 2] ** 2).astype(np.float32)
    Xd, Td = torch.as_tensor(X, device="cuda"), torch.as_tensor(T, device="cuda")
    L0 = float(net.loss_grad(Xd, Td).item())
    for _ in range(400):
        net.loss_grad(Xd, Td)
        net.adam(3e-3)
    assert float(net.loss_grad(Xd, Td).item()) < 0.05 * L0


def test_trained_network_saves_sweeps_on_held_out_draws():
    """A small version of the experiment (32^3 cells, 24 training solves,
    4 held-out draws): starting the plain relaxation from the network's
    guess needs fewer sweeps to the same tolerance than starting from u = 0,
    and the plain solve still reaches the tolerance every time."""
    from paper_2406_11626_gb300 import warmstart as W
    n, L = 32, 8.0
    draws = W.sobol_draws(28)
    store, sweeps, _ = W.solve_draws(draws[:24], n, L, tol=1e-9, check=10, omega=W.optimal_omega(n))
    assert (sweeps > 0).all()
    net = W.MLP(8, 128, 4, 16384)
    net.set_params(W.init_params(seed=0))
    W.train(net, store, draws[:24], n, L, steps=3000, batch=8192, lr=2e-3, lr_final=1e-5)
    res = W.evaluate(net, draws[24:], n, L, tol=1e-9, check=10, omega=W.optimal_omega(n))
    assert (res[:, 0] > 0).all() and (res[:, 1] > 0).all()
    assert res[:, 1].mean() < 0.9 * res[:, 0].mean(), res
