"""Oracle of the warm-start network: a plain FP64 NumPy restatement of the
multilayer perceptron, its mean-squared loss, back-propagation and the Adam
update.

TEST INFRASTRUCTURE ONLY (like the rest of this package): the CUDA kernels
never call it, and nothing in the product falls back to it.

Network: x (n_in) -> depth hidden layers of `width` units with SiLU,
silu(z) = z * sigmoid(z) -> one linear output. Parameters are one flat
vector, layer after layer, each layer its weight matrix (out x in, row
major) then its bias:
    [W_0 (width x n_in), b_0, W_1 (width x width), b_1, ..., W_depth (1 x width), b_depth].
Loss: mean over the batch of (y - t)^2.
Adam (Kingma & Ba): m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
theta <- theta - lr * (m / (1 - b1^k)) / (sqrt(v / (1 - b2^k)) + eps) at step k.
"""
import numpy as np


def layer_shapes(n_in=8, width=128, depth=4):
    dims = [n_in] + [width] * depth + [1]
    return [(dims[l + 1], dims[l]) for l in range(depth + 1)]


def n_params(n_in=8, width=128, depth=4):
    return sum(o * i + o for o, i in layer_shapes(n_in, width, depth))


def unpack(theta, n_in=8, width=128, depth=4):
    """[(W, b), ...] views of the flat parameter vector."""
    out, k = [], 0
    for o, i in layer_shapes(n_in, width, depth):
        W = theta[k:k + o * i].reshape(o, i)
        k += o * i
        b = theta[k:k + o]
        k += o
        out.append((W, b))
    return out


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def silu(z):
    return z * sigmoid(z)


def silu_prime(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def forward(theta, X, n_in=8, width=128, depth=4):
    """Output y (batch,) and the pre-activations of every hidden layer."""
    a = np.asarray(X, dtype=np.float64)
    zs = []
    layers = unpack(np.asarray(theta, dtype=np.float64), n_in, width, depth)
    for l, (W, b) in enumerate(layers):
        z = a @ W.T + b
        if l < len(layers) - 1:
            zs.append(z)
            a = silu(z)
        else:
            a = z
    return a[:, 0], zs


def loss(theta, X, T, **kw):
    y, _ = forward(theta, X, **kw)
    return np.mean((y - np.asarray(T, dtype=np.float64)) ** 2)


def gradient(theta, X, T, n_in=8, width=128, depth=4):
    """(loss, dloss/dtheta) by back-propagation through the layers in reverse."""
    theta = np.asarray(theta, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    layers = unpack(theta, n_in, width, depth)
    # forward, keeping every layer's input
    acts = [X]
    zs = []
    a = X
    for l, (W, b) in enumerate(layers):
        z = a @ W.T + b
        if l < len(layers) - 1:
            zs.append(z)
            a = silu(z)
        else:
            a = z
        acts.append(a)
    y = a[:, 0]
    B = len(y)
    L = np.mean((y - T) ** 2)
    grads = []
    delta = (2.0 / B * (y - T))[:, None]          # dL/dz of the output layer
    for l in range(len(layers) - 1, -1, -1):
        W, b = layers[l]
        gW = delta.T @ acts[l]
        gb = delta.sum(axis=0)
        grads.append((gW, gb))
        if l > 0:
            delta = (delta @ W) * silu_prime(zs[l - 1])
    flat = []
    for gW, gb in reversed(grads):
        flat.append(gW.ravel())
        flat.append(gb)
    return L, np.concatenate(flat)


def adam(theta, m, v, g, k, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (k counts from 1); returns new (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** k)
    vh = v / (1.0 - b2 ** k)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
