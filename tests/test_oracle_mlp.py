"""Pins of the oracle's cost-model network: backpropagation against central
finite differences in FP64, and a forward pass of a hand-sized network."""
import numpy as np
import pytest

from oracle import mlp


@pytest.mark.parametrize("n_in,H,n_out", [(5, 8, 3), (3, 16, 2)])
def test_gradient_matches_central_differences(n_in, H, n_out):
    rng = np.random.default_rng(0)
    p = rng.normal(0, 0.5, mlp.n_params(n_in, H, n_out))
    x = rng.uniform(-1, 1, (7, n_in))
    t = rng.uniform(-1, 1, (7, n_out))
    g = mlp.grad(p, x, t, n_in, H, n_out)
    h = 1e-6
    fd = np.empty_like(p)
    for j in range(len(p)):
        e = np.zeros_like(p)
        e[j] = h
        fd[j] = (mlp.loss(p + e, x, t, n_in, H, n_out) - mlp.loss(p - e, x, t, n_in, H, n_out)) / (2 * h)
    assert np.abs(g - fd).max() <= 1e-6 * max(1.0, np.abs(fd).max())


def test_forward_by_hand():
    # n_in = 1, H = 2, n_out = 1: y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3
    W1 = np.array([[1.0], [-1.0]]); b1 = np.array([0.0, 0.5])
    W2 = np.array([[1.0, 1.0], [0.0, -2.0]]); b2 = np.array([0.0, 1.0])
    W3 = np.array([[2.0, 3.0]]); b3 = np.array([-1.0])
    p = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3])
    x = np.array([[2.0]])
    # a1 = relu([2, -1.5]) = [2, 0]; a2 = relu([2, 1]) = [2, 1]; y = 4 + 3 - 1 = 6
    assert mlp.forward(p, x, 1, 2, 1)[0, 0] == 6.0
