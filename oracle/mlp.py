"""FP64 reference of the cost-model network (test infrastructure only).

Network: y = W3 relu(W2 relu(W1 x + b1) + b2) + b3; loss L = mean over the
batch and the outputs of (y - t)^2.  Parameters in one flat vector:
W1[H][n_in], b1[H], W2[H][H], b2[H], W3[n_out][H], b3[n_out].
The gradient is the textbook backpropagation of that composition; it is
pinned against central finite differences in tests/test_oracle_mlp.py.
"""
import numpy as np


def unpack(p, n_in, H, n_out):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * n_in].reshape(H, n_in); o += H * n_in
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + n_out * H].reshape(n_out, H); o += n_out * H
    b3 = p[o:o + n_out]; o += n_out
    assert o == len(p)
    return W1, b1, W2, b2, W3, b3


def n_params(n_in, H, n_out):
    return H * n_in + H + H * H + H + n_out * H + n_out


def forward(p, x, n_in, H, n_out):
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, H, n_out)
    a1 = np.maximum(x @ W1.T + b1, 0.0)
    a2 = np.maximum(a1 @ W2.T + b2, 0.0)
    return a2 @ W3.T + b3


def loss(p, x, t, n_in, H, n_out):
    y = forward(p, x, n_in, H, n_out)
    return float(np.mean((y - t) ** 2))


def grad(p, x, t, n_in, H, n_out):
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, H, n_out)
    z1 = x @ W1.T + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ W2.T + b2
    a2 = np.maximum(z2, 0.0)
    y = a2 @ W3.T + b3
    B = x.shape[0]
    d3 = 2.0 * (y - t) / (B * n_out)
    gW3 = d3.T @ a2
    gb3 = d3.sum(axis=0)
    d2 = (d3 @ W3) * (z2 > 0)
    gW2 = d2.T @ a1
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (z1 > 0)
    gW1 = d1.T @ x
    gb1 = d1.sum(axis=0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
