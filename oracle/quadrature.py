"""Gauss quadrature rules used by the operators (paper Sec. 2.1: tensor rules
with P+2 Gauss-Lobatto points per direction; Sec. 2.3: tensor rules on the
collapsed coordinates of the Duffy transformation).

Nodes: zeros of Jacobi polynomials as eigenvalues of the symmetric
tridiagonal Jacobi matrix (Golub & Welsch 1969), plus the fixed end points.
Weights: the interpolatory weights, found by requiring the rule to integrate
the orthogonal polynomials P_k^{(alpha,0)}, k < Q, exactly against
(1 - x)^alpha, i.e. sum_l w_l P_k(x_l) = delta_k0 * 2^(alpha+1)/(alpha+1).

* GLL(Q):         Gauss-Lobatto-Legendre, nodes -1, +1 and the zeros of P_{Q-2}^{(1,1)}.
* GRJ(Q, alpha):  Gauss-Radau-Jacobi for the weight (1 - x)^alpha with the node
                  fixed at -1; the other nodes are the zeros of P_{Q-1}^{(alpha,1)}.
"""
import numpy as np

from .jacobi import jacobi


def jacobi_zeros(n, a, b):
    """Zeros of P_n^{(a,b)} (Golub-Welsch)."""
    if n == 0:
        return np.zeros(0)
    ab = a + b
    diag = np.empty(n)
    for i in range(n):
        den = (2.0 * i + ab) * (2.0 * i + ab + 2.0)
        diag[i] = (b - a) / (ab + 2.0) if i == 0 else (b * b - a * a) / den
    off = np.empty(max(n - 1, 0))
    for i in range(1, n):
        num = 4.0 * i * (i + a) * (i + b) * (i + ab)
        den = (2.0 * i + ab) ** 2 * (2.0 * i + ab + 1.0) * (2.0 * i + ab - 1.0)
        off[i - 1] = np.sqrt(num / den)
    J = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    return np.sort(np.linalg.eigvalsh(J))


def interpolatory_weights(x, alpha):
    """Weights of the interpolatory rule on nodes x for the weight (1-x)^alpha."""
    Q = len(x)
    V = np.array([jacobi(k, float(alpha), 0.0, x) for k in range(Q)])
    rhs = np.zeros(Q)
    rhs[0] = 2.0 ** (alpha + 1) / (alpha + 1.0)
    return np.linalg.solve(V, rhs)


def gll(Q):
    """Gauss-Lobatto-Legendre nodes and weights, Q >= 2 points."""
    x = np.concatenate([[-1.0], jacobi_zeros(Q - 2, 1.0, 1.0), [1.0]])
    return x, interpolatory_weights(x, 0)


def grj(Q, alpha):
    """Gauss-Radau-Jacobi nodes (node -1 included, +1 excluded) and weights."""
    x = np.concatenate([[-1.0], jacobi_zeros(Q - 1, float(alpha), 1.0)])
    return x, interpolatory_weights(x, alpha)


def shape_rule(shape, Q, reduced=0):
    """Per-direction (nodes, weights) in the collapsed coordinates eta_1..3.

    The Duffy Jacobian is absorbed into the collapsed directions:
    prism (1-eta3)/2, pyramid ((1-eta3)/2)^2, tet ((1-eta2)/2)((1-eta3)/2)^2,
    so GRJ(alpha=1) weights are halved and GRJ(alpha=2) weights quartered.
    The product of the three weights is the weight of the xi-space integral.
    reduced = 1: Q - 1 points in the collapsed (Gauss-Radau-Jacobi)
    directions, which still integrate degree 2Q - 4 = 2P exactly against
    their Jacobi weight.
    """
    g = gll(Q)
    if shape == 0:
        return [g, g, g]
    Qc = Q - (1 if reduced else 0)
    r1 = grj(Qc, 1)
    r1 = (r1[0], r1[1] / 2.0)
    r2 = grj(Qc, 2)
    r2 = (r2[0], r2[1] / 4.0)
    if shape == 1:
        return [g, g, r1]
    if shape == 2:
        return [g, g, r2]
    if shape == 3:
        return [g, r1, r2]
    raise ValueError(shape)
