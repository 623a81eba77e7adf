"""Jacobi polynomials and the one-dimensional modal functions.

Jacobi polynomials P_n^{(a,b)} by their three-term recurrence
(Abramowitz & Stegun 22.7.1); works for real or complex arguments so that
complex-step derivatives can be taken through it.

One-dimensional functions of the modified C0 basis (Karniadakis & Sherwin,
the basis the paper cites for its 3-D shapes, Sec. 2.3):
  L(z) = (1 - z)/2,  R(z) = (1 + z)/2,
  psi_n(z) = L(z) R(z) P_{n-1}^{(1,1)}(z)              (n >= 1, bubble),
  W_{s,0}(z) = L(z)^{s+1},
  W_{s,r}(z) = L(z)^{s+1} R(z) P_{r-1}^{(2s+1,1)}(z)    (r >= 1, warped family).
"""
import numpy as np


def jacobi(n, a, b, z):
    """P_n^{(a,b)}(z) by the three-term recurrence in n."""
    z = np.asarray(z)
    p0 = np.ones_like(z)
    if n == 0:
        return p0
    p1 = 0.5 * (a - b + (a + b + 2.0) * z)
    for k in range(2, n + 1):
        c = 2.0 * k + a + b
        a1 = 2.0 * k * (k + a + b) * (c - 2.0)
        a2 = (c - 1.0) * (a * a - b * b)
        a3 = (c - 2.0) * (c - 1.0) * c
        a4 = 2.0 * (k + a - 1.0) * (k + b - 1.0) * c
        p0, p1 = p1, ((a2 + a3 * z) * p1 - a4 * p0) / a1
    return p1


def L(z):
    return (1.0 - z) / 2.0


def R(z):
    return (1.0 + z) / 2.0


def psi(n, z):
    """Bubble function of index n >= 1 (polynomial degree n + 1)."""
    return L(z) * R(z) * jacobi(n - 1, 1.0, 1.0, z)


def warped(s, r, z):
    """Member r of the warped family attached to weight s >= 1."""
    if r == 0:
        return L(z) ** (s + 1)
    return L(z) ** (s + 1) * R(z) * jacobi(r - 1, 2.0 * s + 1.0, 1.0, z)


def factor(spec, z):
    """Evaluate a 1-D factor spec: ('1',), ('L',), ('R',), ('psi', n), ('W', s, r)."""
    kind = spec[0]
    if kind == "1":
        return np.ones_like(np.asarray(z))
    if kind == "L":
        return L(z)
    if kind == "R":
        return R(z)
    if kind == "psi":
        return psi(spec[1], z)
    if kind == "W":
        return warped(spec[1], spec[2], z)
    raise ValueError(spec)
