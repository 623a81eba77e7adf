"""Element maps x = chi^e(xi) and their Jacobians (paper Sec. 2.1, chain rule
and J^e = grad chi^e).

Each element is the affine image of its reference element, fixed by vertex 0
and the three vertices adjacent to it along xi_1, xi_2, xi_3:
  A_e(xi) = X_0 + sum_d (xi_d + 1)/2 (X_{v_d} - X_0);
curved elements are further mapped by the smooth deformation
  Phi(x)_i = x_i + 0.05 sin(pi x_j) sin(pi x_k),  (i,j,k) cyclic   (kind 1),
or, for tests that need a polynomial map, the quadratic
  Phi(x)_i = x_i + 0.1 x_j x_k,  (i,j,k) cyclic                     (kind 2),
so x = Phi(A_e(xi)).  The Jacobian J[i][d] = d x_i / d xi_d is taken by
complex-step differentiation of that composition (exact to rounding).
"""
import numpy as np

from .basis import complex_step_gradient

AXIS_VERTS = {0: (1, 3, 4), 1: (1, 3, 4), 2: (1, 3, 4), 3: (1, 2, 3)}


def deform(x1, x2, x3, kind=1):
    if kind == 0:
        return x1, x2, x3
    if kind == 2:
        return x1 + 0.1 * x2 * x3, x2 + 0.1 * x3 * x1, x3 + 0.1 * x1 * x2
    s = lambda t: np.sin(np.pi * t)
    return (x1 + 0.05 * s(x2) * s(x3),
            x2 + 0.05 * s(x3) * s(x1),
            x3 + 0.05 * s(x1) * s(x2))


def element_frame(shape, X):
    """(X0, E) with E[:, d] = X_{v_d} - X0 for the element's vertex coordinates X."""
    v = AXIS_VERTS[shape]
    X = np.asarray(X, dtype=np.float64)
    E = np.stack([X[v[d]] - X[0] for d in range(3)], axis=1)
    return X[0], E


def element_map(shape, X, curved, kind):
    """Return the function xi -> x for one element (complex-capable)."""
    X0, E = element_frame(shape, X)

    def chi(xi1, xi2, xi3):
        t = [(xi1 + 1.0) / 2.0, (xi2 + 1.0) / 2.0, (xi3 + 1.0) / 2.0]
        y = [X0[i] + E[i, 0] * t[0] + E[i, 1] * t[1] + E[i, 2] * t[2] for i in range(3)]
        if curved:
            y = list(deform(y[0], y[1], y[2], kind))
        return np.stack(y, axis=0)
    return chi


def jacobian(shape, X, curved, kind, xi):
    """J[n, i, d] = d x_i / d xi_d at the points xi (3, n)."""
    chi = element_map(shape, X, curved, kind)
    g = complex_step_gradient(chi, xi)          # list over d of (3, n)
    return np.stack(g, axis=-1).transpose(1, 0, 2)


def mesh_element_vertices(mesh, e):
    shape = int(mesh["shape"][e])
    nv = (8, 6, 5, 4)[shape]
    ids = mesh["vert"][e][:nv]
    return mesh["xyz"][ids]
