"""Two-dimensional quadrilateral and triangle expansions and their mass,
Laplacian and Helmholtz operators (test infrastructure: only tests/, smoke()
and bench.py's CPU baseline may use it).

Paper Sec. 2.2, two-dimensional formulation: the elemental Helmholtz operator
of an expansion phi_n on a quadrilateral or a triangle,
  H[m][n] = sum_l w_l |J_l| [ lambda phi_m phi_n + (grad_x phi_m).(grad_x phi_n) ],
evaluated with a tensor rule in the (collapsed) coordinates, its split
H = lambda M + L, and the collocated form (Eq. helm1 in two dimensions)
B^T { sum_i [sum_d D_d^T Lam_di] W [sum_d' Lam_d'i D_d'] + lambda W } B.

Bases (the modified C0 basis of Karniadakis & Sherwin that the paper uses,
in the 1-D factors of jacobi.py):
  quadrilateral  phi_{ab}(xi) = A_a(xi_1) A_b(xi_2), A = (L, R, psi_1 .. psi_{P-1});
  triangle       on eta_1 = 2 (1 + xi_1)/(1 - xi_2) - 1, eta_2 = xi_2 (Sec. 2.3):
                 vertices L L, R L and the collapsed vertex 1 R; edges psi_p W_{p,0},
                 L psi_r, R psi_r; interior psi_p W_{p,r} (p, r >= 1, p + r < P).
Mode order: by the key (a, b), b fastest; a: L or 1 -> 0, R -> 1, psi_n ->
n + 1; b: the same rule on the second factor, except that a psi_p first
factor makes the key of W_{p,r} r (the triangle's warped family).

Quadrature: Gauss-Lobatto-Legendre with Q = P + 2 points in xi_1 / eta_1 and
in the quadrilateral's xi_2; Gauss-Radau-Jacobi (alpha = 1) with Q points in
the triangle's eta_2, its weights halved to absorb the Duffy factor
(1 - eta_2)/2 of d xi / d eta (quadrature.py).  Point order (i, j), j fastest.

Element maps: the affine map of vertex 0 and its two neighbours along xi_1
and xi_2 (quadrilateral vertices 1 and 3, triangle vertices 1 and 2),
  A_e(xi) = X_0 + (xi_1 + 1)/2 (X_{v1} - X_0) + (xi_2 + 1)/2 (X_{v2} - X_0),
then, on curved elements, the smooth map of the unit square onto itself
  Phi(x)_i = x_i + 0.05 sin(pi x_1) sin(pi x_2)   (i = 1, 2; deformation 1).
The Jacobian d x / d xi is taken by complex step (exact to rounding).
"""
from functools import lru_cache

import numpy as np

from . import quadrature
from .basis import _A, _a_key, _weight
from .jacobi import factor

QUAD, TRI = 4, 5
AXIS_VERTS_2D = {QUAD: (1, 3), TRI: (1, 2)}
NV_2D = {QUAD: 4, TRI: 3}


def n_modes(shape, P):
    return (P + 1) ** 2 if shape == QUAD else (P + 1) * (P + 2) // 2


def _key(shape, mode):
    fa, fb = mode
    ka = _a_key(fa)
    kb = fb[2] if (shape == TRI and fa[0] == "psi") else _a_key(fb)
    return (ka, kb)


def modes(shape, P):
    A = _A(P)
    if shape == QUAD:
        out = [(fa, fb) for fa in A for fb in A]
    else:
        out = [(("L",), ("L",)), (("R",), ("L",)), (("1",), ("R",))]
        out += [(("psi", p), ("W", p, 0)) for p in range(1, P)]
        out += [(("L",), ("psi", r)) for r in range(1, P)]
        out += [(("R",), ("psi", r)) for r in range(1, P)]
        out += [(("psi", p), ("W", p, r)) for p in range(1, P) for r in range(1, P) if p + r < P]
    return sorted(out, key=lambda m: _key(shape, m))


def eta_from_xi(shape, xi1, xi2):
    if shape == QUAD:
        return xi1, xi2
    return 2.0 * (1.0 + xi1) / (1.0 - xi2) - 1.0, xi2


def xi_from_eta(shape, e1, e2):
    if shape == QUAD:
        return e1, e2
    return (1.0 + e1) * (1.0 - e2) / 2.0 - 1.0, e2


def evaluate(shape, P, xi1, xi2):
    """phi_m(xi) for all modes: (n_points, n_modes); complex inputs allowed."""
    a, b = eta_from_xi(shape, np.asarray(xi1), np.asarray(xi2))
    return np.stack([factor(fa, a) * factor(fb, b) for fa, fb in modes(shape, P)], axis=-1)


def complex_step_gradient2(fun, xi, h=1e-30):
    out = []
    for d in range(2):
        z = [np.asarray(xi[k], dtype=np.complex128) for k in range(2)]
        z[d] = z[d] + 1j * h
        out.append(np.imag(fun(*z)) / h)
    return out


def shape_rule(shape, Q):
    g = quadrature.gll(Q)
    if shape == QUAD:
        return [g, g]
    r = quadrature.grj(Q, 1)
    return [g, (r[0], r[1] / 2.0)]


def lagrange_derivative_matrix(x):
    """D[i][j] = h_j'(x_i) of the Lagrange basis on the nodes x."""
    from .jacobi import jacobi
    V = np.stack([jacobi(k, 0.0, 0.0, x) for k in range(len(x))], axis=1)
    Vd = np.stack([np.imag(jacobi(k, 0.0, 0.0, x + 1j * 1e-30)) / 1e-30 for k in range(len(x))], axis=1)
    return Vd @ np.linalg.inv(V)


@lru_cache(maxsize=None)
def reference(shape, P, Q):
    (x1, w1), (x2, w2) = shape_rule(shape, Q)
    e1, e2 = np.meshgrid(x1, x2, indexing="ij")
    eta = np.stack([e1.ravel(), e2.ravel()])
    W = np.einsum("i,j->ij", w1, w2).ravel()
    xi = np.stack(xi_from_eta(shape, *eta))
    B = evaluate(shape, P, *xi)
    Dxi = complex_step_gradient2(lambda a, b: evaluate(shape, P, a, b), xi)
    # T[l, d, a] = d eta_d / d xi_a
    T = np.stack(complex_step_gradient2(lambda a, b: np.stack(eta_from_xi(shape, a, b)), xi),
                 axis=-1).transpose(1, 0, 2)
    D1 = [lagrange_derivative_matrix(x) for x in (x1, x2)]
    return dict(eta=eta, xi=xi, W=W, B=B, Dxi=Dxi, T=T, nodes=(x1, x2), D1=D1, NP=B.shape[1],
                NQ=B.shape[0], Q=Q)


def deform2(x1, x2, kind=1):
    if kind == 0:
        return x1, x2
    s = 0.05 * np.sin(np.pi * x1) * np.sin(np.pi * x2)
    return x1 + s, x2 + s


def block_points(shape, X, curved, kind, xi):
    """x[i, e, l] = chi^e(xi_l) for vertex arrays X (Ne, nv, 2)."""
    v1, v2 = AXIS_VERTS_2D[shape]
    X0 = X[:, 0, :]
    E1, E2 = X[:, v1, :] - X0, X[:, v2, :] - X0
    t1, t2 = (xi[0] + 1.0) / 2.0, (xi[1] + 1.0) / 2.0
    y = [X0[:, i:i + 1] + E1[:, i:i + 1] * t1[None, :] + E2[:, i:i + 1] * t2[None, :] for i in range(2)]
    if curved:
        y = list(deform2(y[0], y[1], kind))
    return np.stack(y)


def block_jacobian(shape, X, curved, kind, xi):
    """J[e, l, i, d] = d x_i / d xi_d."""
    g = complex_step_gradient2(lambda a, b: block_points(shape, X, curved, kind, np.stack([a, b])), xi)
    return np.stack(g, axis=-1).transpose(1, 2, 0, 3)


def block_metrics(shape, P, Q, X, curved, kind):
    ref = reference(shape, P, Q)
    J = block_jacobian(shape, X, curved, kind, ref["xi"])
    detJ = np.linalg.det(J)
    Jinv = np.linalg.inv(J)                                  # [e, l, d, i] = d xi_d / d x_i
    return dict(J=J, detJ=detJ, Jinv=Jinv, wJ=ref["W"][None, :] * detJ)


def element_matrices(shape, P, Q, X, curved, kind):
    """Explicit (M, L) of each element: (Ne, NP, NP) each."""
    ref = reference(shape, P, Q)
    g = block_metrics(shape, P, Q, X, curved, kind)
    B = ref["B"]
    M = np.einsum("lm,el,ln->emn", B, g["wJ"], B)
    Gx = np.einsum("eldi,dlm->eilm", g["Jinv"], np.stack(ref["Dxi"]))    # d phi_m / d x_i at l
    L = np.einsum("eilm,el,eiln->emn", Gx, g["wJ"], Gx)
    return M, L


def geometric_factors_block(shape, P, Q, X, curved, kind):
    """Per point: G_dd' = w|J| sum_i (d eta_d/dx_i)(d eta_d'/dx_i) (3: 11, 12, 22) and w|J|."""
    ref = reference(shape, P, Q)
    g = block_metrics(shape, P, Q, X, curved, kind)
    Gx = np.einsum("elda,elai->eldi", ref["T"][None].repeat(len(X), 0), g["Jinv"])
    G = np.einsum("el,eldi,elki->eldk", g["wJ"], Gx, Gx)
    return np.stack([G[:, :, 0, 0], G[:, :, 0, 1], G[:, :, 1, 1], g["wJ"]], axis=1)   # (Ne, 4, NQ)


def helmholtz_collocated_block(shape, P, Q, X, curved, kind, uh, lam):
    """Eq. (helm1) in two dimensions, with Lagrange differentiation along the
    eta lines of the tensor points."""
    ref = reference(shape, P, Q)
    g = block_metrics(shape, P, Q, X, curved, kind)
    u = uh @ ref["B"].T
    U = u.reshape(-1, Q, Q)
    D1, D2 = ref["D1"]
    v = np.stack([np.einsum("im,emj->eij", D1, U), np.einsum("jm,eim->eij", D2, U)]).reshape(2, len(X), -1)
    Gx = np.einsum("elda,elai->eldi", ref["T"][None].repeat(len(X), 0), g["Jinv"])
    G = np.einsum("el,eldi,elki->eldk", g["wJ"], Gx, Gx)
    w = np.stack([G[:, :, d, 0] * v[0] + G[:, :, d, 1] * v[1] for d in range(2)]).reshape(2, len(X), Q, Q)
    up = (np.einsum("mi,emj->eij", D1, w[0]) + np.einsum("mj,eim->eij", D2, w[1])).reshape(u.shape)
    return (up + lam * g["wJ"] * u) @ ref["B"]


def layout(mesh):
    npm = np.array([n_modes(int(s), int(p)) for s, p in zip(mesh["shape"], mesh["P"])], dtype=np.int64)
    nq = (mesh["P"].astype(np.int64) + 2) ** 2
    return (np.concatenate([[0], np.cumsum(npm)]).astype(np.int64),
            np.concatenate([[0], np.cumsum(nq)]).astype(np.int64))


def _blocks(mesh, elems=None):
    elems = np.arange(mesh["n_elem"]) if elems is None else np.asarray(elems)
    keys = {}
    for e in elems:
        keys.setdefault((int(mesh["shape"][e]), int(mesh["P"][e]), int(mesh["curved"][e])), []).append(int(e))
    return keys


def _verts(mesh, shape, elems):
    return mesh["xy"][mesh["vert"][elems][:, :NV_2D[shape]]]


def apply(op, mesh, data, lam=1.0, elems=None):
    """op in mass / laplacian / helmholtz / helmholtz_collocated on the ragged
    coefficient vector ``data`` (elements in user order); with ``elems`` only
    those elements' outputs are computed (the others stay zero)."""
    co, _ = layout(mesh)
    out = np.zeros(co[-1])
    for (shape, P, cv), el in _blocks(mesh, elems).items():
        el = np.array(el)
        X = _verts(mesh, shape, el)
        idx = co[el][:, None] + np.arange(n_modes(shape, P))[None, :]
        uh = data[idx]
        Q = P + 2
        if op == "helmholtz_collocated":
            y = helmholtz_collocated_block(shape, P, Q, X, bool(cv), mesh["deformation"], uh, lam)
        else:
            M, L = element_matrices(shape, P, Q, X, bool(cv), mesh["deformation"])
            H = {"mass": M, "laplacian": L, "helmholtz": L + lam * M}[op]
            y = np.einsum("emn,en->em", H, uh)
        out[idx] = y
    return out
