"""Oracle of the assembled Helmholtz problem (test infrastructure only).

Paper Sec. 2.1: find u in the C0 space with (grad u, grad v) + lambda (u, v)
= (f, v) for all v, homogeneous Dirichlet conditions.  The oracle does not
number global DOFs at all: it takes the element spaces side by side, writes
continuity across every shared face and vanishing on every boundary face as
linear constraints on the element coefficients (point values on the faces,
basis evaluated in closed form), and takes the null space of those
constraints (SVD) as the C0 space.  The Galerkin system on that space is
solved densely.  Only for tiny meshes.
"""
import numpy as np
import scipy.linalg as sla

from . import basis
from .geometry import AXIS_VERTS, element_map
from .operators import layout, element_matrices, reference, block_metrics

FACES = {0: [(0, 1, 2, 3), (4, 5, 6, 7), (0, 1, 5, 4), (1, 2, 6, 5), (3, 2, 6, 7), (3, 0, 4, 7)],
         1: [(0, 1, 4), (3, 2, 5), (0, 1, 2, 3), (0, 3, 5, 4), (1, 2, 5, 4)],
         2: [(0, 1, 2, 3), (0, 1, 4), (1, 2, 4), (2, 3, 4), (3, 0, 4)],
         3: [(0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3)]}
NV = (8, 6, 5, 4)


def _affine_inverse(mesh, e, x):
    s = int(mesh["shape"][e])
    X = mesh["xyz"][mesh["vert"][e][:NV[s]]]
    v = AXIS_VERTS[s]
    E = np.stack([X[v[d]] - X[0] for d in range(3)], axis=1)
    return 2.0 * np.linalg.solve(E, (x - X[0]).T) - 1.0


def constraint_matrix(mesh, pts_per_face, seed=0):
    """Rows: u_e1(x) - u_e2(x) = 0 at points x of every shared face and
    u_e(x) = 0 at points of every boundary face (points as convex
    combinations of the face's vertices, reference coordinates through the
    affine vertex maps, which neighbouring elements share on their face)."""
    co, _ = layout(mesh)
    faces = {}
    for e in range(mesh["n_elem"]):
        for f in FACES[int(mesh["shape"][e])]:
            ids = tuple(sorted(int(mesh["vert"][e][v]) for v in f))
            faces.setdefault(ids, []).append(e)
    rng = np.random.default_rng(seed)
    rows = []
    for ids, els in faces.items():
        V = mesh["xyz"][list(ids)]
        w = rng.dirichlet(np.ones(len(ids)), size=pts_per_face)
        x = w @ V
        blk = np.zeros((pts_per_face, co[-1]))
        for sgn, e in zip((1.0, -1.0), els):
            s = int(mesh["shape"][e])
            xi = _affine_inverse(mesh, e, x)
            blk[:, co[e]:co[e + 1]] += sgn * basis.evaluate(s, int(mesh["P"][e]), xi[0], xi[1], xi[2])
        rows.append(blk)
    return np.concatenate(rows)


def c0_space(mesh, pts_per_face=None, seed=0):
    """Orthonormal basis Z (n_coeff x dim) of the C0 space with zero boundary values."""
    P = int(mesh["P"].max())
    k = pts_per_face or (P + 1) ** 2 + 3      # a face trace has at most (P+1)^2 dimensions
    C = constraint_matrix(mesh, k, seed)
    return sla.null_space(C, rcond=1e-10)


def element_rhs(mesh, f):
    """(f, phi_m) on each element by the quadrature of the element operators."""
    co, _ = layout(mesh)
    b = np.zeros(co[-1])
    for e in range(mesh["n_elem"]):
        s, P, Q = int(mesh["shape"][e]), int(mesh["P"][e]), int(mesh["Q"][e])
        ref = reference(s, P, Q)
        X = mesh["xyz"][mesh["vert"][e][:NV[s]]]
        chi = element_map(s, X, bool(mesh["curved"][e]), mesh["deformation"])
        x = chi(*ref["xi"])
        g = block_metrics(s, P, Q, X[None], bool(mesh["curved"][e]), mesh["deformation"], mesh.get("geometry", 0))
        b[co[e]:co[e + 1]] = ref["B"].T @ (g["wJ"][0] * f(x[0], x[1], x[2]))
    return b


def solve(mesh, lam, f, Z=None):
    """Element coefficients of the discrete C0 solution."""
    co, _ = layout(mesh)
    if Z is None:
        Z = c0_space(mesh)
    H = np.zeros((co[-1], co[-1]))
    for e in range(mesh["n_elem"]):
        s, P, Q = int(mesh["shape"][e]), int(mesh["P"][e]), int(mesh["Q"][e])
        X = mesh["xyz"][mesh["vert"][e][:NV[s]]][None]
        M, L = element_matrices(s, P, Q, X, bool(mesh["curved"][e]), mesh["deformation"], mesh.get("geometry", 0))
        H[co[e]:co[e + 1], co[e]:co[e + 1]] = lam * M[0] + L[0]
    b = element_rhs(mesh, f)
    A = Z.T @ H @ Z
    y = np.linalg.solve(A, Z.T @ b)
    return Z @ y
