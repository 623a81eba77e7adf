"""Pins of the oracle's element operators against closed forms, invariants
and the paper's own exactness claims (Sec. 2.1 / 2.2)."""
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.special as sp

from oracle import basis, operators as ops
from paper_2604_04644_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SHAPES = [0, 1, 2, 3]


def one_element(shape, curved, scale=1.0, cell=0):
    m = inputs.single_element_mesh(shape, 1, curved=curved, scale=scale, cell=cell)
    X = m["xyz"][m["vert"][0][: (8, 6, 5, 4)[shape]]]
    return X[None]


def vertex_coeffs(shape, P, values):
    """Coefficient vector with 'values' (one per reference vertex) on the vertex modes."""
    ml = basis.modes(shape, P)
    V = np.array(basis.REF_VERTS[shape], dtype=float)
    centre = V.mean(axis=0)
    pts = (V + 1e-10 * (centre - V)).T
    B = basis.evaluate(shape, P, *pts)
    uh = np.zeros(len(ml))
    for i, m in enumerate(ml):
        if all(f[0] in ("1", "L", "R") for f in m):
            v = int(np.argmax(B[:, i]))
            uh[i] = values[v]
    return uh


def element_volume_affine(shape, X):
    X0 = X[0]
    v = ops.AXIS_VERTS[shape]
    det = abs(np.linalg.det(np.stack([X[v[d]] - X0 for d in range(3)], axis=1)))
    return det / 8.0 * basis.REF_VOLUME[shape]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("P", [1, 2, 4, 7])
def test_volume_from_mass_of_constant(shape, P):
    X = one_element(shape, False, scale=0.3)
    uh = vertex_coeffs(shape, P, np.ones(len(basis.REF_VERTS[shape])))
    Mu = ops.apply_block("mass", shape, P, P + 2, X, False, 1, uh[None])[0]
    # the constant 1 is the sum of the vertex modes, so (1, 1) = uh . (M uh)
    assert uh @ Mu == pytest.approx(element_volume_affine(shape, X[0]), rel=1e-13)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("curved", [False, True])
def test_laplacian_of_constant_is_zero(shape, curved):
    P = 5
    X = one_element(shape, curved)
    uh = vertex_coeffs(shape, P, np.ones(len(basis.REF_VERTS[shape])))
    M, L = ops.element_matrices(shape, P, P + 2, X, curved, 1)
    assert np.abs(L[0] @ uh).max() < 1e-13 * np.abs(L[0]).max()


@pytest.mark.parametrize("shape", SHAPES)
def test_energy_of_linear_function_equals_volume(shape):
    """Affine element, u = x_i (reproduced by the vertex modes): u^T L u = vol."""
    P = 3
    X = one_element(shape, False, scale=0.7)
    vol = element_volume_affine(shape, X[0])
    M, L = ops.element_matrices(shape, P, P + 2, X, False, 1)
    for i in range(3):
        uh = vertex_coeffs(shape, P, X[0][:, i])
        assert uh @ L[0] @ uh == pytest.approx(vol, rel=1e-13)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("curved", [False, True])
def test_symmetry_and_definiteness(shape, curved):
    P = 4
    X = one_element(shape, curved)
    M, L = ops.element_matrices(shape, P, P + 2, X, curved, 1)
    M, L = M[0], L[0]
    for A in (M, L):
        assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max() * 10
    np.linalg.cholesky(M)
    np.linalg.cholesky(M + L)
    ev = np.linalg.eigvalsh(L)
    assert ev[0] > -1e-12 * ev[-1]
    assert ev[1] > 1e-8 * ev[-1]           # only the constants are in the kernel


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("curved", [False, True])
@pytest.mark.parametrize("P", [1, 3, 6])
def test_collocated_equals_plain(shape, curved, P):
    """Paper Sec. 2.2: the collocated form (Eq. helm1) is exact whenever the
    Lagrange span at the quadrature points contains the expansion."""
    X = one_element(shape, curved)
    rng = np.random.default_rng(P)
    uh = rng.uniform(-1, 1, (1, basis.n_modes(shape, P)))
    a = ops.apply_block("helmholtz", shape, P, P + 2, X, curved, 1, uh, 1.3)
    b = ops.apply_block("helmholtz_collocated", shape, P, P + 2, X, curved, 1, uh, 1.3)
    assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("P", [1, 2, 4])
def test_quadrature_independence_affine(shape, P):
    X = one_element(shape, False, scale=0.5)
    M1, L1 = ops.element_matrices(shape, P, P + 2, X, False, 1)
    M2, L2 = ops.element_matrices(shape, P, P + 5, X, False, 1)
    assert np.abs(M1 - M2).max() <= 1e-12 * np.abs(M1).max()
    assert np.abs(L1 - L2).max() <= 1e-12 * np.abs(L1).max()


def _frac(s):
    return float(Fraction(s))


def test_p1_hex_textbook_matrices():
    vals = {l.split()[0]: [_frac(t) for t in l.split()[1:]]
            for l in open(os.path.join(GOLDEN, "p1_textbook_matrices.txt")) if l.strip() and l[0] != "#"}
    m1 = np.array(vals["m1"]).reshape(2, 2)
    k1 = np.array(vals["k1"]).reshape(2, 2)
    # reference hex [-1,1]^3: vertices at the reference coordinates
    X = np.array(basis.REF_VERTS[0], dtype=float)[None]
    M, L = ops.element_matrices(0, 1, 3, X, False, 1)
    kron = lambda a, b, c: np.kron(np.kron(a, b), c)
    np.testing.assert_allclose(M[0], kron(m1, m1, m1), atol=1e-14)
    np.testing.assert_allclose(L[0], kron(k1, m1, m1) + kron(m1, k1, m1) + kron(m1, m1, k1), atol=1e-14)


def test_p1_tet_textbook_matrices():
    vals = {l.split()[0]: [_frac(t) for t in l.split()[1:]]
            for l in open(os.path.join(GOLDEN, "p1_textbook_matrices.txt")) if l.strip() and l[0] != "#"}
    X = np.array([[0.1, 0.2, 0.0], [1.3, 0.1, 0.2], [0.2, 0.9, 0.1], [0.3, 0.3, 1.1]])
    M, L = ops.element_matrices(3, 1, 3, X[None], False, 1)
    vol = abs(np.linalg.det(np.stack([X[i] - X[0] for i in (1, 2, 3)], axis=1))) / 6
    # barycentric gradients: rows of inv([[1, x, y, z]])
    A = np.hstack([np.ones((4, 1)), X])
    grads = np.linalg.inv(A)[1:, :].T            # (vertex, 3)
    # the oracle's vertex-mode order: identify each mode's vertex
    perm = [int(np.argmax(np.abs(vertex_coeffs(3, 1, np.eye(4)[v])))) for v in range(4)]
    Mv = vol * vals["tet_mass_factor"][0] * (np.ones((4, 4)) + np.eye(4))
    Lv = vol * grads @ grads.T
    Mo = M[0][np.ix_(perm, perm)]
    Lo = L[0][np.ix_(perm, perm)]
    np.testing.assert_allclose(Mo, Mv, atol=1e-14)
    np.testing.assert_allclose(Lo, Lv, atol=1e-13)


def _cell_integral(coef, lo, hi):
    """Exact integral over a box of sum coef[(a,b,c)] x^a y^b z^c."""
    tot = 0.0
    for (a, b, c), v in coef.items():
        tot += v * np.prod([(hi[d] ** (k + 1) - lo[d] ** (k + 1)) / (k + 1) for d, k in enumerate((a, b, c))])
    return tot


def test_split_consistency_cubic():
    """Integral of a cubic over one cube cell: the hex, its 2 prisms, 6 pyramids
    and 6 tets all give the closed-form value, each via the mass action on the
    element's interpolant (sum of (M uhat) over the vertex modes)."""
    rng = np.random.default_rng(5)
    coef = {}
    for a in range(4):
        for b in range(4 - a):
            for c in range(4 - a - b):
                coef[(a, b, c)] = rng.uniform(-1, 1)
    p = lambda x: sum(v * x[0] ** a * x[1] ** b * x[2] ** c for (a, b, c), v in coef.items())
    exact = _cell_integral(coef, [0, 0, 0], [1, 1, 1])
    P, Q = 3, 5
    for shape in SHAPES:
        m = inputs.slab_mesh(1, 1, 1, P, curved=False, slabs=(shape,))
        total = 0.0
        for e in range(m["n_elem"]):
            nv = (8, 6, 5, 4)[shape]
            X = m["xyz"][m["vert"][e][:nv]][None]
            ref = ops.reference(shape, P, Q)
            g = ops.block_metrics(shape, P, Q, X, False, 1)
            # physical coordinates of the quadrature points (affine map)
            X0 = X[0, 0]
            v = ops.AXIS_VERTS[shape]
            E = np.stack([X[0, v[d]] - X0 for d in range(3)], axis=1)
            xq = X0[:, None] + E @ ((ref["xi"] + 1) / 2)
            uh, *_ = np.linalg.lstsq(ref["B"], p(xq), rcond=None)
            assert np.abs(ref["B"] @ uh - p(xq)).max() < 1e-12
            Mu = ops.apply_block("mass", shape, P, Q, X, False, 1, uh[None])[0]
            ones = vertex_coeffs(shape, P, np.ones(nv))
            total += ones @ Mu
        assert total == pytest.approx(exact, rel=1e-13), shape


def test_curved_mesh_volume_matches_independent_quadrature():
    """Sum of element volumes of the curved slab mesh = int_[0,1]^3 det(D Phi),
    the latter by a 40-point Gauss-Legendre tensor rule (scipy)."""
    mesh = inputs.slab_mesh(2, 2, 4, 6, curved=True)
    coeff, _ = ops.layout(mesh)
    uh = np.zeros(coeff[-1])
    for e in range(mesh["n_elem"]):
        s = int(mesh["shape"][e])
        uh[coeff[e]:coeff[e + 1]] = vertex_coeffs(s, 6, np.ones((8, 6, 5, 4)[s]))
    vol = uh @ ops.apply("mass", mesh, uh)
    x, w = sp.roots_legendre(40)
    x = (x + 1) / 2
    w = w / 2
    X1, X2, X3 = np.meshgrid(x, x, x, indexing="ij")
    a = 0.05 * np.pi
    s = lambda t: np.sin(np.pi * t)
    c = lambda t: np.cos(np.pi * t)
    Dm = np.empty(X1.shape + (3, 3))
    Dm[..., 0, 0] = 1; Dm[..., 1, 1] = 1; Dm[..., 2, 2] = 1
    Dm[..., 0, 1] = a * c(X2) * s(X3); Dm[..., 0, 2] = a * s(X2) * c(X3)
    Dm[..., 1, 2] = a * c(X3) * s(X1); Dm[..., 1, 0] = a * s(X3) * c(X1)
    Dm[..., 2, 0] = a * c(X1) * s(X2); Dm[..., 2, 1] = a * s(X1) * c(X2)
    ref_vol = np.einsum("i,j,k,ijk->", w, w, w, np.linalg.det(Dm))
    assert vol == pytest.approx(ref_vol, rel=1e-9)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("curved", [False, True])
def test_building_blocks_compose(shape, curved):
    """phys_deriv of bwd_trans (Lagrange route) = analytic gradient, and
    iproduct_wrt_deriv(phys_deriv(bwd_trans(u))) = laplacian(u);
    iproduct_wrt_base(bwd_trans(u)) = mass(u)."""
    P = 4
    X = one_element(shape, curved)
    rng = np.random.default_rng(2)
    uh = rng.uniform(-1, 1, (1, basis.n_modes(shape, P)))
    Q = P + 2
    u = ops.apply_block("bwd_trans", shape, P, Q, X, curved, 1, uh)
    du = ops.apply_block("phys_deriv", shape, P, Q, X, curved, 1, u)
    ref = ops.reference(shape, P, Q)
    g = ops.block_metrics(shape, P, Q, X, curved, 1)
    gx = ops._grad_x(ref, g, uh)
    assert np.abs(du - gx).max() <= 1e-11 * np.abs(gx).max()
    lap = ops.apply_block("laplacian", shape, P, Q, X, curved, 1, uh)
    lap2 = ops.apply_block("iproduct_wrt_deriv", shape, P, Q, X, curved, 1, du)
    assert np.abs(lap - lap2).max() <= 1e-12 * np.abs(lap).max()
    mass = ops.apply_block("mass", shape, P, Q, X, curved, 1, uh)
    mass2 = ops.apply_block("iproduct_wrt_base", shape, P, Q, X, curved, 1, u)
    assert np.abs(mass - mass2).max() <= 1e-13 * np.abs(mass).max()


def test_mesh_apply_matches_block_apply_and_subset():
    mesh = inputs.slab_mesh(2, 2, 4, 3, curved=True)
    coeff, _ = ops.layout(mesh)
    uh = inputs.random_coefficients(7, coeff)
    full = ops.apply("helmholtz", mesh, uh, 2.0)
    part = ops.apply("helmholtz", mesh, uh, 2.0, elems=[1, 9, 30])
    for e in (1, 9, 30):
        np.testing.assert_allclose(part[coeff[e]:coeff[e + 1]], full[coeff[e]:coeff[e + 1]], rtol=0, atol=1e-14)
    lin = 2.0 * ops.apply("mass", mesh, uh) + ops.apply("laplacian", mesh, uh)
    assert np.abs(full - lin).max() <= 1e-13 * np.abs(full).max()


def test_unit_cube_of_64_hexes_volume():
    """The 4x4x4 affine hex mesh of [0,1]^3 at P = 4 (Q = 6): the constant 1 on
    every element (vertex modes = 1) gives uhat_e . (M uhat)_e = 1/64 per
    hexahedron and 1 over the cube."""
    mesh = inputs.hex_cube_mesh(4, 4)
    co, _ = ops.layout(mesh)
    uh1 = vertex_coeffs(0, 4, np.ones(8))
    uh = np.tile(uh1, mesh["n_elem"])
    Mu = ops.apply("mass", mesh, uh, 1.0)
    per = np.array([uh[co[e]:co[e + 1]] @ Mu[co[e]:co[e + 1]] for e in range(mesh["n_elem"])])
    assert mesh["n_elem"] == 64 and np.allclose(per, 1.0 / 64, rtol=1e-13, atol=0)
    assert per.sum() == pytest.approx(1.0, rel=1e-13)
