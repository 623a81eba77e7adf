"""Pins of the two-dimensional oracle (quadrilaterals and triangles, the
paper's two-dimensional formulation, Sec. 2.2) against facts that do not come
from it: closed-form integrals over the reference triangle, a tensor product
of 1-D mass matrices built with numpy's Gauss-Legendre rule, a Duffy /
Gauss-Legendre brute force, the energy of linear functions, the area and
first moment of the deformed unit square, and the collocated form
(Eq. helm1) against the plain one."""
import math

import numpy as np
import pytest

from oracle import twod
from oracle.jacobi import factor
from paper_2604_04644_gb300 import inputs

QUAD, TRI = twod.QUAD, twod.TRI


@pytest.fixture(autouse=True)
def _clear_cache():
    twod.reference.cache_clear()
    yield
    twod.reference.cache_clear()


@pytest.mark.parametrize("shape", [QUAD, TRI])
@pytest.mark.parametrize("P", [1, 2, 3, 5, 8])
def test_mode_counts_and_unique_keys(shape, P):
    ms = twod.modes(shape, P)
    assert len(ms) == twod.n_modes(shape, P) == ((P + 1) ** 2 if shape == QUAD else (P + 1) * (P + 2) // 2)
    keys = [twod._key(shape, m) for m in ms]
    assert len(set(keys)) == len(keys) and keys == sorted(keys)


@pytest.mark.parametrize("shape", [QUAD, TRI])
def test_vertex_modes_are_a_partition_of_unity(shape):
    rng = np.random.default_rng(0)
    xi = rng.uniform(-1, 1, (2, 50))
    if shape == TRI:
        xi = xi[:, xi[0] + xi[1] < -1e-3]
    B = twod.evaluate(shape, 4, *xi)
    ms = twod.modes(shape, 4)
    vm = [(("L",), ("L",)), (("L",), ("R",)), (("R",), ("L",)), (("R",), ("R",))] if shape == QUAD else \
        [(("L",), ("L",)), (("1",), ("R",)), (("R",), ("L",))]
    vidx = [ms.index(m) for m in vm]
    rest = [k for k in range(len(ms)) if k not in vidx]
    assert np.allclose(B[:, vidx].sum(1), 1.0, atol=1e-14)
    # the other modes vanish at the vertices
    V = np.array([[-1, -1], [1, -1], [1, 1], [-1, 1]] if shape == QUAD else [[-1, -1], [1, -1], [-1, 0.999999999]])
    BV = twod.evaluate(shape, 4, V[:, 0], V[:, 1])
    assert np.abs(BV[:, rest]).max() < 1e-8


@pytest.mark.parametrize("P", [1, 2, 4, 7])
def test_triangle_rule_integrates_monomials(P):
    """sum_l W_l x^a y^b with x = (xi1+1)/2, y = (xi2+1)/2 over the reference
    triangle = 4 a! b! / (a + b + 2)! for a + b <= 2P (the degree of a mass integrand)."""
    ref = twod.reference(TRI, P, P + 2)
    x, y = (ref["xi"][0] + 1) / 2, (ref["xi"][1] + 1) / 2
    for a in range(2 * P + 1):
        for b in range(2 * P + 1 - a):
            exact = 4.0 * math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs(np.dot(ref["W"], x ** a * y ** b) - exact) <= 1e-14 * max(1.0, exact) * 10, (a, b)


def _square_cell(h, shape):
    """One quadrilateral or the lower triangle of the cell [0,h]^2."""
    X = np.array([[0.0, 0.0], [h, 0.0], [h, h], [0.0, h]]) if shape == QUAD else np.array([[0.0, 0.0], [h, 0.0], [0.0, h]])
    return X[None]


@pytest.mark.parametrize("P", [1, 3, 6])
def test_quad_mass_is_tensor_product_of_1d_mass(P):
    h = 0.3
    M, _ = twod.element_matrices(QUAD, P, P + 2, _square_cell(h, QUAD), False, 1)
    z, w = np.polynomial.legendre.leggauss(P + 3)
    A = [("L",), ("R",)] + [("psi", n) for n in range(1, P)]
    F = np.stack([factor(f, z) for f in A], 1)
    M1 = (F * w[:, None]).T @ F
    assert np.allclose(M[0], (h / 2) ** 2 * np.kron(M1, M1), rtol=0, atol=1e-15)


@pytest.mark.parametrize("P", [1, 2, 4, 6])
def test_triangle_mass_matches_duffy_gauss_legendre(P):
    X = np.array([[[0.1, 0.2], [0.9, 0.3], [0.4, 1.1]]])
    M, _ = twod.element_matrices(TRI, P, P + 2, X, False, 1)
    z, w = np.polynomial.legendre.leggauss(P + 4)
    e1, e2 = np.meshgrid(z, z, indexing="ij")
    W = np.outer(w, w).ravel() * (1 - e2.ravel()) / 2
    xi1, xi2 = twod.xi_from_eta(TRI, e1.ravel(), e2.ravel())
    B = twod.evaluate(TRI, P, xi1, xi2)
    E = np.stack([X[0, 1] - X[0, 0], X[0, 2] - X[0, 0]], 1) / 2
    Mb = (B * (W * abs(np.linalg.det(E)))[:, None]).T @ B
    assert np.allclose(M[0], Mb, rtol=0, atol=1e-14 * np.abs(Mb).max())


@pytest.mark.parametrize("shape", [QUAD, TRI])
@pytest.mark.parametrize("P", [1, 3, 5])
def test_laplacian_energy_of_linear_functions(shape, P):
    """Vertex-mode coefficients of x1, x2 (the vertex values) on an affine
    element: u^T L u = area for u = x_i, 0 between x1 and x2, L 1 = 0."""
    # the quadrilateral is the parallelogram of vertices 0, 1, 3 (its affine map)
    X = np.array([[[0.2, 0.1], [1.0, 0.3], [1.1, 1.0], [0.3, 0.8]]]) if shape == QUAD else \
        np.array([[[0.2, 0.1], [1.0, 0.3], [0.3, 0.8]]])
    _, L = twod.element_matrices(shape, P, P + 2, X, False, 1)
    nv = X.shape[1]
    # vertex modes in mode order: quad LL, LR, RL, RR = vertices 0, 3, 1, 2; triangle LL, 1R, RL = 0, 2, 1
    vmap = [0, 3, 1, 2] if shape == QUAD else [0, 2, 1]
    ms = twod.modes(shape, P)
    vidx = [ms.index(m) for m in ([(("L",), ("L",)), (("L",), ("R",)), (("R",), ("L",)), (("R",), ("R",))]
                                  if shape == QUAD else [(("L",), ("L",)), (("1",), ("R",)), (("R",), ("L",))])]
    E1, E2 = X[0, 1] - X[0, 0], X[0, 3 if shape == QUAD else 2] - X[0, 0]
    area = abs(E1[0] * E2[1] - E1[1] * E2[0]) * (1.0 if shape == QUAD else 0.5)
    u = np.zeros((2, L.shape[1]))
    for k, v in zip(vidx, vmap):
        u[:, k] = X[0, v]
    one = np.zeros(L.shape[1])
    one[vidx] = 1.0
    assert abs(u[0] @ L[0] @ u[0] - area) < 1e-13
    assert abs(u[1] @ L[0] @ u[1] - area) < 1e-13
    assert abs(u[0] @ L[0] @ u[1]) < 1e-13
    assert np.abs(L[0] @ one).max() < 1e-13
    assert nv == len(vmap)


@pytest.mark.parametrize("P", [4, 8])
def test_deformed_square_area_and_first_moment(P):
    """The deformation fixes the boundary of the unit square, so the curved
    mesh still covers it: sum of w|J| = 1 and sum of w|J| x1 = 1/2."""
    mesh = inputs.square_mesh_2d(3, 3, P, curved=True)
    area = mom = 0.0
    for (shape, PP, cv), el in twod._blocks(mesh).items():
        el = np.array(el)
        X = twod._verts(mesh, shape, el)
        ref = twod.reference(shape, PP, PP + 2)
        g = twod.block_metrics(shape, PP, PP + 2, X, bool(cv), 1)
        x = twod.block_points(shape, X, bool(cv), 1, ref["xi"])
        area += g["wJ"].sum()
        mom += (g["wJ"] * x[0]).sum()
    tol = 1e-6 if P == 4 else 1e-10
    assert abs(area - 1.0) < tol and abs(mom - 0.5) < tol


@pytest.mark.parametrize("P", [1, 3, 6])
def test_collocated_form_equals_plain_form(P):
    mesh = inputs.square_mesh_2d(2, 2, P, curved_rule="x_half")
    co, _ = twod.layout(mesh)
    x = inputs.random_coefficients(5, co)
    a = twod.apply("helmholtz", mesh, x, 1.7)
    b = twod.apply("helmholtz_collocated", mesh, x, 1.7)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_helmholtz_is_laplacian_plus_lambda_mass_and_symmetric():
    mesh = inputs.square_mesh_2d(2, 2, 3, curved=True)
    co, _ = twod.layout(mesh)
    x = inputs.random_coefficients(6, co)
    h = twod.apply("helmholtz", mesh, x, 2.5)
    assert np.allclose(h, twod.apply("laplacian", mesh, x, 0.0) + 2.5 * twod.apply("mass", mesh, x), atol=1e-13)
    X = twod._verts(mesh, TRI, np.array([1]))
    M, L = twod.element_matrices(TRI, 3, 5, X, True, 1)
    assert np.allclose(M, M.transpose(0, 2, 1), atol=1e-15) and np.allclose(L, L.transpose(0, 2, 1), atol=1e-13)
    assert np.linalg.eigvalsh(M[0]).min() > 0


# planted mistakes (on the CPU): each must be caught by a pin above
def _fails(fn, *args):
    with pytest.raises((AssertionError, np.linalg.LinAlgError)):
        fn(*args)


def test_mutation_unhalved_radau_weights_is_caught(monkeypatch):
    import oracle.quadrature as oq
    orig = twod.shape_rule
    monkeypatch.setattr(twod, "shape_rule", lambda s, Q: orig(s, Q) if s == QUAD else
                        [orig(s, Q)[0], oq.grj(Q, 1)])
    _fails(test_triangle_rule_integrates_monomials, 2)


def test_mutation_shifted_collapsed_coordinate_is_caught(monkeypatch):
    monkeypatch.setattr(twod, "eta_from_xi", lambda s, a, b: (a, b) if s == QUAD else
                        (2.0 * (1.0 + a) / (1.0 - b), b))
    _fails(test_vertex_modes_are_a_partition_of_unity, TRI)


def test_mutation_transposed_inverse_jacobian_is_caught(monkeypatch):
    orig = twod.block_metrics

    def bad(*a):
        g = orig(*a)
        g["Jinv"] = g["Jinv"].transpose(0, 1, 3, 2)
        return g
    monkeypatch.setattr(twod, "block_metrics", bad)
    _fails(test_laplacian_energy_of_linear_functions, TRI, 3)


def test_mutation_dropped_cross_metric_term_is_caught(monkeypatch):
    orig = twod.helmholtz_collocated_block

    def bad(shape, P, Q, X, curved, kind, uh, lam):
        # the collocated form with G_12 = 0 (evaluated through a sheared copy of the metric)
        ref = twod.reference(shape, P, Q)
        g = twod.block_metrics(shape, P, Q, X, curved, kind)
        u = uh @ ref["B"].T
        U = u.reshape(-1, Q, Q)
        D1, D2 = ref["D1"]
        v = np.stack([np.einsum("im,emj->eij", D1, U), np.einsum("jm,eim->eij", D2, U)]).reshape(2, len(X), -1)
        Gx = np.einsum("elda,elai->eldi", ref["T"][None].repeat(len(X), 0), g["Jinv"])
        G = np.einsum("el,eldi,elki->eldk", g["wJ"], Gx, Gx)
        w = np.stack([G[:, :, 0, 0] * v[0], G[:, :, 1, 1] * v[1]]).reshape(2, len(X), Q, Q)
        up = (np.einsum("mi,emj->eij", D1, w[0]) + np.einsum("mj,eim->eij", D2, w[1])).reshape(u.shape)
        return (up + lam * g["wJ"] * u) @ ref["B"]
    monkeypatch.setattr(twod, "helmholtz_collocated_block", bad)
    _fails(test_collocated_form_equals_plain_form, 3)
    assert orig is not bad
