"""Pins of the reduced quadrature (Q - 1 Gauss-Radau-Jacobi points in the
collapsed directions, Q = P + 2 elsewhere) against facts that do not come from
it: the reference volumes, exact integration of polynomials of degree 2Q - 4
against the Jacobi weight (numpy's Gauss-Legendre rule as the check), and the
mass and Laplacian matrices of affine elements, which the reduced rule still
integrates exactly (after the Duffy factor is absorbed into the weight their
integrands have degree <= 2P in each collapsed coordinate): equal to the full
rule's to rounding.  On curved elements the two rules differ by a quadrature
error."""
import numpy as np
import pytest

from oracle import operators as ops
from oracle import quadrature as oq
from oracle.basis import REF_VOLUME
from paper_2604_04644_gb300 import inputs


@pytest.fixture(autouse=True)
def _clear_cache():
    ops.reference.cache_clear()
    yield
    ops.reference.cache_clear()


@pytest.mark.parametrize("shape", [1, 2, 3])
@pytest.mark.parametrize("P", [1, 3, 6])
def test_point_counts_and_volumes(shape, P):
    ref = ops.reference(shape, P, P + 2, 1)
    Q = P + 2
    assert ref["dims"] == ((Q, Q, Q - 1) if shape in (1, 2) else (Q, Q - 1, Q - 1))
    assert ref["NQ"] == ops.n_points(shape, Q, 1)
    assert ref["W"].sum() == pytest.approx(REF_VOLUME[shape], rel=1e-14)


@pytest.mark.parametrize("alpha", [1, 2])
@pytest.mark.parametrize("Q", [3, 5, 8])
def test_radau_rule_degree(alpha, Q):
    """GRJ with Q - 1 points integrates x^k (1 - x)^alpha exactly for k <= 2Q - 4."""
    x, w = oq.grj(Q - 1, alpha)
    z, wz = np.polynomial.legendre.leggauss(Q + 4)
    for k in range(2 * Q - 3):
        exact = np.dot(wz, z ** k * (1 - z) ** alpha)
        assert abs(np.dot(w, x ** k) - exact) <= 1e-13 * max(1.0, abs(exact)), k


@pytest.mark.parametrize("shape", [1, 2, 3])
@pytest.mark.parametrize("P", [1, 2, 4, 6])
def test_affine_element_matrices_are_exact(shape, P):
    X = inputs.single_element_mesh(shape, P, curved=False)
    Xv = ops._verts(X, shape, np.array([0]))
    Mf, Lf = ops.element_matrices(shape, P, P + 2, Xv, False, 1)
    Mr, Lr = ops.element_matrices(shape, P, P + 2, Xv, False, 1, reduced=1)
    assert np.abs(Mr - Mf).max() <= 1e-14 * np.abs(Mf).max()
    assert np.abs(Lr - Lf).max() <= 1e-13 * np.abs(Lf).max()


def test_mesh_layout_and_apply():
    mesh = inputs.slab_mesh(2, 2, 4, 3, curved_rule="x_half")
    mesh["quadrature"] = 1
    co, po = ops.layout(mesh)
    npts = np.diff(po)
    want = [ops.n_points(int(s), 5, 1) for s in mesh["shape"]]
    assert np.array_equal(npts, want) and set(npts.tolist()) == {125, 100, 80}
    x = inputs.random_coefficients(4, co)
    m_r = ops.apply("mass", mesh, x)
    mesh0 = dict(mesh)
    mesh0["quadrature"] = 0
    m_f = ops.apply("mass", mesh0, x)
    aff = np.repeat(mesh["curved"] == 0, np.diff(co))
    assert np.abs(m_r - m_f)[aff].max() <= 1e-13 * np.abs(m_f).max()      # exact on affine elements
    assert np.abs(m_r - m_f)[~aff].max() > 1e-12 * np.abs(m_f).max()      # curved: a quadrature error


def test_mutation_wrong_jacobi_weight_is_caught(monkeypatch):
    orig = oq.grj
    monkeypatch.setattr(oq, "grj", lambda Q, a: orig(Q, 0) if a == 2 else orig(Q, a))
    ops.reference.cache_clear()
    with pytest.raises(AssertionError):
        test_point_counts_and_volumes(3, 2)


def test_mutation_reduced_rule_ignored_is_caught(monkeypatch):
    orig = oq.shape_rule
    monkeypatch.setattr(oq, "shape_rule", lambda s, Q, reduced=0: orig(s, Q, 0))
    ops.reference.cache_clear()
    with pytest.raises(AssertionError):
        test_point_counts_and_volumes(3, 3)
