"""Pins of the oracle's iso-parametric geometry (the element map projected
onto the element's own degree-P expansion, Sec. 4 "iso-parametric" curved
elements): it reproduces every map already in the expansion space exactly
(affine maps at any P, the quadratic deformation from P = 2 on), it
converges spectrally to the smooth sine deformation as P grows, and the
element volumes it gives converge to the exact ones."""
import numpy as np
import pytest

from oracle import operators as ops
from paper_2604_04644_gb300 import inputs

SHAPES = (0, 1, 2, 3)


def _elements(shape, n=2, seed=0):
    """Vertex arrays (Ne, nv, 3) of a few elements of one shape from the slab
    construction on [0, 1]^3 (cells of side 1/2)."""
    mesh = inputs.slab_mesh(2, 2, 4, 1, curved=True, slabs=(shape,) * 4)
    nv = (8, 6, 5, 4)[shape]
    X = mesh["xyz"][mesh["vert"][:, :nv]]
    return X[np.random.default_rng(seed).choice(len(X), n, replace=False)]


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("P", [1, 3])
def test_affine_maps_are_reproduced(shape, P):
    X = _elements(shape)
    ref = ops.reference(shape, P, P + 2)
    J_iso = ops.isoparametric_jacobian(shape, P, P + 2, X, False, 0)
    J = ops.block_jacobian(shape, X, False, 0, ref["xi"])
    assert _rel(J_iso, J) <= 1e-11      # exact up to rounding


@pytest.mark.parametrize("shape", SHAPES)
def test_quadratic_map_is_reproduced_from_degree_two(shape):
    """x_i + 0.1 x_j x_k composed with the affine map is a quadratic in xi:
    inside every expansion of degree >= 2 (the pyramid's included); outside
    the tetrahedron's degree-1 expansion (the linear polynomials; the hex,
    prism and pyramid degree-1 spaces hold some bilinear terms)."""
    X = _elements(shape)
    for P in (1, 2, 3):
        ref = ops.reference(shape, P, P + 2)
        J_iso = ops.isoparametric_jacobian(shape, P, P + 2, X, True, 2)
        J = ops.block_jacobian(shape, X, True, 2, ref["xi"])
        if P == 1:
            if shape == 3:
                assert _rel(J_iso, J) > 1e-4
        else:
            assert _rel(J_iso, J) <= 1e-11, P


@pytest.mark.parametrize("shape", SHAPES)
def test_sine_deformation_converges_spectrally(shape):
    X = _elements(shape)
    errs = []
    for P in (2, 4, 6, 8):
        ref = ops.reference(shape, P, P + 2)
        J_iso = ops.isoparametric_jacobian(shape, P, P + 2, X, True, 1)
        errs.append(_rel(J_iso, ops.block_jacobian(shape, X, True, 1, ref["xi"])))
    assert all(b < 0.2 * a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-5, errs


def test_volumes_converge_to_the_exact_ones():
    """The mesh of the unit cube deformed by the sine map keeps volume 1 (the
    deformation maps [0,1]^3 onto itself... up to its boundary bending, so the
    reference is the analytic map's volume): the iso-parametric volumes tend to
    the analytic ones spectrally."""
    errs = []
    for P in (2, 4, 6):
        mesh = inputs.slab_mesh(2, 2, 4, P, curved=True)
        vol = {}
        for geometry in (0, 1):
            mesh["geometry"] = geometry
            six, _ = ops.geometric_factors(mesh)
            vol[geometry] = sum(float(s[6].sum()) for s in six)
        errs.append(abs(vol[1] - vol[0]) / vol[0])
    assert errs[1] < 0.1 * errs[0] and errs[2] < 0.1 * errs[1], errs


@pytest.mark.parametrize("P", [1, 2, 4, 6, 8])
def test_hex_projection_annihilates_the_next_legendre_polynomial(P):
    """On the hexahedron the expansion of degree P holds every polynomial of
    degree <= P in xi_1, and the Legendre polynomial L_{P+1}(xi_1) is
    L2-orthogonal to all of them: its L2 projection is zero (the GLL rule
    with P + 2 points integrates L_{P+1} times the degree-P modes exactly).
    A projection with the wrong weights (least squares without W, say) does
    not annihilate it.  Members of the space are reproduced."""
    from oracle.jacobi import jacobi
    ref = ops.reference(0, P, P + 2)
    Pi = ops.projection_operator(0, P, P + 2)
    f = jacobi(P + 1, 0.0, 0.0, ref["xi"][0])
    assert np.abs(Pi @ f).max() <= 1e-11 * np.abs(f).max()     # rounding; a wrong weight leaves O(1)
    g = ref["xi"][0] ** P * ref["xi"][2] ** (P // 2)
    assert np.abs(Pi @ g - g).max() <= 1e-12
