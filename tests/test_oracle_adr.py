"""Pins of the oracle's advection part of the linear advection-diffusion-
reaction operator (-div grad u + a . grad u + lambda u tested against the
basis; Sec. 2.2 names it among the operators the B^T {pointwise} B
decomposition covers).  C[m][n] = int phi_m (a . grad phi_n) with a constant
velocity a:
- a = 0 gives the Helmholtz operator;
- C annihilates constants (grad 1 = 0);
- tested with v = 1 against u = x_j, int a . grad x_j = a_j |element|
  (affine elements, where the quadrature is exact);
- on modes that vanish on the element boundary C is skew-symmetric:
  int phi_m a.grad phi_n + phi_n a.grad phi_m = int a.grad(phi_m phi_n)
  = boundary integral = 0 (affine elements, exact quadrature)."""
import numpy as np
import pytest

from oracle import basis
from oracle import operators as ops
from paper_2604_04644_gb300 import inputs

A = np.array([0.7, -1.3, 0.4])


def _elements(shape, curved=False, n=3):
    mesh = inputs.slab_mesh(2, 2, 4, 1, curved=curved, slabs=(shape,) * 4)
    nv = (8, 6, 5, 4)[shape]
    return mesh["xyz"][mesh["vert"][:, :nv]][:n]


def test_zero_velocity_is_helmholtz():
    mesh = inputs.slab_mesh(2, 2, 4, 3, curved_rule="x_half")
    co, _ = ops.layout(mesh)
    x = inputs.random_coefficients(9, co)
    a = ops.apply("adr", mesh, x, 1.7, adv=(0.0, 0.0, 0.0))
    h = ops.apply("helmholtz", mesh, x, 1.7)
    assert np.abs(a - h).max() <= 1e-14 * np.abs(h).max()


def _vertex_ones(shape, P):
    """Coefficients of u = 1: the vertex modes sum to 1 (partition of unity)."""
    ml = basis.modes(shape, P)
    ref = ops.reference(shape, P, P + 2)
    B = ref["B"]
    one = np.linalg.lstsq(B, np.ones(B.shape[0]), rcond=None)[0]
    assert np.abs(B @ one - 1).max() < 1e-12
    return one


@pytest.mark.parametrize("shape", [0, 1, 2, 3])
@pytest.mark.parametrize("curved", [False, True])
def test_constants_are_annihilated(shape, curved):
    P = 3
    X = _elements(shape, curved)
    C = ops.element_advection_matrices(shape, P, P + 2, X, curved, 1, A)
    one = _vertex_ones(shape, P)
    assert np.abs(C @ one).max() <= 1e-12 * np.abs(C).max()


@pytest.mark.parametrize("shape", [0, 1, 2, 3])
def test_linear_function_against_one_gives_velocity_times_volume(shape):
    P = 2
    Q = P + 2
    X = _elements(shape)
    ref = ops.reference(shape, P, Q)
    C = ops.element_advection_matrices(shape, P, Q, X, False, 0, A)
    one = _vertex_ones(shape, P)
    from oracle.geometry import element_frame
    x = ops.block_points(shape, X, False, 0, ref["xi"])                   # (3, Ne, NQ)
    ref_vol = (8.0, 4.0, 8.0 / 3.0, 4.0 / 3.0)[shape]
    for j in range(3):
        for e in range(len(X)):
            uj = np.linalg.lstsq(ref["B"], x[j, e], rcond=None)[0]        # x_j is in every expansion
            vol = ref_vol * abs(np.linalg.det(element_frame(shape, X[e])[1])) / 8.0   # |det E| / 8 per unit
            assert abs(one @ C[e] @ uj - A[j] * vol) <= 1e-12 * abs(vol)


@pytest.mark.parametrize("shape", [0, 1, 2, 3])
def test_interior_block_is_skew_symmetric(shape):
    P = 4
    X = _elements(shape)
    C = ops.element_advection_matrices(shape, P, P + 2, X, False, 0, A)
    # modes that vanish on every face of the reference element, found by
    # evaluating them at random face points
    rng = np.random.default_rng(1)
    pts = []
    for _ in range(400):
        t = rng.uniform(-1, 1, 3)
        pts.append(t)
    pts = np.array(pts)
    faces = {0: lambda p: [np.array([p[0], p[1], s]) for s in (-1, 1)] + [np.array([p[0], s, p[2]]) for s in (-1, 1)]
             + [np.array([s, p[1], p[2]]) for s in (-1, 1)]}
    def on_faces(p):
        if shape == 0:
            return faces[0](p)
        if shape == 1:      # xi1 + xi3 = 0 slanted face, xi2 = +-1, xi3 = -1, xi1 = -1
            a, b = p[0], p[2]
            return [np.array([a, p[1], -a]), np.array([a, -1, b]), np.array([a, 1, b]), np.array([a, p[1], -1]),
                    np.array([-1, p[1], b])]
        if shape == 2:      # base xi3 = -1, faces xi1 = -1, xi2 = -1, xi1 = -xi3, xi2 = -xi3 (apex (-1,-1,1))
            return [np.array([p[0], p[1], -1]), np.array([-1, p[1], p[2]]), np.array([p[0], -1, p[2]]),
                    np.array([-p[2], p[1], p[2]]), np.array([p[0], -p[2], p[2]])]
        return [np.array([p[0], p[1], -1]), np.array([p[0], -1, p[2]]), np.array([-1, p[1], p[2]]),
                np.array([p[0], p[1], -1 - p[0] - p[1]])]
    vals = []
    for p in pts:
        for f in on_faces(p):
            vals.append(f)
    V = np.array(vals).T
    phi = basis.evaluate(shape, P, V[0], V[1], V[2])                        # (npts, NP)
    interior = np.nonzero(np.abs(phi).max(axis=0) < 1e-12)[0]
    assert len(interior) >= 1
    Ci = C[:, interior][:, :, interior]
    assert np.abs(Ci + Ci.transpose(0, 2, 1)).max() <= 1e-12 * np.abs(C).max()
    # the whole matrix is not skew (boundary modes carry the flux)
    assert np.abs(C + C.transpose(0, 2, 1)).max() > 1e-3 * np.abs(C).max()
