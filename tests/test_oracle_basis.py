"""Pins of the oracle's modal bases: mode counts, partition of unity, vertex
interpolation, polynomial span, linear independence, and the complex-step
derivative against finite differences."""
import itertools

import numpy as np
import pytest

from oracle import basis

SHAPES = [0, 1, 2, 3]


def random_points(shape, n, seed=0):
    """Uniform random points strictly inside the reference element."""
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < n:
        x = rng.uniform(-1, 1, 3)
        inside = {0: True,
                  1: x[0] + x[2] < 0,
                  2: x[0] + x[2] < 0 and x[1] + x[2] < 0,
                  3: x.sum() < -1}[shape]
        if inside:
            pts.append(x)
    return np.array(pts).T


def closed_form_count(shape, P):
    # counted directly from the topology: vertices + edges + faces + interior
    if shape == 0:
        return 8 + 12 * (P - 1) + 6 * (P - 1) ** 2 + (P - 1) ** 3
    tri = (P - 1) * (P - 2) // 2
    if shape == 1:
        return 6 + 9 * (P - 1) + 2 * tri + 3 * (P - 1) ** 2 + (P - 1) * tri
    if shape == 2:
        interior = sum((P - 1 - r) ** 2 for r in range(1, P)) if P > 1 else 0
        return 5 + 8 * (P - 1) + (P - 1) ** 2 + 4 * tri + interior
    return 4 + 6 * (P - 1) + 4 * tri + (P - 1) * (P - 2) * (P - 3) // 6


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("P", range(1, 11))
def test_mode_counts(shape, P):
    ml = basis.modes(shape, P)
    assert len(ml) == basis.n_modes(shape, P) == closed_form_count(shape, P)
    keys = [basis.slot_key(shape, m) for m in ml]
    assert len(set(keys)) == len(keys)
    assert keys == sorted(keys)


def _vertex_modes(shape, P):
    ml = basis.modes(shape, P)
    return [i for i, m in enumerate(ml) if all(f[0] in ("1", "L", "R") for f in m)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("P", [1, 3, 5])
def test_vertex_modes_partition_of_unity(shape, P):
    x = random_points(shape, 50)
    B = basis.evaluate(shape, P, *x)
    vm = _vertex_modes(shape, P)
    assert len(vm) == len(basis.REF_VERTS[shape])
    np.testing.assert_allclose(B[:, vm].sum(axis=1), 1.0, atol=1e-14)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("P", [1, 2, 4])
def test_vertex_interpolation(shape, P):
    """Each vertex mode is 1 at its own vertex and 0 at the others; all other
    modes vanish at every vertex (approached from inside: collapsed vertices
    are singular points of the eta map)."""
    V = np.array(basis.REF_VERTS[shape], dtype=float)
    centre = V.mean(axis=0)
    pts = (V + 1e-9 * (centre - V)).T
    B = basis.evaluate(shape, P, *pts)
    vm = _vertex_modes(shape, P)
    sub = B[:, vm]
    # a permutation matrix up to O(1e-8)
    assert np.allclose(np.sort(sub, axis=1)[:, -1], 1.0, atol=1e-7)
    assert np.allclose(np.sort(sub, axis=0)[-1, :], 1.0, atol=1e-7)
    others = np.delete(B, vm, axis=1)
    if others.size:
        assert np.abs(others).max() < 1e-7


def _monomials(shape, P):
    out = []
    for a, b, c in itertools.product(range(P + 1), repeat=3):
        if shape == 0:
            ok = True
        elif shape == 1:
            ok = a + c <= P
        else:
            ok = a + b + c <= P
        if ok:
            out.append((a, b, c))
    return out


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("P", [1, 2, 3, 4, 6])
def test_polynomial_span(shape, P):
    """hex: Q_P; prism: P_P(xi1,xi3) x P_P(xi2); tet: P_P (same dimension, so
    the spans are equal); pyramid: contains P_P."""
    nm = basis.n_modes(shape, P)
    x = random_points(shape, 3 * nm + 20, seed=P)
    B = basis.evaluate(shape, P, *x)
    # linear independence
    s = np.linalg.svd(B, compute_uv=False)
    assert s[-1] / s[0] > 1e-10
    mons = _monomials(shape, P)
    if shape != 2:
        assert len(mons) == nm
    for a, b, c in mons:
        f = x[0] ** a * x[1] ** b * x[2] ** c
        coef, *_ = np.linalg.lstsq(B, f, rcond=None)
        assert np.abs(B @ coef - f).max() < 1e-11, (a, b, c)


@pytest.mark.parametrize("shape", SHAPES)
def test_complex_step_matches_finite_difference(shape):
    P = 4
    x = random_points(shape, 7, seed=11)
    g = basis.complex_step_gradient(lambda a, b, c: basis.evaluate(shape, P, a, b, c), x)
    h = 1e-6
    for d in range(3):
        xp = x.copy(); xp[d] += h
        xm = x.copy(); xm[d] -= h
        fd = (basis.evaluate(shape, P, *xp) - basis.evaluate(shape, P, *xm)) / (2 * h)
        np.testing.assert_allclose(g[d], fd, atol=1e-7)


@pytest.mark.parametrize("shape", [1, 2, 3])
def test_eta_maps_are_inverse(shape):
    x = random_points(shape, 40, seed=3)
    eta = basis.eta_from_xi(shape, *x)
    back = basis.xi_from_eta(shape, *eta)
    np.testing.assert_allclose(np.array(back), x, atol=1e-13)
    assert np.all(np.abs(np.array(eta)) <= 1.0 + 1e-14)
