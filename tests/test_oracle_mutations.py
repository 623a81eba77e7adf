"""Plant plausible mistakes in the oracle (on the CPU) and check that at least
one pin catches each of them, so the pins are strong enough to trust."""
import numpy as np
import pytest

import oracle.jacobi as oj
import oracle.operators as ops
import oracle.quadrature as oq
from tests import test_oracle_operators as T_ops
from tests import test_oracle_quadrature as T_q
from tests import test_oracle_basis as T_b


@pytest.fixture(autouse=True)
def _clear_cache():
    ops.reference.cache_clear()
    yield
    ops.reference.cache_clear()


def _fails(fn, *args):
    with pytest.raises((AssertionError, np.linalg.LinAlgError)):
        fn(*args)


def test_dropped_duffy_scaling_is_caught(monkeypatch):
    orig = oq.grj
    monkeypatch.setattr(oq, "grj", lambda Q, a: (orig(Q, a)[0], orig(Q, a)[1] * 2.0))
    _fails(T_q.test_reference_volumes, 3, 4.0 / 3.0)


def test_wrong_bubble_degree_is_caught(monkeypatch):
    monkeypatch.setattr(oj, "psi", lambda n, z: oj.L(z) * oj.R(z) * oj.jacobi(n, 1.0, 1.0, z))
    _fails(T_b.test_polynomial_span, 3, 3)


def test_wrong_warp_parameter_is_caught(monkeypatch):
    def bad(s, r, z):
        if r == 0:
            return oj.L(z) ** s           # missing one power of L
        return oj.L(z) ** (s + 1) * oj.R(z) * oj.jacobi(r - 1, 2.0 * s + 1.0, 1.0, z)
    monkeypatch.setattr(oj, "warped", bad)
    _fails(T_b.test_polynomial_span, 3, 3)


def test_transposed_inverse_jacobian_is_caught(monkeypatch):
    orig = ops.block_metrics

    def bad(*a):
        g = orig(*a)
        g["Jinv"] = np.swapaxes(g["Jinv"], -1, -2)
        return g
    monkeypatch.setattr(ops, "block_metrics", bad)
    _fails(T_ops.test_p1_tet_textbook_matrices)


def test_missing_jacobian_determinant_is_caught(monkeypatch):
    orig = ops.block_metrics

    def bad(*a):
        g = orig(*a)
        g["wJ"] = g["wJ"] / g["detJ"]
        return g
    monkeypatch.setattr(ops, "block_metrics", bad)
    _fails(T_ops.test_volume_from_mass_of_constant, 0, 2)


def test_wrong_lagrange_derivative_is_caught(monkeypatch):
    orig = ops.lagrange_derivative_matrix
    monkeypatch.setattr(ops, "lagrange_derivative_matrix", lambda x: orig(x).T)
    _fails(T_ops.test_collocated_equals_plain, 3, True, 3)


def test_unweighted_geometry_projection_is_caught(monkeypatch):
    from tests import test_oracle_isoparametric as T_iso

    def bad(shape, P, Q):
        B = ops.reference(shape, P, Q)["B"]
        Qo, _ = np.linalg.qr(B)                        # least squares at the points, W dropped
        return Qo @ Qo.T
    monkeypatch.setattr(ops, "projection_operator", bad)
    _fails(T_iso.test_hex_projection_annihilates_the_next_legendre_polynomial, 4)


def test_transposed_iso_jacobian_is_caught(monkeypatch):
    from tests import test_oracle_isoparametric as T_iso
    orig = ops.isoparametric_jacobian
    monkeypatch.setattr(ops, "isoparametric_jacobian", lambda *a: np.swapaxes(orig(*a), -1, -2))
    _fails(T_iso.test_quadratic_map_is_reproduced_from_degree_two, 3)


def test_advection_without_jacobian_weight_is_caught(monkeypatch):
    from tests import test_oracle_adr as T_adr
    orig = ops.block_metrics

    def bad(*a):
        g = orig(*a)
        g["wJ"] = g["wJ"] / g["detJ"]
        return g
    monkeypatch.setattr(ops, "block_metrics", bad)
    _fails(T_adr.test_linear_function_against_one_gives_velocity_times_volume, 3)


def test_advection_with_transposed_roles_is_caught(monkeypatch):
    from tests import test_oracle_adr as T_adr
    orig = ops.element_advection_matrices
    monkeypatch.setattr(ops, "element_advection_matrices", lambda *a, **k: orig(*a, **k).transpose(0, 2, 1))
    _fails(T_adr.test_constants_are_annihilated, 1, True)
