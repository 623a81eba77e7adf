"""Plain FP64 CPU oracle for the spectral/hp element operators.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

What it computes is the plain definition of each operator (paper Sec. 2.1,
the discrete elemental Helmholtz operator written as a sum over quadrature
points, and Eq. (mass) M = B^T W B): the modal basis is evaluated in closed
form at the quadrature points, its xi-gradient and the Jacobian of the
element map are taken by complex-step differentiation, and the sums over
modes and points are dense matrix products.  It shares no code with the
CUDA library; the only common module is the seeded input generator.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
(closed forms, invariants, brute-force cross-checks); none is unpinned.
"""
from . import jacobi, quadrature, basis, geometry, operators, mlp, assembly  # noqa: F401
