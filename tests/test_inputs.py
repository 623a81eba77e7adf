"""The seeded input generators: slab-mesh counts, orientation, affine
consistency, and the counter-based random numbers."""
import numpy as np
import pytest

from paper_2604_04644_gb300 import inputs

AXIS = inputs.AXIS_VERTS


def _frame(mesh, e):
    s = int(mesh["shape"][e])
    X = mesh["xyz"][mesh["vert"][e][: inputs.N_VERTS[s]]]
    v = AXIS[s]
    return s, X, np.stack([X[v[d]] - X[0] for d in range(3)], axis=1)


def test_slab_counts_16_cube():
    m = inputs.slab_mesh(16, 16, 16, 4)
    counts = np.bincount(m["shape"], minlength=4)
    assert list(counts) == [1024, 2048, 6144, 6144]
    assert m["n_elem"] == 15360


def test_slab_counts_40_40_32():
    m = inputs.slab_mesh(40, 40, 32, (2, 8), order_seed=3, curved_rule="x_half")
    assert m["n_elem"] == 12800 + 25600 + 76800 + 76800
    assert set(np.unique(m["P"])) == set(range(2, 9))
    assert 0 < m["curved"].mean() < 1


@pytest.mark.parametrize("slabs", [(0,), (1,), (2,), (3,)])
def test_orientation_and_affine_consistency(slabs):
    m = inputs.slab_mesh(2, 2, 2, 2, slabs=slabs)
    vol = 0.0
    for e in range(m["n_elem"]):
        s, X, E = _frame(m, e)
        det = np.linalg.det(E)
        assert det > 0
        vol += det / 8.0 * (8.0, 4.0, 8.0 / 3.0, 4.0 / 3.0)[s]
        # every vertex is the affine image of its reference vertex
        ref = {0: [(-1, -1, -1), (1, -1, -1), (1, 1, -1), (-1, 1, -1), (-1, -1, 1), (1, -1, 1), (1, 1, 1), (-1, 1, 1)],
               1: [(-1, -1, -1), (1, -1, -1), (1, 1, -1), (-1, 1, -1), (-1, -1, 1), (-1, 1, 1)],
               2: [(-1, -1, -1), (1, -1, -1), (1, 1, -1), (-1, 1, -1), (-1, -1, 1)],
               3: [(-1, -1, -1), (1, -1, -1), (-1, 1, -1), (-1, -1, 1)]}[s]
        for k, xi in enumerate(ref):
            np.testing.assert_allclose(X[0] + E @ ((np.array(xi) + 1) / 2), X[k], atol=1e-15)
    assert vol == pytest.approx(1.0, rel=1e-14)


def test_random_coefficients_layout_independent():
    off = np.array([0, 5, 9, 20])
    a = inputs.random_coefficients(11, off)
    assert a.shape == (20,)
    assert np.all(a >= -1) and np.all(a < 1)
    # element 1, mode 2 does not depend on the other elements' sizes
    off2 = np.array([0, 3, 7, 30])
    b = inputs.random_coefficients(11, off2)
    assert a[5 + 2] == b[3 + 2]
    assert inputs.random_coefficients(12, off)[0] != a[0]


def test_splitmix64_reference_values():
    # SplitMix64 with state 0: the first outputs of the published generator
    # (state += golden gamma, then the mix); the first output is 0xE220A8397B1DCDAF.
    assert int(inputs.splitmix64(np.array([0], dtype=np.uint64))[0]) == 0xE220A8397B1DCDAF
