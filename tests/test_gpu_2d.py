"""Two-dimensional quadrilateral / triangle operators (the paper's
two-dimensional formulation, Sec. 2.2) through the C ABI against the 2-D
oracle.  FP64: relative infinity-norm error <= 1e-12 (the 3-D FP64 bound);
FP32: the 3-D FP32 bound fp32_tol(P).  Metric factors against the oracle's at
1e-13."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import twod  # noqa: E402
from paper_2604_04644_gb300 import inputs  # noqa: E402
from tests.test_gpu_parity import FP64_TOL, fp32_tol, rel_err  # noqa: E402

KIND = {"mass": 0, "laplacian": 1, "helmholtz": 2}


@pytest.fixture(scope="module")
def hp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_04644_gb300 import hp as _hp
    return _hp


def run2d(hp, mesh, opname, x, lam, dtype=0):
    h = hp.hp_mesh2d_create(mesh, 0)
    try:
        co, po = hp.hp_mesh2d_layout(h, mesh["n_elem"])
        tdt = torch.float64 if dtype == hp.HP_FP64 else torch.float32
        xt = torch.tensor(x, device="cuda:0", dtype=tdt)
        y = torch.full((int(co[-1]),), float("nan"), device="cuda:0", dtype=tdt)
        hp.hp_op2d_apply(h, KIND[opname], dtype, lam, xt, y)
        hp.hp_mesh2d_sync(h)
        return y.double().cpu().numpy(), co, po
    finally:
        hp.hp_mesh2d_destroy(h)


@pytest.mark.parametrize("P", [1, 2, 3, 4, 6, 8, 10])
@pytest.mark.parametrize("opname", ["mass", "laplacian", "helmholtz"])
def test_fp64_matches_oracle(hp, P, opname):
    mesh = inputs.square_mesh_2d(3, 3, P, curved_rule="x_half")
    co, _ = twod.layout(mesh)
    x = inputs.random_coefficients(200 + P, co)
    y, co2, _ = run2d(hp, mesh, opname, x, 1.3)
    assert np.array_equal(co, co2)
    ref = twod.apply(opname, mesh, x, 1.3)
    assert rel_err(y, ref) <= FP64_TOL, rel_err(y, ref)


@pytest.mark.parametrize("opname", ["mass", "helmholtz"])
def test_fp32_matches_oracle(hp, opname):
    for P in (2, 5, 9):
        mesh = inputs.square_mesh_2d(4, 3, P, curved_rule="x_half")
        co, _ = twod.layout(mesh)
        x = inputs.random_coefficients(300 + P, co)
        x32 = x.astype(np.float32).astype(np.float64)
        y, _, _ = run2d(hp, mesh, opname, x, 0.9, hp.HP_FP32)
        assert rel_err(y, twod.apply(opname, mesh, x32, 0.9)) <= fp32_tol(P)


def test_p_adaptive_mesh_and_ragged_groups(hp):
    """Orders 1..10 drawn per element (many small blocks, groups of elements
    that do not fill a CTA), curved everywhere."""
    mesh = inputs.square_mesh_2d(6, 5, (1, 10), order_seed=3, curved=True)
    co, _ = twod.layout(mesh)
    x = inputs.random_coefficients(17, co)
    y, _, _ = run2d(hp, mesh, "helmholtz", x, 2.0)
    assert rel_err(y, twod.apply("helmholtz", mesh, x, 2.0)) <= FP64_TOL


@pytest.mark.parametrize("cells,P", [("quad", 4), ("tri", 6)])
def test_large_block_sampled(hp, cells, P):
    """Tens of thousands of elements of one shape (many CTAs, a persistent
    loop over groups): sampled elements against the oracle."""
    mesh = inputs.square_mesh_2d(150, 100, P, cells=cells, curved=True)
    co, _ = twod.layout(mesh)
    x = inputs.random_coefficients(23, co)
    y, _, _ = run2d(hp, mesh, "helmholtz", x, 1.0)
    rng = np.random.default_rng(4)
    n = mesh["n_elem"]
    sample = np.unique(np.concatenate([rng.choice(n, 60, replace=False), [0, n - 1]]))
    ref = twod.apply("helmholtz", mesh, x, 1.0, elems=sample)
    idx = np.concatenate([np.arange(co[e], co[e + 1]) for e in sample])
    assert rel_err(y[idx], ref[idx]) <= FP64_TOL


@pytest.mark.parametrize("P", [2, 7])
def test_metric_factors_match_oracle(hp, P):
    mesh = inputs.square_mesh_2d(3, 2, P, curved_rule="x_half")
    h = hp.hp_mesh2d_create(mesh, 0)
    try:
        co, po = hp.hp_mesh2d_layout(h, mesh["n_elem"])
        g = hp.hp_mesh2d_factors(h, po[-1])
    finally:
        hp.hp_mesh2d_destroy(h)
    for (shape, PP, cv), el in twod._blocks(mesh).items():
        el = np.array(el)
        ref = twod.geometric_factors_block(shape, PP, PP + 2, twod._verts(mesh, shape, el), bool(cv), 1)
        for t, e in enumerate(el):
            got = g[4 * po[e]: 4 * po[e + 1]].reshape(4, -1)
            assert np.abs(got - ref[t]).max() <= 1e-13 * np.abs(ref[t]).max()


def test_energy_of_linear_function_on_gpu(hp):
    """A GPU pin without the oracle: on an affine mesh the vertex-mode
    coefficients of x_1 (its vertex values) give u^T L u = area per element."""
    mesh = inputs.square_mesh_2d(3, 3, 4, curved=False)
    co, _ = twod.layout(mesh)
    u = np.zeros(co[-1])
    for e in range(mesh["n_elem"]):
        shape = int(mesh["shape"][e])
        ms = twod.modes(shape, 4)
        if shape == twod.QUAD:
            pairs = [((("L",), ("L",)), 0), ((("R",), ("L",)), 1), ((("R",), ("R",)), 2), ((("L",), ("R",)), 3)]
        else:
            pairs = [((("L",), ("L",)), 0), ((("R",), ("L",)), 1), ((("1",), ("R",)), 2)]
        for m, v in pairs:
            u[co[e] + ms.index(m)] = mesh["xy"][mesh["vert"][e][v]][0]
    y, _, _ = run2d(hp, mesh, "laplacian", u, 0.0)
    assert abs(np.dot(u, y) - 1.0) < 1e-12          # the unit square's area


def test_errors(hp):
    mesh = inputs.square_mesh_2d(2, 2, 3)
    bad = dict(mesh)
    bad["vert"] = mesh["vert"].copy()
    q = int(np.nonzero(mesh["shape"] == twod.TRI)[0][0])
    bad["vert"][q, [1, 2]] = bad["vert"][q, [2, 1]]           # clockwise triangle: |J| < 0
    with pytest.raises(hp.HpError) as ei:
        hp.hp_mesh2d_create(bad, 0)
    assert ei.value.status == hp.HP_ERR_GEOM
    h = hp.hp_mesh2d_create(mesh, 0)
    try:
        co, _ = hp.hp_mesh2d_layout(h, mesh["n_elem"])
        x = torch.zeros(int(co[-1]), device="cuda:0", dtype=torch.float64)
        y = torch.zeros_like(x)
        for kind, dt in ((hp.HP_BWDTRANS, hp.HP_FP64), (hp.HP_HELMHOLTZ, hp.HP_BF16)):
            with pytest.raises(hp.HpError) as ei:
                hp.hp_op2d_apply(h, kind, dt, 1.0, x, y)
            assert ei.value.status == hp.HP_ERR_UNSUPPORTED
        with pytest.raises(hp.HpError) as ei:
            hp.hp_op2d_apply(h, hp.HP_MASS, hp.HP_FP64, 1.0, x, x)
        assert ei.value.status == hp.HP_ERR_ARG
    finally:
        hp.hp_mesh2d_destroy(h)
