"""GPU parity of the iso-parametric geometry (mesh option geometry = 1: the
curved elements' map projected onto their own degree-P expansion, Sec. 4
"iso-parametric" curved elements) against the oracle's projection, and a
GPU-side pin that needs no oracle: a quadratic map is in every expansion of
degree >= 2, so there the iso-parametric factors equal the analytic ones.

Tolerance.  The projection weights the points by the reference quadrature,
whose weights vanish towards the collapse points, so near those points the
projected map, and most of all d eta / d x (no weight factor damps it), is
sensitive to rounding.  iso_spread(shape, P) measures that sensitivity on the
oracle side alone: the largest relative difference per element between two
FP64 evaluations of the same definition (the oracle's, and one with the
QR columns reversed and barycentric collocation matrices), over the curved
elements of that shape, separately for the weighted factors (G, w|J|) and
for d eta / d x.  The GPU is a third such evaluation:
tolerance = max(1e-12, 20 iso_spread)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import operators as oracle_ops  # noqa: E402
from paper_2604_04644_gb300 import inputs  # noqa: E402
from tests.test_gpu_parity import FP64_TOL, OPS, rel_err  # noqa: E402


@pytest.fixture(scope="module")
def hp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_04644_gb300 import hp as _hp
    return _hp


_SPREAD = {}


def _bary(x):
    n = len(x)
    w = np.array([1.0 / np.prod([x[j] - x[k] for k in range(n) if k != j]) for j in range(n)])
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (w[j] / w[i]) / (x[i] - x[j])
        D[i, i] = -D[i].sum()
    return D


def _factors_from_J(ref, J):
    detJ = np.linalg.det(J)
    Jinv = np.linalg.inv(J)
    wJ = ref["W"][None, :] * detJ
    Gx = np.einsum("lda,elai->eldi", ref["T"], Jinv)
    G = np.einsum("el,eldi,elki->eldk", wJ, Gx, Gx)
    six = np.stack([G[:, :, 0, 0], G[:, :, 0, 1], G[:, :, 0, 2], G[:, :, 1, 1], G[:, :, 1, 2], G[:, :, 2, 2], wJ], 1)
    return six, Gx.transpose(0, 2, 3, 1).reshape(len(J), 9, -1)


def iso_spread(shape, P):
    """(weighted factors, d eta / d x): the two-evaluation spread described above."""
    if (shape, P) not in _SPREAD:
        mesh = inputs.slab_mesh(2, 2, 4, 1, curved_rule="x_half")
        nv = (8, 6, 5, 4)[shape]
        els = np.nonzero((mesh["shape"] == shape) & (mesh["curved"] == 1))[0]
        X = mesh["xyz"][mesh["vert"][els][:, :nv]]
        Q = P + 2
        ref = oracle_ops.reference(shape, P, Q)
        J1 = oracle_ops.isoparametric_jacobian(shape, P, Q, X, True, 1)
        sw = np.sqrt(ref["W"])
        Qo, _ = np.linalg.qr((sw[:, None] * ref["B"])[:, ::-1])
        x = oracle_ops.block_points(shape, X, True, 1, ref["xi"])
        xp = np.einsum("cel,lm,km->cek", x * sw, Qo, Qo) / sw
        U = xp.reshape(3, -1, Q, Q, Q)
        D = [_bary(z) for z in ref["nodes"]]
        v = np.stack([np.einsum("am,cemjk->ceajk", D[0], U), np.einsum("bm,ceimk->ceibk", D[1], U),
                      np.einsum("km,ceijm->ceijk", D[2], U)])
        J2 = np.einsum("elcd,lda->elca", v.reshape(3, 3, len(els), -1).transpose(2, 3, 1, 0), ref["T"])
        (s1, n1), (s2, n2) = _factors_from_J(ref, J1), _factors_from_J(ref, J2)
        rel = lambda a, b: max(np.abs(a[k] - b[k]).max() / np.abs(a[k]).max() for k in range(len(a)))
        _SPREAD[(shape, P)] = (rel(s1, s2), rel(n1, n2))
    return _SPREAD[(shape, P)]


def iso_tol(mesh, P, which=0):
    return max(FP64_TOL, 20 * max(iso_spread(int(s), P)[which] for s in set(mesh["shape"].tolist())))


def _mesh(P, geometry, deformation=1, n=2):
    mesh = inputs.slab_mesh(n, n, 4, P, curved_rule="x_half", deformation=deformation)
    mesh["geometry"] = geometry
    return mesh


def _factors(hp, mesh):
    h = hp.hp_mesh_create(mesh, 0)
    try:
        co, po, nc, nph = hp.hp_mesh_layout(h, mesh["n_elem"])
        g7, g9 = hp.hp_geom_copy(h, nph, want_deriv=True)
    finally:
        hp.hp_mesh_destroy(h)
    return po, g7, g9


@pytest.mark.parametrize("P", [1, 2, 3, 5, 8])
def test_iso_factors_match_oracle(hp, P):
    mesh = _mesh(P, 1)
    po, g7, g9 = _factors(hp, mesh)
    six, nine = oracle_ops.geometric_factors(mesh)
    for e in range(mesh["n_elem"]):
        sp = iso_spread(int(mesh["shape"][e]), P) if mesh["curved"][e] else (0.0, 0.0)
        t7, t9 = max(FP64_TOL, 20 * sp[0]), max(FP64_TOL, 20 * sp[1])
        a = g7[po[e] * 7: po[e + 1] * 7].reshape(7, -1)
        b = g9[po[e] * 9: po[e + 1] * 9].reshape(9, -1)
        assert np.abs(a - six[e]).max() <= t7 * np.abs(six[e]).max(), (e, t7)
        assert np.abs(b - nine[e]).max() <= t9 * np.abs(nine[e]).max(), (e, t9)


def test_iso_factors_converge_to_the_analytic_map(hp):
    """On the sine deformation the projection is not exact: the two
    geometries differ on the curved elements, by a factor of five less or more
    with every two orders (spectral convergence)."""
    d = []
    for P in (2, 4, 6):
        _, a7, _ = _factors(hp, _mesh(P, 0))
        _, i7, _ = _factors(hp, _mesh(P, 1))
        d.append(rel_err(i7, a7))
    assert d[0] > 1e-4 and d[1] < d[0] / 5 and d[2] < d[1] / 5, d


@pytest.mark.parametrize("P", [2, 3])
def test_quadratic_map_iso_equals_analytic_on_gpu(hp, P):
    _, a7, a9 = _factors(hp, _mesh(P, 0, deformation=2))
    _, i7, i9 = _factors(hp, _mesh(P, 1, deformation=2))
    assert rel_err(i7, a7) <= max(1e-11, 20 * max(iso_spread(s, P)[0] for s in range(4)))
    assert rel_err(i9, a9) <= max(1e-11, 20 * max(iso_spread(s, P)[1] for s in range(4)))


@pytest.mark.parametrize("op", ["helmholtz", "mass", "phys_deriv"])
@pytest.mark.parametrize("P", [2, 4])
def test_iso_operators_match_oracle(hp, op, P):
    mesh = _mesh(P, 1)
    co, po = oracle_ops.layout(mesh)
    data = inputs.random_coefficients(61, co) if op != "phys_deriv" else inputs.random_phys(61, po)
    h = hp.hp_mesh_create(mesh, 0)
    try:
        nc, nph = int(co[-1]), int(po[-1])
        o = hp.hp_op_create(h, OPS[op], hp.HP_STRAT_SUMFAC, hp.HP_FP64)
        x = torch.tensor(data, device="cuda:0", dtype=torch.float64)
        y = torch.full((3 * nph if op == "phys_deriv" else nc,), float("nan"), device="cuda:0",
                       dtype=torch.float64)
        hp.hp_op_apply(o, 1.3, x, y)
        hp.hp_op_sync(o)
        hp.hp_op_destroy(o)
    finally:
        hp.hp_mesh_destroy(h)
    ref = oracle_ops.apply(op, mesh, data, 1.3)
    assert rel_err(y.cpu().numpy(), ref) <= iso_tol(mesh, P, 1 if op == "phys_deriv" else 0)
