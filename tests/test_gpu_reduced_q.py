"""Reduced quadrature (mesh option quadrature = 1: Q - 1 Gauss-Radau-Jacobi
points in the collapsed directions) through the C ABI: the elemental-matrix
operators in FP64 against the oracle's reduced rule (1e-12), the metric
factors at its points (1e-13), the TF32 / BF16 tensor-core operators within
their normwise and per-output bounds, and a pin without the oracle: on
affine elements the reduced rule is exact, so its FP64 result equals the
full rule's sum-factorised one to rounding."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import operators as oracle_ops  # noqa: E402
from paper_2604_04644_gb300 import inputs  # noqa: E402
from tests import roundoff  # noqa: E402
from tests.test_gpu_parity import FP64_TOL, OPS, rel_err  # noqa: E402
from tests.test_gpu_tc import BF16_TOL, BF16_U, TF32_TOL, TF32_U  # noqa: E402


@pytest.fixture(scope="module")
def hp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_04644_gb300 import hp as _hp
    return _hp


def _mesh(P, rq=1, curved_rule="x_half", curved=True):
    mesh = inputs.slab_mesh(2, 2, 4, P, curved=curved, curved_rule=curved_rule)
    mesh["quadrature"] = rq
    return mesh


def apply(hp, mesh, opname, x, lam, strategy, dtype):
    h = hp.hp_mesh_create(mesh, 0)
    try:
        co, po, nc, nph = hp.hp_mesh_layout(h, mesh["n_elem"])
        op = hp.hp_op_create(h, OPS[opname], strategy, dtype)
        try:
            tdt = torch.float64 if dtype == hp.HP_FP64 else torch.float32
            xt = torch.tensor(x, device="cuda:0", dtype=tdt)
            y = torch.full((nc,), float("nan"), device="cuda:0", dtype=tdt)
            hp.hp_op_apply(op, lam, xt, y)
            hp.hp_op_sync(op)
            return y.double().cpu().numpy(), po
        finally:
            hp.hp_op_destroy(op)
    finally:
        hp.hp_mesh_destroy(h)


@pytest.mark.parametrize("P", [1, 2, 3, 5, 7])
@pytest.mark.parametrize("opname", ["mass", "laplacian", "helmholtz"])
def test_fp64_elemental_matrix_matches_oracle(hp, P, opname):
    mesh = _mesh(P)
    co, po = oracle_ops.layout(mesh)
    x = inputs.random_coefficients(800 + P, co)
    y, po2 = apply(hp, mesh, opname, x, 1.3, hp.HP_STRAT_ELEMAT, hp.HP_FP64)
    assert np.array_equal(po, po2)                       # point counts of the reduced rule
    assert rel_err(y, oracle_ops.apply(opname, mesh, x, 1.3)) <= FP64_TOL


@pytest.mark.parametrize("P", [2, 6])
def test_metric_factors_match_oracle(hp, P):
    mesh = _mesh(P)
    h = hp.hp_mesh_create(mesh, 0)
    try:
        co, po, nc, nph = hp.hp_mesh_layout(h, mesh["n_elem"])
        g7, _ = hp.hp_geom_copy(h, nph, want_deriv=False)
    finally:
        hp.hp_mesh_destroy(h)
    six, _ = oracle_ops.geometric_factors(mesh)
    for e in range(mesh["n_elem"]):
        a = g7[po[e] * 7: po[e + 1] * 7].reshape(7, -1)
        assert np.abs(a - six[e]).max() <= 1e-13 * np.abs(six[e]).max(), e


@pytest.mark.parametrize("P", [2, 4, 6])
def test_affine_reduced_rule_equals_full_rule(hp, P):
    mesh_f = _mesh(P, rq=0, curved_rule=None, curved=False)
    mesh_r = _mesh(P, rq=1, curved_rule=None, curved=False)
    co, _ = oracle_ops.layout(mesh_f)
    x = inputs.random_coefficients(900 + P, co)
    yf, _ = apply(hp, mesh_f, "helmholtz", x, 0.8, hp.HP_STRAT_SUMFAC, hp.HP_FP64)
    yr, _ = apply(hp, mesh_r, "helmholtz", x, 0.8, hp.HP_STRAT_ELEMAT, hp.HP_FP64)
    assert rel_err(yr, yf) <= FP64_TOL


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("P", [2, 4, 6])
def test_tensor_core_matches_oracle(hp, prec, P):
    """Blocks of at most 256 modes (P = 6: tets, pyramids, prisms and hexes
    all fit except the hex's 343 -- the mesh keeps P = 6 hexes out)."""
    mesh = _mesh(P)
    if P == 6:
        mesh = inputs.subset_mesh(mesh, np.nonzero(mesh["shape"] != 0)[0])
    co, _ = oracle_ops.layout(mesh)
    x = inputs.random_coefficients(950 + P, co)
    x32 = x.astype(np.float32).astype(np.float64)
    dt = hp.HP_TF32 if prec == "tf32" else hp.HP_BF16
    y, _ = apply(hp, mesh, "helmholtz", x, 1.1, hp.HP_STRAT_ELEMAT, dt)
    ref = oracle_ops.apply("helmholtz", mesh, x32, 1.1)
    assert rel_err(y, ref) <= (TF32_TOL if prec == "tf32" else BF16_TOL)
    bound = roundoff.tc_bound(mesh, x32, 1.1, "helmholtz", TF32_U if prec == "tf32" else BF16_U)
    assert (np.abs(y - ref) <= bound).all(), np.max(np.abs(y - ref) / bound)


def test_reduced_rule_gating(hp):
    mesh = _mesh(3)
    h = hp.hp_mesh_create(mesh, 0)
    try:
        for kind, strat, dt in ((hp.HP_HELMHOLTZ, hp.HP_STRAT_SUMFAC, hp.HP_FP64),
                                (hp.HP_HELMHOLTZ, hp.HP_STRAT_HYBRID, hp.HP_BF16),
                                (hp.HP_BWDTRANS, hp.HP_STRAT_ELEMAT, hp.HP_FP64)):
            with pytest.raises(hp.HpError) as ei:
                hp.hp_op_create(h, kind, strat, dt)
            assert ei.value.status == hp.HP_ERR_UNSUPPORTED
        op = hp.hp_op_create(h, hp.HP_MASS, hp.HP_STRAT_AUTO, hp.HP_FP64)      # AUTO: the elemental matrix
        nb = len(set(zip(mesh["shape"].tolist(), mesh["curved"].tolist())))
        assert (hp.hp_op_strategies(op, nb) == hp.HP_STRAT_ELEMAT).all()
        with pytest.raises(hp.HpError) as ei:
            hp.hp_op_strategies(op, nb, np.full(nb, hp.HP_STRAT_SUMFAC))
        assert ei.value.status == hp.HP_ERR_UNSUPPORTED
        hp.hp_op_destroy(op)
        with pytest.raises(hp.HpError) as ei:
            hp.hp_c0_create(h)
        assert ei.value.status == hp.HP_ERR_UNSUPPORTED
    finally:
        hp.hp_mesh_destroy(h)
    big = _mesh(8)                                  # hex P8: 729 modes, no tensor-core form
    h = hp.hp_mesh_create(big, 0)
    try:
        with pytest.raises(hp.HpError) as ei:
            hp.hp_op_create(h, hp.HP_HELMHOLTZ, hp.HP_STRAT_ELEMAT, hp.HP_BF16)
        assert ei.value.status == hp.HP_ERR_UNSUPPORTED
    finally:
        hp.hp_mesh_destroy(h)
    iso = _mesh(3)
    iso["geometry"] = 1
    with pytest.raises(hp.HpError) as ei:
        hp.hp_mesh_create(iso, 0)
    assert ei.value.status == hp.HP_ERR_UNSUPPORTED
