"""The advection-diffusion-reaction operator on the GPU (the Helmholtz passes
with the advection term added at the points; Sec. 2.2 names this operator
among those the B^T {pointwise} B decomposition covers) against the oracle's
plain definition, through the C ABI."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import operators as oracle_ops  # noqa: E402
from paper_2604_04644_gb300 import inputs  # noqa: E402
from tests.test_gpu_parity import FP64_TOL, fp32_tol, mixed_mesh, rel_err  # noqa: E402

VEL = (0.7, -1.3, 0.4)


@pytest.fixture(scope="module")
def hp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_04644_gb300 import hp as _hp
    return _hp


def run_adr(hp, mesh, x, lam, vel, dtype=0, graph=False):
    h = hp.hp_mesh_create(mesh, 0)
    try:
        co, po, nc, nph = hp.hp_mesh_layout(h, mesh["n_elem"])
        op = hp.hp_op_create(h, hp.HP_ADVECTION_DIFFUSION_REACTION, hp.HP_STRAT_SUMFAC, dtype)
        try:
            hp.hp_op_set_advection(op, vel)
            tdt = torch.float64 if dtype == hp.HP_FP64 else torch.float32
            xt = torch.tensor(x, device="cuda:0", dtype=tdt)
            y = torch.full((nc,), float("nan"), device="cuda:0", dtype=tdt)
            (hp.hp_op_apply_graph if graph else hp.hp_op_apply)(op, lam, xt, y)
            hp.hp_op_sync(op)
            return y.double().cpu().numpy()
        finally:
            hp.hp_op_destroy(op)
    finally:
        hp.hp_mesh_destroy(h)


@pytest.mark.parametrize("P", [1, 2, 3, 4, 6, 8])
def test_adr_fp64_matches_oracle(hp, P):
    mesh = mixed_mesh(P)
    co, _ = oracle_ops.layout(mesh)
    x = inputs.random_coefficients(800 + P, co)
    ref = oracle_ops.apply("adr", mesh, x, 1.7, adv=VEL)
    y = run_adr(hp, mesh, x, 1.7, VEL)
    assert rel_err(y, ref) <= FP64_TOL, rel_err(y, ref)


@pytest.mark.parametrize("P", [2, 5])
def test_adr_fp32_and_graph(hp, P):
    mesh = mixed_mesh(P)
    co, _ = oracle_ops.layout(mesh)
    x = inputs.random_coefficients(900 + P, co)
    x32 = x.astype(np.float32).astype(np.float64)
    ref = oracle_ops.apply("adr", mesh, x32, 0.9, adv=VEL)
    y = run_adr(hp, mesh, x, 0.9, VEL, dtype=hp.HP_FP32)
    assert rel_err(y, ref) <= fp32_tol(P)
    yg = run_adr(hp, mesh, x, 0.9, VEL, graph=True)
    assert rel_err(yg, oracle_ops.apply("adr", mesh, x, 0.9, adv=VEL)) <= FP64_TOL


def test_adr_zero_velocity_is_helmholtz_and_argument_checks(hp):
    mesh = mixed_mesh(3)
    co, _ = oracle_ops.layout(mesh)
    x = inputs.random_coefficients(5, co)
    y = run_adr(hp, mesh, x, 1.3, (0.0, 0.0, 0.0))
    ref = oracle_ops.apply("helmholtz", mesh, x, 1.3)
    assert rel_err(y, ref) <= FP64_TOL
    h = hp.hp_mesh_create(mesh, 0)
    try:
        op = hp.hp_op_create(h, hp.HP_HELMHOLTZ)
        with pytest.raises(hp.HpError) as ei:       # only the ADR operator has a velocity
            hp.hp_op_set_advection(op, VEL)
        assert ei.value.status == hp.HP_ERR_ARG
        hp.hp_op_destroy(op)
        for strat in (hp.HP_STRAT_ELEMAT, hp.HP_STRAT_MATRIX):
            with pytest.raises(hp.HpError) as ei:
                hp.hp_op_create(h, hp.HP_ADVECTION_DIFFUSION_REACTION, strat, hp.HP_FP64)
            assert ei.value.status == hp.HP_ERR_UNSUPPORTED
    finally:
        hp.hp_mesh_destroy(h)
