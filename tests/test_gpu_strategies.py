"""Elemental-matrix (StdMat, non-collocated) and hybrid strategies against
the oracle; all strategies agree with each other."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import operators as oracle_ops  # noqa: E402
from paper_2604_04644_gb300 import inputs  # noqa: E402
from tests.test_gpu_parity import OPS, FP64_TOL, fp32_tol, make_input, mixed_mesh, rel_err  # noqa: E402


@pytest.fixture(scope="module")
def hp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_04644_gb300 import hp as _hp
    return _hp


def run(hp, mesh, opname, x, lam, strategy, dtype):
    h = hp.hp_mesh_create(mesh, 0)
    try:
        co, po, nc, nph = hp.hp_mesh_layout(h, mesh["n_elem"])
        op = hp.hp_op_create(h, OPS[opname], strategy, dtype)
        try:
            tdt = torch.float64 if dtype == hp.HP_FP64 else torch.float32
            out_n = nph if opname == "bwd_trans" else nc
            xt = torch.tensor(x, device="cuda:0", dtype=tdt)
            y = torch.full((out_n,), float("nan"), device="cuda:0", dtype=tdt)
            hp.hp_op_apply(op, lam, xt, y)
            hp.hp_op_sync(op)
            return y.double().cpu().numpy()
        finally:
            hp.hp_op_destroy(op)
    finally:
        hp.hp_mesh_destroy(h)


STRATS = {"elemat": 1, "hybrid": 2}


@pytest.mark.parametrize("strategy", list(STRATS))
@pytest.mark.parametrize("P", [1, 3, 5, 8])
@pytest.mark.parametrize("opname", ["mass", "laplacian", "helmholtz", "bwd_trans", "iproduct_wrt_base"])
def test_fp64_strategy_matches_oracle(hp, strategy, P, opname):
    mesh = mixed_mesh(P)
    x = make_input(mesh, opname, 300 + P)
    ref = oracle_ops.apply(opname, mesh, x, 0.9)
    y = run(hp, mesh, opname, x, 0.9, STRATS[strategy], hp.HP_FP64)
    assert rel_err(y, ref) <= FP64_TOL


@pytest.mark.parametrize("strategy", list(STRATS))
@pytest.mark.parametrize("P", [2, 6])
def test_fp32_strategy_matches_oracle(hp, strategy, P):
    mesh = mixed_mesh(P)
    x = make_input(mesh, "helmholtz", 400 + P)
    x32 = x.astype(np.float32).astype(np.float64)
    ref = oracle_ops.apply("helmholtz", mesh, x32, 0.9)
    y = run(hp, mesh, "helmholtz", x, 0.9, STRATS[strategy], hp.HP_FP32)
    assert rel_err(y, ref) <= fp32_tol(P)


def test_high_order_elemat(hp):
    mesh = inputs.slab_mesh(1, 1, 4, 10, curved_rule="x_half")
    x = make_input(mesh, "helmholtz", 5)
    ref = oracle_ops.apply("helmholtz", mesh, x, 1.0)
    for s in (1, 2):
        assert rel_err(run(hp, mesh, "helmholtz", x, 1.0, s, hp.HP_FP64), ref) <= FP64_TOL


def test_derivative_blocks_need_sumfac(hp):
    mesh = mixed_mesh(2, n=1)
    h = hp.hp_mesh_create(mesh, 0)
    try:
        for s in (1, 2):
            with pytest.raises(hp.HpError) as ei:
                hp.hp_op_create(h, hp.HP_PHYSDERIV, s, hp.HP_FP64)
            assert ei.value.status == hp.HP_ERR_UNSUPPORTED
    finally:
        hp.hp_mesh_destroy(h)
