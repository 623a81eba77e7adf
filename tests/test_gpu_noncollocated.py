"""GPU parity of the non-collocated FP64 sum-factorised Laplacian / Helmholtz
(the form the paper's collocation study, Sec. 5, compares the collocated
approach against) with the CPU oracle and with the collocated kernel, through
the C ABI.

Both forms compute (lambda M + L) uhat of Sec. 2.2 exactly up to rounding (the
1-D factors have degree <= P < Q, so collocation differentiation of their
values is exact), so the FP64 bar of 1e-12 relative applies to both.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import operators as oracle_ops  # noqa: E402
from paper_2604_04644_gb300 import inputs  # noqa: E402

FP64_TOL = 1e-12
KINDS = {"mass": 0, "laplacian": 1, "helmholtz": 2}


@pytest.fixture(scope="module")
def hp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_04644_gb300 import hp as _hp
    return _hp


def rel_err(y, ref):
    return np.abs(y - ref).max() / max(np.abs(ref).max(), 1e-300)


def apply(hp, mesh, kind, x, lam, collocated, graph=False):
    h = hp.hp_mesh_create(mesh, 0)
    try:
        co, po, nc, nph = hp.hp_mesh_layout(h, mesh["n_elem"])
        op = hp.hp_op_create(h, KINDS[kind], hp.HP_STRAT_SUMFAC, hp.HP_FP64)
        try:
            hp.hp_op_set_collocated(op, collocated)
            xt = torch.tensor(x, device="cuda:0", dtype=torch.float64)
            y = torch.full((nc,), float("nan"), device="cuda:0", dtype=torch.float64)
            (hp.hp_op_apply_graph if graph else hp.hp_op_apply)(op, lam, xt, y)
            hp.hp_op_sync(op)
            return y.cpu().numpy()
        finally:
            hp.hp_op_destroy(op)
    finally:
        hp.hp_mesh_destroy(h)


@pytest.mark.parametrize("P", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("kind", ["laplacian", "helmholtz"])
def test_noncollocated_matches_oracle(hp, P, kind):
    """Mixed mesh (all four shapes, curved and affine blocks, ragged element groups)."""
    mesh = inputs.slab_mesh(3, 3, 4, P, curved_rule="x_half")
    co, po = oracle_ops.layout(mesh)
    x = inputs.random_coefficients(300 + P, co)
    ref = oracle_ops.apply(kind, mesh, x, 1.3)
    y = apply(hp, mesh, kind, x, 1.3, False)
    assert not np.isnan(y).any()
    assert rel_err(y, ref) <= FP64_TOL, rel_err(y, ref)
    yc = apply(hp, mesh, kind, x, 1.3, True)
    assert rel_err(y, yc) <= FP64_TOL


@pytest.mark.parametrize("P", [9, 10])
def test_noncollocated_high_order(hp, P):
    mesh = inputs.slab_mesh(1, 1, 4, P, curved_rule="x_half")
    co, po = oracle_ops.layout(mesh)
    x = inputs.random_coefficients(17, co)
    ref = oracle_ops.apply("helmholtz", mesh, x, 0.7)
    assert rel_err(apply(hp, mesh, "helmholtz", x, 0.7, False), ref) <= FP64_TOL


def test_noncollocated_single_elements(hp):
    """One element of each shape, affine and curved (a group with one element)."""
    for shape in range(4):
        for curved in (False, True):
            mesh = inputs.single_element_mesh(shape, 5, curved=curved)
            co, po = oracle_ops.layout(mesh)
            x = inputs.random_coefficients(3, co)
            ref = oracle_ops.apply("helmholtz", mesh, x, 0.3)
            assert rel_err(apply(hp, mesh, "helmholtz", x, 0.3, False), ref) <= FP64_TOL, (shape, curved)


def test_noncollocated_regular_blocks_sampled(hp):
    """Large regular (affine) single-shape blocks, the configuration of the
    collocation study: sampled elements against the oracle, and the whole
    output against the collocated kernel."""
    for shape in range(4):
        mesh = inputs.replicated_mesh(shape, 4, 20000, curved=False)
        co, po = oracle_ops.layout(mesh)
        x = inputs.random_coefficients(40 + shape, co)
        y = apply(hp, mesh, "helmholtz", x, 1.0, False)
        yc = apply(hp, mesh, "helmholtz", x, 1.0, True)
        assert rel_err(y, yc) <= FP64_TOL, shape
        sample = np.sort(np.random.default_rng(shape).choice(mesh["n_elem"], 40, replace=False))
        ref = oracle_ops.apply("helmholtz", mesh, x, 1.0, elems=sample)
        idx = np.concatenate([np.arange(co[e], co[e + 1]) for e in sample])
        assert rel_err(y[idx], ref[idx]) <= FP64_TOL, shape


def test_collocation_switch_graph_and_other_kinds(hp):
    mesh = inputs.slab_mesh(2, 2, 4, 3, curved_rule="x_half")
    co, po = oracle_ops.layout(mesh)
    x = inputs.random_coefficients(9, co)
    ref = oracle_ops.apply("helmholtz", mesh, x, 2.0)
    # the captured graph follows the switch
    h = hp.hp_mesh_create(mesh, 0)
    try:
        op = hp.hp_op_create(h, KINDS["helmholtz"], hp.HP_STRAT_SUMFAC, hp.HP_FP64)
        xt = torch.tensor(x, device="cuda:0", dtype=torch.float64)
        outs = []
        for coll in (True, False, True):
            y = torch.full((len(x),), float("nan"), device="cuda:0", dtype=torch.float64)
            hp.hp_op_set_collocated(op, coll)
            hp.hp_op_apply_graph(op, 2.0, xt, y)
            hp.hp_op_sync(op)
            outs.append(y.cpu().numpy())
        for o in outs:
            assert rel_err(o, ref) <= FP64_TOL
        assert np.array_equal(outs[0], outs[2])
        assert hp._lib.hp_op_set_collocated(op, 2) == hp.HP_ERR_ARG
        hp.hp_op_destroy(op)
        op32 = hp.hp_op_create(h, KINDS["helmholtz"], hp.HP_STRAT_SUMFAC, hp.HP_FP32)
        with pytest.raises(hp.HpError) as ei:
            hp.hp_op_set_collocated(op32, False)
        assert ei.value.status == hp.HP_ERR_UNSUPPORTED
        hp.hp_op_set_collocated(op32, True)
        hp.hp_op_destroy(op32)
    finally:
        hp.hp_mesh_destroy(h)
    # the mass operator has no derivative step: the switch leaves it bit for bit
    assert np.array_equal(apply(hp, mesh, "mass", x, 1.0, False), apply(hp, mesh, "mass", x, 1.0, True))
