"""Batched p-adaptive apply: many (shape, P, curved) blocks in one operator,
the CUDA-graph launch, and the autotuned tile variants."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import operators as oracle_ops  # noqa: E402
from paper_2604_04644_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def hp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_04644_gb300 import hp as _hp
    return _hp


@pytest.fixture(scope="module")
def padaptive():
    # 3x3x8 cells, P ~ U{2..8} per element, affine for x < 0.5, curved otherwise
    return inputs.slab_mesh(3, 3, 8, (2, 8), order_seed=5, curved_rule="x_half")


def n_blocks(mesh):
    return len(set(zip(mesh["shape"].tolist(), mesh["P"].tolist(), mesh["curved"].tolist())))


def test_padaptive_matches_oracle_all_paths(hp, padaptive):
    mesh = padaptive
    h = hp.hp_mesh_create(mesh, 0)
    try:
        co, po, nc, nph = hp.hp_mesh_layout(h, mesh["n_elem"])
        uh = inputs.random_coefficients(31, co)
        ref = oracle_ops.apply("helmholtz", mesh, uh, 1.0)
        op = hp.hp_op_create(h, hp.HP_HELMHOLTZ)
        x = torch.tensor(uh, device="cuda:0")
        y0 = torch.full((nc,), np.nan, device="cuda:0", dtype=torch.float64)
        hp.hp_op_apply(op, 1.0, x, y0)
        hp.hp_op_sync(op)
        a = y0.cpu().numpy()
        assert np.abs(a - ref).max() <= 1e-12 * np.abs(ref).max()
        # graph launch: same kernels, same per-element arithmetic -> bitwise equal
        y1 = torch.full_like(y0, np.nan)
        hp.hp_op_apply_graph(op, 1.0, x, y1)
        hp.hp_op_apply_graph(op, 1.0, x, y1)
        hp.hp_op_sync(op)
        assert torch.equal(y0, y1)
        # new output pointer rebuilds the graph
        y2 = torch.full_like(y0, np.nan)
        hp.hp_op_apply_graph(op, 1.0, x, y2)
        hp.hp_op_sync(op)
        assert torch.equal(y0, y2)
        # every tile variant gives the same bits
        nb = n_blocks(mesh)
        for t in range(3):
            hp.hp_op_tiles(op, nb, np.full(nb, t))
            y3 = torch.full_like(y0, np.nan)
            hp.hp_op_apply(op, 1.0, x, y3)
            hp.hp_op_sync(op)
            assert torch.equal(y0, y3), t
        # autotune picks valid tiles; the result is unchanged
        y4 = torch.empty_like(y0)
        hp.hp_op_tune(op, 1.0, x, y4)
        tiles = hp.hp_op_tiles(op, nb)
        assert tiles.min() >= 0 and tiles.max() <= 2
        y5 = torch.full_like(y0, np.nan)
        hp.hp_op_apply_graph(op, 1.0, x, y5)
        hp.hp_op_sync(op)
        assert torch.equal(y0, y5)
        hp.hp_op_destroy(op)
    finally:
        hp.hp_mesh_destroy(h)


def test_tiles_argument_checks(hp, padaptive):
    h = hp.hp_mesh_create(padaptive, 0)
    try:
        op = hp.hp_op_create(h, hp.HP_MASS)
        nb = n_blocks(padaptive)
        # a new operator starts every block on tile 1 (the 20 KB budget)
        assert (hp.hp_op_tiles(op, nb) == 1).all()
        with pytest.raises(hp.HpError):
            hp.hp_op_tiles(op, nb + 1)
        with pytest.raises(hp.HpError):
            hp.hp_op_tiles(op, nb, np.full(nb, 7))
        hp.hp_op_destroy(op)
    finally:
        hp.hp_mesh_destroy(h)


@pytest.mark.parametrize("kind", ["helmholtz", "laplacian", "mass"])
def test_persistent_worklist_is_bitwise_the_per_block_launch(hp, padaptive, kind):
    """hp_op_set_batching(op, 1): one persistent work-list launch over all the
    p-adaptive mesh's blocks (plain and graph-captured) gives the bits of the
    per-block launches (the same body per element), and matches the oracle;
    switching a block to another strategy returns the op to per-block launches."""
    kinds = {"helmholtz": hp.HP_HELMHOLTZ, "laplacian": hp.HP_LAPLACIAN, "mass": hp.HP_MASS}
    mesh = padaptive
    nb = n_blocks(mesh)
    h = hp.hp_mesh_create(mesh, 0)
    try:
        co, po, nc, nph = hp.hp_mesh_layout(h, mesh["n_elem"])
        uh = inputs.random_coefficients(37, co)
        op = hp.hp_op_create(h, kinds[kind])
        x = torch.tensor(uh, device="cuda:0")
        y0 = torch.full((nc,), np.nan, device="cuda:0", dtype=torch.float64)
        hp.hp_op_apply(op, 1.4, x, y0)
        hp.hp_op_set_batching(op, 1)
        y1 = torch.full_like(y0, np.nan)
        hp.hp_op_apply(op, 1.4, x, y1)
        y2 = torch.full_like(y0, np.nan)
        for _ in range(3):
            hp.hp_op_apply_graph(op, 1.4, x, y2)
        hp.hp_op_sync(op)
        assert torch.equal(y0, y1) and torch.equal(y0, y2)
        ref = oracle_ops.apply(kind, mesh, uh, 1.4)
        assert np.abs(y1.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
        hp.hp_op_strategies(op, nb, np.full(nb, hp.HP_STRAT_HYBRID))
        y3 = torch.full_like(y0, np.nan)
        hp.hp_op_apply(op, 1.4, x, y3)           # per-block launches again (hybrid blocks)
        hp.hp_op_sync(op)
        assert np.abs(y3.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
        hp.hp_op_destroy(op)
        op32 = hp.hp_op_create(h, hp.HP_HELMHOLTZ, hp.HP_STRAT_SUMFAC, hp.HP_FP32)
        with pytest.raises(hp.HpError) as ei:
            hp.hp_op_set_batching(op32, 1)
        assert ei.value.status == hp.HP_ERR_UNSUPPORTED
        hp.hp_op_destroy(op32)
    finally:
        hp.hp_mesh_destroy(h)
