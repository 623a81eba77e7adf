"""GPU parity of the matrix-based strategy (HP_STRAT_MATRIX: stored per-element
dense H^e, Sec. 3.3 implementation strategies) with the CPU oracle, through the
C ABI.

FP64: 1e-12 relative (infinity norm), the operators' FP64 bar (the stored
matrix is the FP64 operator's own, exact up to its rounding; the matrix-vector
product adds at most N_P roundings per output).

FP32: per output m, |y_m - ref_m| <= 2 (N_P + 2) u (|H^e| |x|)_m with
u = 2^-24: one rounding of each stored entry to FP32 and at most N_P + 1
roundings of the accumulation (eight partial sums of N_P / 8 fused
multiply-adds, then their sum), to first order, with a factor 2 of margin.
|H^e| comes from the oracle's explicit element matrices.
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


def block_keys(mesh):
    """(shape, P, curved) of each block, in order of first appearance in user element order."""
    keys = []
    for k in zip(mesh["shape"].tolist(), mesh["P"].tolist(), mesh["curved"].tolist()):
        if k not in keys:
            keys.append(k)
    return keys


def apply(hp, mesh, kind, x, lam, dtype=0, strategy=None, lams=None):
    """Apply with HP_STRAT_MATRIX; with ``lams``, one apply per lambda on the same op."""
    strategy = hp.HP_STRAT_MATRIX if strategy is None else strategy
    h = hp.hp_mesh_create(mesh, 0)
    try:
        co, po, nc, nph = hp.hp_mesh_layout(h, mesh["n_elem"])
        op = hp.hp_op_create(h, KINDS[kind], strategy, dtype)
        try:
            tdt = torch.float64 if dtype == hp.HP_FP64 else torch.float32
            xt = torch.tensor(x, device="cuda:0", dtype=tdt)
            outs = []
            for la in (lams or [lam]):
                y = torch.full((nc,), float("nan"), device="cuda:0", dtype=tdt)
                hp.hp_op_apply(op, la, xt, y)
                hp.hp_op_sync(op)
                outs.append(y.double().cpu().numpy())
            return outs if lams else outs[0]
        finally:
            hp.hp_op_destroy(op)
    finally:
        hp.hp_mesh_destroy(h)


def abs_bound(mesh, x, lam, kind):
    """(|H^e| |x|) per output, from the oracle's explicit element matrices."""
    co, po = oracle_ops.layout(mesh)
    out = np.zeros(co[-1])
    for (shape, P, Q, cv), el in oracle_ops._blocks(mesh).items():
        el = np.array(el)
        X = oracle_ops._verts(mesh, shape, el)
        M, L = oracle_ops.element_matrices(shape, P, Q, X, bool(cv), mesh["deformation"])
        H = {"mass": M, "laplacian": L, "helmholtz": lam * M + L}[kind]
        idx = co[el][:, None] + np.arange(co[el[0] + 1] - co[el[0]])[None, :]
        out[idx] = np.einsum("emn,en->em", np.abs(H), np.abs(x[idx]))
    return out


@pytest.mark.parametrize("P", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("kind", ["mass", "laplacian", "helmholtz"])
def test_matrix_fp64_matches_oracle(hp, P, kind):
    mesh = inputs.slab_mesh(3, 3, 4, P, curved_rule="x_half")
    co, po = oracle_ops.layout(mesh)
    x = inputs.random_coefficients(500 + P, co)
    ref = oracle_ops.apply(kind, mesh, x, 1.9)
    y = apply(hp, mesh, kind, x, 1.9)
    assert not np.isnan(y).any()
    assert rel_err(y, ref) <= FP64_TOL, rel_err(y, ref)


@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_matrix_fp32_within_bound(hp, P):
    mesh = inputs.slab_mesh(3, 3, 4, P, curved_rule="x_half")
    co, po = oracle_ops.layout(mesh)
    x = inputs.random_coefficients(600 + P, co).astype(np.float32).astype(np.float64)
    ref = oracle_ops.apply("helmholtz", mesh, x, 1.9)
    y = apply(hp, mesh, "helmholtz", x, 1.9, dtype=hp.HP_FP32)
    npm = np.diff(co)
    per_out = np.repeat(npm, npm).astype(np.float64)          # N_P of each output's element
    bound = 2.0 * (per_out + 2.0) * 2.0 ** -24 * abs_bound(mesh, x, 1.9, "helmholtz")
    assert (np.abs(y - ref) <= bound).all(), np.max(np.abs(y - ref) / bound)


def test_matrix_lambda_change_rebuilds(hp):
    mesh = inputs.slab_mesh(2, 2, 4, 3, curved_rule="x_half")
    co, po = oracle_ops.layout(mesh)
    x = inputs.random_coefficients(41, co)
    lams = [1.0, 3.5, 1.0]
    ys = apply(hp, mesh, "helmholtz", x, None, lams=lams)
    for la, y in zip(lams, ys):
        assert rel_err(y, oracle_ops.apply("helmholtz", mesh, x, la)) <= FP64_TOL, la
    assert np.array_equal(ys[0], ys[2])


def test_matrix_large_blocks_run_sum_factorisation(hp):
    """P = 6: the hexahedron (343 modes) exceeds the stored-matrix size and runs
    sum factorisation; the other shapes are stored."""
    P = 6
    mesh = inputs.slab_mesh(2, 2, 4, P, curved_rule="x_half")
    co, po = oracle_ops.layout(mesh)
    x = inputs.random_coefficients(42, co)
    h = hp.hp_mesh_create(mesh, 0)
    try:
        op = hp.hp_op_create(h, KINDS["helmholtz"], hp.HP_STRAT_MATRIX, hp.HP_FP64)
        keys = block_keys(mesh)
        nb = len(keys)
        s = hp.hp_op_strategies(op, nb)
        expect = [hp.HP_STRAT_SUMFAC if k[0] == 0 else hp.HP_STRAT_MATRIX for k in keys]
        assert s.tolist() == expect, (s, keys)
        with pytest.raises(hp.HpError) as ei:
            hp.hp_op_strategies(op, nb, np.full(nb, hp.HP_STRAT_MATRIX))
        assert ei.value.status == hp.HP_ERR_UNSUPPORTED
        xt = torch.tensor(x, device="cuda:0", dtype=torch.float64)
        y = torch.full((len(x),), float("nan"), device="cuda:0", dtype=torch.float64)
        hp.hp_op_apply(op, 0.8, xt, y)
        hp.hp_op_sync(op)
        hp.hp_op_destroy(op)
    finally:
        hp.hp_mesh_destroy(h)
    assert rel_err(y.cpu().numpy(), oracle_ops.apply("helmholtz", mesh, x, 0.8)) <= FP64_TOL


def test_matrix_strategy_switch_graph_and_errors(hp):
    mesh = inputs.slab_mesh(2, 2, 4, 2, curved_rule="x_half")
    co, po = oracle_ops.layout(mesh)
    x = inputs.random_coefficients(43, co)
    ref = oracle_ops.apply("helmholtz", mesh, x, 2.0)
    h = hp.hp_mesh_create(mesh, 0)
    try:
        op = hp.hp_op_create(h, KINDS["helmholtz"], hp.HP_STRAT_SUMFAC, hp.HP_FP64)
        nb = len(block_keys(mesh))
        xt = torch.tensor(x, device="cuda:0", dtype=torch.float64)
        outs = []
        for strat in (hp.HP_STRAT_MATRIX, hp.HP_STRAT_SUMFAC, hp.HP_STRAT_MATRIX):
            hp.hp_op_strategies(op, nb, np.full(nb, strat))
            y = torch.full((len(x),), float("nan"), device="cuda:0", dtype=torch.float64)
            hp.hp_op_apply_graph(op, 2.0, xt, y)
            hp.hp_op_sync(op)
            outs.append(y.cpu().numpy())
        for o in outs:
            assert rel_err(o, ref) <= FP64_TOL
        assert np.array_equal(outs[0], outs[2])
        hp.hp_op_destroy(op)
        for kind, dtype in ((3, hp.HP_FP64), (2, hp.HP_TF32), (5, hp.HP_FP64)):
            with pytest.raises(hp.HpError) as ei:
                hp.hp_op_create(h, kind, hp.HP_STRAT_MATRIX, dtype)
            assert ei.value.status == hp.HP_ERR_UNSUPPORTED, (kind, dtype)
        op = hp.hp_op_create(h, KINDS["mass"], hp.HP_STRAT_SUMFAC, hp.HP_FP64)
        with pytest.raises(hp.HpError) as ei:
            hp.hp_op_strategies(op, nb, np.full(nb, hp.HP_STRAT_AUTO))
        assert ei.value.status == hp.HP_ERR_ARG
        hp.hp_op_destroy(op)
    finally:
        hp.hp_mesh_destroy(h)


def test_matrix_large_block_sampled(hp):
    """100 000 curved tets at P = 3 (a 320 MB stored block): sampled elements
    against the oracle, and the symmetry of H at full size."""
    mesh = inputs.replicated_mesh(3, 3, 100000, curved=True)
    co, po = oracle_ops.layout(mesh)
    x = inputs.random_coefficients(44, co)
    z = inputs.random_coefficients(45, co)
    h = hp.hp_mesh_create(mesh, 0)
    try:
        op = hp.hp_op_create(h, KINDS["helmholtz"], hp.HP_STRAT_MATRIX, hp.HP_FP64)
        ys = []
        for v in (x, z):
            vt = torch.tensor(v, device="cuda:0", dtype=torch.float64)
            y = torch.full((len(v),), float("nan"), device="cuda:0", dtype=torch.float64)
            hp.hp_op_apply(op, 1.0, vt, y)
            hp.hp_op_sync(op)
            ys.append(y.cpu().numpy())
        hp.hp_op_destroy(op)
    finally:
        hp.hp_mesh_destroy(h)
    sample = np.sort(np.random.default_rng(3).choice(mesh["n_elem"], 60, replace=False))
    ref = oracle_ops.apply("helmholtz", mesh, x, 1.0, elems=sample)
    idx = np.concatenate([np.arange(co[e], co[e + 1]) for e in sample])
    assert rel_err(ys[0][idx], ref[idx]) <= FP64_TOL
    assert abs(x @ ys[1] - z @ ys[0]) <= 1e-12 * abs(x @ ys[0])


def test_graph_schedule_may_store_matrices(hp):
    """FP64 graph-aware schedule of a p-adaptive mesh (P = 1..6): every block
    keeps a strategy built for it (stored matrices only up to 256 modes), and
    the scheduled graph matches the oracle at the FP64 bar, at a lambda other
    than the one scheduled with (stored Helmholtz matrices are rebuilt)."""
    from oracle.basis import n_modes
    mesh = inputs.slab_mesh(2, 2, 4, (1, 6), order_seed=5, curved_rule="x_half")
    keys = block_keys(mesh)
    nb = len(keys)
    co, po = oracle_ops.layout(mesh)
    uh = inputs.random_coefficients(46, co)
    h = hp.hp_mesh_create(mesh, 0)
    try:
        op = hp.hp_op_create(h, KINDS["helmholtz"], hp.HP_STRAT_SUMFAC, hp.HP_FP64)
        x = torch.tensor(uh, device="cuda:0", dtype=torch.float64)
        y = torch.zeros(len(uh), device="cuda:0", dtype=torch.float64)
        ms = hp.hp_op_schedule_graph(op, 1.0, x, y, 3, 1)
        assert ms > 0
        st = hp.hp_op_strategies(op, nb)
        assert np.isin(st, [hp.HP_STRAT_SUMFAC, hp.HP_STRAT_ELEMAT, hp.HP_STRAT_HYBRID, hp.HP_STRAT_MATRIX]).all()
        for (s, P, c), k in zip(keys, st):
            if k == hp.HP_STRAT_MATRIX:
                assert n_modes(s, P) <= 256
        y.fill_(float("nan"))
        hp.hp_op_apply_graph(op, 1.3, x, y)
        hp.hp_op_sync(op)
        hp.hp_op_destroy(op)
    finally:
        hp.hp_mesh_destroy(h)
    assert rel_err(y.cpu().numpy(), oracle_ops.apply("helmholtz", mesh, uh, 1.3)) <= FP64_TOL


def test_matrix_graph_after_lambda_change(hp):
    """A graph captured at lambda_1, a plain apply at lambda_2 (the stored
    Helmholtz matrices are rebuilt in place), then the graph at lambda_1 again:
    it must not replay on the lambda_2 matrices."""
    mesh = inputs.slab_mesh(2, 2, 4, 2, curved_rule="x_half")
    co, po = oracle_ops.layout(mesh)
    x = inputs.random_coefficients(47, co)
    h = hp.hp_mesh_create(mesh, 0)
    try:
        op = hp.hp_op_create(h, KINDS["helmholtz"], hp.HP_STRAT_MATRIX, hp.HP_FP64)
        xt = torch.tensor(x, device="cuda:0", dtype=torch.float64)
        y1 = torch.full((len(x),), float("nan"), device="cuda:0", dtype=torch.float64)
        y2 = torch.full((len(x),), float("nan"), device="cuda:0", dtype=torch.float64)
        hp.hp_op_apply_graph(op, 1.0, xt, y1)
        hp.hp_op_apply(op, 4.0, xt, y2)
        y1.fill_(float("nan"))
        hp.hp_op_apply_graph(op, 1.0, xt, y1)
        hp.hp_op_sync(op)
        hp.hp_op_destroy(op)
    finally:
        hp.hp_mesh_destroy(h)
    assert rel_err(y1.cpu().numpy(), oracle_ops.apply("helmholtz", mesh, x, 1.0)) <= FP64_TOL
    assert rel_err(y2.cpu().numpy(), oracle_ops.apply("helmholtz", mesh, x, 4.0)) <= FP64_TOL


def test_matrix_graph_after_block_apply_at_other_lambda(hp):
    """A graph captured at lambda_1, then hp_op_apply_block of every block at
    lambda_2 (each rebuilds that block's stored Helmholtz matrices in place),
    then the graph at lambda_1 again: both outputs match the oracle."""
    mesh = inputs.slab_mesh(2, 2, 4, 2, curved_rule="x_half")
    co, po = oracle_ops.layout(mesh)
    x = inputs.random_coefficients(53, co)
    nb = len(set(zip(mesh["shape"].tolist(), mesh["P"].tolist(), mesh["curved"].tolist())))
    h = hp.hp_mesh_create(mesh, 0)
    try:
        op = hp.hp_op_create(h, KINDS["helmholtz"], hp.HP_STRAT_MATRIX, hp.HP_FP64)
        xt = torch.tensor(x, device="cuda:0", dtype=torch.float64)
        y1 = torch.full((len(x),), float("nan"), device="cuda:0", dtype=torch.float64)
        y2 = torch.full((len(x),), float("nan"), device="cuda:0", dtype=torch.float64)
        hp.hp_op_apply_graph(op, 1.0, xt, y1)
        for b in range(nb):
            hp.hp_op_apply_block(op, b, 2.5, xt, y2)
        y1.fill_(float("nan"))
        hp.hp_op_apply_graph(op, 1.0, xt, y1)
        hp.hp_op_sync(op)
        hp.hp_op_destroy(op)
    finally:
        hp.hp_mesh_destroy(h)
    assert rel_err(y1.cpu().numpy(), oracle_ops.apply("helmholtz", mesh, x, 1.0)) <= FP64_TOL
    assert rel_err(y2.cpu().numpy(), oracle_ops.apply("helmholtz", mesh, x, 2.5)) <= FP64_TOL
