"""Tensor-core hybrid (HP_STRAT_HYBRID with HP_TF32 / HP_BF16) against the FP64
oracle, through the C ABI: u = B uhat and out = B^T u' as tcgen05 products
with the reference matrix B, the collocated derivatives and the metric between
them in FP32 on the CUDA cores (the collocated Helmholtz algorithm of
Sec. 3.3 with its two sum-factorised passes as dense tensor-core products).

Tolerance.  Per output coefficient: the first-order rounding bound of
tests/roundoff.py (hyb_bound: four roundings to the operand type and FP32
along the rest of the chain), checked element by element.  Normwise: the
same 8 u as the tensor-core elemental matrix (TF32 u = 2^-11, BF16 u = 2^-8).
Blocks beyond the hybrid's mode budget (N_P > 512 BF16, > 352 TF32) run FP32
sum factorisation and are held to its bound."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import operators as oracle_ops  # noqa: E402
from oracle.basis import n_modes  # noqa: E402
from paper_2604_04644_gb300 import inputs  # noqa: E402
from tests import roundoff  # noqa: E402
from tests.test_gpu_parity import OPS, fp32_tol, make_input, mixed_mesh, rel_err  # noqa: E402
from tests.test_gpu_tc import BF16_TOL, BF16_U, TF32_TOL, TF32_U, n_blocks  # noqa: E402

HYB_MAX = {"tf32": 352, "bf16": 512}


@pytest.fixture(scope="module")
def hp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_04644_gb300 import hp as _hp
    return _hp


def _dt(hp, prec):
    return hp.HP_TF32 if prec == "tf32" else hp.HP_BF16


def run_hyb(hp, mesh, opname, x, lam, prec, reps=1):
    h = hp.hp_mesh_create(mesh, 0)
    try:
        co, po, nc, nph = hp.hp_mesh_layout(h, mesh["n_elem"])
        op = hp.hp_op_create(h, OPS[opname], hp.HP_STRAT_HYBRID, _dt(hp, prec))
        try:
            strat = hp.hp_op_strategies(op, n_blocks(mesh))
            xt = torch.tensor(x, device="cuda:0", dtype=torch.float32)
            ys = []
            for _ in range(reps):
                y = torch.full((nc,), float("nan"), device="cuda:0", dtype=torch.float32)
                hp.hp_op_apply(op, lam, xt, y)
                hp.hp_op_sync(op)
                ys.append(y.double().cpu().numpy())
            return ys if reps > 1 else ys[0], strat
        finally:
            hp.hp_op_destroy(op)
    finally:
        hp.hp_mesh_destroy(h)


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("P", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("opname", ["mass", "laplacian", "helmholtz"])
def test_hybrid_matches_oracle(hp, P, opname, prec):
    """Mixed mesh (all four shapes, affine and curved halves, ragged tiles);
    at P = 6, 7 the hex blocks (343, 512 modes) take the hybrid's second
    output MMA (BF16) or fall back to FP32 sum factorisation (TF32 at 512)."""
    mesh = mixed_mesh(P)
    co, _ = oracle_ops.layout(mesh)
    x = make_input(mesh, opname, 700 + P)
    x32 = x.astype(np.float32).astype(np.float64)
    ref = oracle_ops.apply(opname, mesh, x32, 1.3)
    y, strat = run_hyb(hp, mesh, opname, x, 1.3, prec)
    assert not np.isnan(y).any()
    u = TF32_U if prec == "tf32" else BF16_U
    fits = np.array([n_modes(int(s), P) <= HYB_MAX[prec] for s in mesh["shape"]])
    want = hp.HP_STRAT_HYBRID if fits.all() else None
    if want is not None:
        assert (strat == hp.HP_STRAT_HYBRID).all()
    for s in range(4):
        els = np.nonzero(mesh["shape"] == s)[0]
        if len(els) == 0:
            continue
        idx = np.concatenate([np.arange(co[e], co[e + 1]) for e in els])
        tol = (TF32_TOL if prec == "tf32" else BF16_TOL) if fits[els[0]] else fp32_tol(P)
        assert rel_err(y[idx], ref[idx]) <= tol, (s, rel_err(y[idx], ref[idx]), tol)
    bound = np.where(np.repeat(fits, np.diff(co)), roundoff.hyb_bound(mesh, x32, 1.3, opname, u),
                     roundoff.sf32_bound(mesh, x32, 1.3, opname))
    assert (np.abs(y - ref) <= bound).all(), np.max(np.abs(y - ref) / bound)


@pytest.mark.parametrize("shape,P,curved,prec", [(3, 4, True, "bf16"), (2, 3, False, "tf32"), (0, 6, True, "tf32"),
                                                (0, 6, False, "bf16"), (0, 7, True, "bf16"), (1, 7, True, "bf16")])
def test_hybrid_large_block(hp, shape, P, curved, prec):
    """Many tiles of 128 elements (a ragged last one): sampled elements
    against the oracle; hex P6 / P7 and prism P7 exceed 256 modes (two output
    MMAs in BF16; TF32 hex P6 has 343 modes, K_P = 352)."""
    n = 3000 + 37
    mesh = inputs.replicated_mesh(shape, P, n, curved=curved)
    co, _ = oracle_ops.layout(mesh)
    x = inputs.random_coefficients(78, co)
    y, strat = run_hyb(hp, mesh, "helmholtz", x, 1.0, prec)
    assert strat.tolist() == [hp.HP_STRAT_HYBRID]
    rng = np.random.default_rng(2)
    sample = np.unique(np.concatenate([rng.choice(n, 40, replace=False), [0, 127, 128, n - 1]]))
    x32 = x.astype(np.float32).astype(np.float64)
    ref = oracle_ops.apply("helmholtz", mesh, x32, 1.0, elems=sample)
    idx = np.concatenate([np.arange(co[e], co[e + 1]) for e in sample])
    assert rel_err(y[idx], ref[idx]) <= (TF32_TOL if prec == "tf32" else BF16_TOL)


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_hybrid_single_element_and_repeat_is_bitwise(hp, prec):
    """One element per shape (a tile of one row); the hybrid has no atomics,
    so two applies agree bit for bit."""
    for shape in range(4):
        mesh = inputs.single_element_mesh(shape, 3, curved=True)
        x = make_input(mesh, "helmholtz", 19)
        ref = oracle_ops.apply("helmholtz", mesh, x.astype(np.float32).astype(np.float64), 0.7)
        (y1, y2), _ = run_hyb(hp, mesh, "helmholtz", x, 0.7, prec, reps=2)
        assert rel_err(y1, ref) <= (TF32_TOL if prec == "tf32" else BF16_TOL), shape
        assert np.array_equal(y1, y2)


def test_hybrid_strategy_gating(hp):
    """The hybrid is accepted for TF32 / BF16 blocks within its mode budget
    and refused beyond it (hex P8: 729 modes); hp_op_create puts such blocks
    on FP32 sum factorisation; building blocks stay sum-factorised only."""
    mesh = mixed_mesh(8, n=1)
    h = hp.hp_mesh_create(mesh, 0)
    try:
        keys = []
        for k in zip(mesh["shape"].tolist(), mesh["curved"].tolist()):
            if k not in keys:
                keys.append(k)
        for prec in ("tf32", "bf16"):
            op = hp.hp_op_create(h, hp.HP_HELMHOLTZ, hp.HP_STRAT_HYBRID, _dt(hp, prec))
            strat = hp.hp_op_strategies(op, len(keys))
            want = [hp.HP_STRAT_HYBRID if n_modes(s, 8) <= HYB_MAX[prec] else hp.HP_STRAT_SUMFAC for s, _ in keys]
            assert strat.tolist() == want
            with pytest.raises(hp.HpError) as ei:
                hp.hp_op_strategies(op, len(keys), np.full(len(keys), hp.HP_STRAT_HYBRID))
            assert ei.value.status == hp.HP_ERR_UNSUPPORTED
            hp.hp_op_destroy(op)
        with pytest.raises(hp.HpError) as ei:
            hp.hp_op_create(h, hp.HP_BWDTRANS, hp.HP_STRAT_HYBRID, hp.HP_BF16)
        assert ei.value.status == hp.HP_ERR_UNSUPPORTED
    finally:
        hp.hp_mesh_destroy(h)


def test_hybrid_in_graph_and_mixed_strategies(hp):
    """Per-block strategies mixing the tensor-core elemental matrix, the
    tensor-core hybrid and FP32 sum factorisation, launched as the concurrent
    graph (the hybrid's point vectors are per-block ranges of one buffer):
    equal to the same strategies applied block after block."""
    mesh = mixed_mesh(4)
    nb = n_blocks(mesh)
    co, _ = oracle_ops.layout(mesh)
    x = inputs.random_coefficients(31, co)
    h = hp.hp_mesh_create(mesh, 0)
    try:
        nc = int(co[-1])
        op = hp.hp_op_create(h, hp.HP_HELMHOLTZ, hp.HP_STRAT_HYBRID, hp.HP_BF16)
        st = np.array([(hp.HP_STRAT_HYBRID, hp.HP_STRAT_ELEMAT, hp.HP_STRAT_SUMFAC)[i % 3] for i in range(nb)],
                      dtype=np.int32)
        hp.hp_op_strategies(op, nb, st)
        hp.hp_op_set_deterministic(op, 1)          # the elemental-matrix blocks' split tiles in a fixed order
        xt = torch.tensor(x, device="cuda:0", dtype=torch.float32)
        y1 = torch.full((nc,), float("nan"), device="cuda:0", dtype=torch.float32)
        y2 = torch.full((nc,), float("nan"), device="cuda:0", dtype=torch.float32)
        hp.hp_op_apply(op, 1.1, xt, y1)
        hp.hp_op_apply_graph(op, 1.1, xt, y2)
        hp.hp_op_apply_graph(op, 1.1, xt, y2)
        hp.hp_op_sync(op)
        hp.hp_op_destroy(op)
    finally:
        hp.hp_mesh_destroy(h)
    assert torch.equal(y1, y2)
    ref = oracle_ops.apply("helmholtz", mesh, x.astype(np.float32).astype(np.float64), 1.1)
    assert rel_err(y1.double().cpu().numpy(), ref) <= BF16_TOL
