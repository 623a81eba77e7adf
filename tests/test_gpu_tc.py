"""Tensor-core (tcgen05, TF32 and BF16) elemental-matrix operators against the
FP64 oracle, through the C ABI.

Tolerance (relative, infinity norm over the whole output vector):
TF32_TOL = 8 u with u = 2^-11, the unit roundoff of TF32 (10 stored mantissa
bits, round to nearest).  Each term of out_e = sum A_c^T M A_c' uhat carries
three TF32 roundings (the coefficient, the reference-matrix entry and the
metric-weighted point value V') and the rounding of the metric factor to FP16
(11 significant bits after a per-element power-of-two scale, so at most u as
well), so |error_m| <= 4 u (|A|^T |M| |A| |uhat|)_m to first order, plus FP32
accumulation (~1e-7).  The ratio of that absolute sum to ||out||_inf is the
cancellation factor; random-sign rounding errors keep the measured error near
1 u, and 8 u allows a cancellation factor of 2 at full correlation.  Blocks whose mode
count exceeds the tensor-memory budget (N_P > 256; BF16: > 320) run FP32 sum factorisation
and are held to the FP32 bound of test_gpu_parity.  BF16 (8 significant
bits) takes the same argument with u = 2^-8: BF16_TOL = 8 u.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import operators as oracle_ops  # noqa: E402
from paper_2604_04644_gb300 import inputs  # noqa: E402
from tests.test_gpu_parity import OPS, fp32_tol, make_input, mixed_mesh, rel_err  # noqa: E402

TF32_U = 2.0 ** -11
TF32_TOL = 8 * TF32_U
BF16_U = 2.0 ** -8          # 8 significant bits, round to nearest
BF16_TOL = 8 * BF16_U
MAX_TC_MODES = 256
# blocks an elemental-matrix operator puts on the tensor cores by default (BF16
# builds the form up to 512 modes, but those past 320 start on FP32 sum factorisation)
MAX_TC_MODES_PREC = {"tf32": 256, "bf16": 320}


@pytest.fixture(scope="module")
def hp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_04644_gb300 import hp as _hp
    return _hp


def n_blocks(mesh):
    return len(set(zip(mesh["shape"].tolist(), mesh["P"].tolist(), mesh["curved"].tolist())))


def run_tc(hp, mesh, opname, x, lam, dtype=None, force=False):
    h = hp.hp_mesh_create(mesh, 0)
    try:
        co, po, nc, nph = hp.hp_mesh_layout(h, mesh["n_elem"])
        op = hp.hp_op_create(h, OPS[opname], hp.HP_STRAT_ELEMAT, hp.HP_TF32 if dtype is None else dtype)
        try:
            if force:   # every block on the tensor-core elemental matrix (the BF16 blocks past 256 modes)
                hp.hp_op_strategies(op, n_blocks(mesh), np.full(n_blocks(mesh), hp.HP_STRAT_ELEMAT))
            strat = hp.hp_op_strategies(op, n_blocks(mesh))
            xt = torch.tensor(x, device="cuda:0", dtype=torch.float32)
            y = torch.full((nc,), float("nan"), device="cuda:0", dtype=torch.float32)
            hp.hp_op_apply(op, lam, xt, y)
            hp.hp_op_sync(op)
            return y.double().cpu().numpy(), strat
        finally:
            hp.hp_op_destroy(op)
    finally:
        hp.hp_mesh_destroy(h)


def per_shape_errors(mesh, co, y, ref):
    out = {}
    for s in range(4):
        els = np.nonzero(mesh["shape"] == s)[0]
        if len(els) == 0:
            continue
        idx = np.concatenate([np.arange(co[e], co[e + 1]) for e in els])
        out[s] = rel_err(y[idx], ref[idx])
    return out


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("P", [1, 2, 3, 4, 5, 6, 8])
@pytest.mark.parametrize("opname", ["mass", "laplacian", "helmholtz"])
def test_tensor_core_matches_oracle(hp, P, opname, prec):
    """Mixed mesh (all four shapes, affine and curved halves, ragged tiles):
    tensor-core blocks within TF32_TOL / BF16_TOL, FP32 sum-factorisation
    blocks within the FP32 bound."""
    mesh = mixed_mesh(P)
    co, _ = oracle_ops.layout(mesh)
    x = make_input(mesh, opname, 600 + P)
    x32 = x.astype(np.float32).astype(np.float64)
    ref = oracle_ops.apply(opname, mesh, x32, 1.3)
    y, strat = run_tc(hp, mesh, opname, x, 1.3, hp.HP_TF32 if prec == "tf32" else hp.HP_BF16)
    assert not np.isnan(y).any()
    from oracle.basis import n_modes
    errs = per_shape_errors(mesh, co, y, ref)
    for s, err in errs.items():
        tol = (TF32_TOL if prec == "tf32" else BF16_TOL) if n_modes(s, P) <= MAX_TC_MODES_PREC[prec] else fp32_tol(P)
        assert err <= tol, (s, err, tol)
    # per output: the first-order rounding bound of the form each block runs
    from tests import roundoff
    tc = roundoff.tc_bound(mesh, x32, 1.3, opname, TF32_U if prec == "tf32" else BF16_U)
    sf = roundoff.sf32_bound(mesh, x32, 1.3, opname)
    fits = np.repeat([n_modes(int(s), P) <= MAX_TC_MODES_PREC[prec] for s in mesh["shape"]], np.diff(co))
    bound = np.where(fits, tc, sf)
    assert (np.abs(y - ref) <= bound).all(), np.max(np.abs(y - ref) / bound)


def test_tf32_strategy_per_block(hp):
    """Elemental matrix on the tensor core exactly where N_P <= 256, FP32 sum
    factorisation elsewhere (reported per block; blocks in order of first
    appearance of their (shape, P, curved) in the mesh)."""
    from oracle.basis import n_modes
    mesh = mixed_mesh(6, n=1)
    h = hp.hp_mesh_create(mesh, 0)
    try:
        op = hp.hp_op_create(h, hp.HP_HELMHOLTZ, hp.HP_STRAT_ELEMAT, hp.HP_TF32)
        strat = hp.hp_op_strategies(op, n_blocks(mesh))
        keys = []
        for k in zip(mesh["shape"].tolist(), mesh["curved"].tolist()):
            if k not in keys:
                keys.append(k)
        want = [hp.HP_STRAT_ELEMAT if n_modes(s, 6) <= MAX_TC_MODES else hp.HP_STRAT_SUMFAC for s, _ in keys]
        assert strat.tolist() == want
        with pytest.raises(hp.HpError) as ei:       # stored matrices are FP64 / FP32 only
            hp.hp_op_strategies(op, len(keys), np.full(len(keys), hp.HP_STRAT_MATRIX))
        assert ei.value.status == hp.HP_ERR_UNSUPPORTED
        # the tensor-core hybrid covers every block here (N_P <= 343 <= 352)
        hp.hp_op_strategies(op, len(keys), np.full(len(keys), hp.HP_STRAT_HYBRID))
        assert (hp.hp_op_strategies(op, len(keys)) == hp.HP_STRAT_HYBRID).all()
        hp.hp_op_destroy(op)
        for kind, strategy in ((hp.HP_BWDTRANS, hp.HP_STRAT_ELEMAT), (hp.HP_HELMHOLTZ, hp.HP_STRAT_SUMFAC)):
            with pytest.raises(hp.HpError) as ei:
                hp.hp_op_create(h, kind, strategy, hp.HP_TF32)
            assert ei.value.status == hp.HP_ERR_UNSUPPORTED
    finally:
        hp.hp_mesh_destroy(h)


@pytest.mark.parametrize("shape,P,curved,prec", [(3, 2, True, "tf32"), (2, 4, False, "tf32"), (0, 3, True, "tf32"),
                                                (3, 4, True, "bf16"), (1, 5, False, "bf16")])
def test_large_block_single_part(hp, shape, P, curved, prec):
    """More tiles than SMs (each tile in one part, plain stores): 20 000
    elements of one shape, sampled elements against the oracle."""
    mesh = inputs.replicated_mesh(shape, P, 20000, curved=curved)
    co, _ = oracle_ops.layout(mesh)
    x = inputs.random_coefficients(77, co)
    y, strat = run_tc(hp, mesh, "helmholtz", x, 1.0, hp.HP_TF32 if prec == "tf32" else hp.HP_BF16)
    assert strat.tolist() == [hp.HP_STRAT_ELEMAT]
    rng = np.random.default_rng(1)
    sample = np.sort(np.concatenate([rng.choice(mesh["n_elem"], 150, replace=False), [mesh["n_elem"] - 1]]))
    sample = np.unique(sample)
    x32 = x.astype(np.float32).astype(np.float64)
    ref = oracle_ops.apply("helmholtz", mesh, x32, 1.0, elems=sample)
    idx = np.concatenate([np.arange(co[e], co[e + 1]) for e in sample])
    assert rel_err(y[idx], ref[idx]) <= (TF32_TOL if prec == "tf32" else BF16_TOL)


def test_tf32_single_element(hp):
    for shape in range(4):
        mesh = inputs.single_element_mesh(shape, 3, curved=True)
        x = make_input(mesh, "helmholtz", 9)
        ref = oracle_ops.apply("helmholtz", mesh, x.astype(np.float32).astype(np.float64), 0.7)
        y, _ = run_tc(hp, mesh, "helmholtz", x, 0.7)
        assert rel_err(y, ref) <= TF32_TOL, shape


@pytest.mark.parametrize("shape,P,curved", [(3, 2, True), (3, 4, True), (2, 4, False)])
def test_bf16_two_ctas_per_sm(hp, shape, P, curved):
    """BF16 blocks of at most 64 modes with at least two 128-element tiles per SM
    (40 960 elements = 320 tiles on 152 SMs) run two CTAs per SM with eight
    epilogue warps each: sampled elements against the oracle within BF16_TOL."""
    mesh = inputs.replicated_mesh(shape, P, 40960, curved=curved)
    co, _ = oracle_ops.layout(mesh)
    x = inputs.random_coefficients(91, co)
    y, strat = run_tc(hp, mesh, "helmholtz", x, 0.9, hp.HP_BF16)
    assert strat.tolist() == [hp.HP_STRAT_ELEMAT]
    assert not np.isnan(y).any()
    rng = np.random.default_rng(7)
    sample = np.unique(np.concatenate([rng.choice(mesh["n_elem"], 120, replace=False), [0, mesh["n_elem"] - 1]]))
    ref = oracle_ops.apply("helmholtz", mesh, x.astype(np.float32).astype(np.float64), 0.9, elems=sample)
    idx = np.concatenate([np.arange(co[e], co[e + 1]) for e in sample])
    assert rel_err(y[idx], ref[idx]) <= BF16_TOL


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("opname,lam", [("mass", 1.0), ("helmholtz", 5e11)])
def test_tensor_core_small_elements(hp, prec, opname, lam):
    """Elements of size h ~ 1e-5 (the mixed mesh scaled by 2e-5): w|J| ~ h^3
    and the Laplacian factors ~ h differ by ~1e10, so each group keeps its own
    power-of-two scale in FP16 (one shared scale would leave w|J| subnormal).
    The mass operator and a Helmholtz operator whose two terms are of one size
    (lambda = 5e11) stay within the tolerance of their form."""
    base = mixed_mesh(3)
    mesh = dict(base)
    mesh["xyz"] = base["xyz"] * 2e-5
    co, _ = oracle_ops.layout(mesh)
    x = make_input(mesh, opname, 17)
    ref = oracle_ops.apply(opname, mesh, x.astype(np.float32).astype(np.float64), lam)
    y, _ = run_tc(hp, mesh, opname, x, lam, hp.HP_TF32 if prec == "tf32" else hp.HP_BF16)
    assert not np.isnan(y).any()
    assert rel_err(y, ref) <= (TF32_TOL if prec == "tf32" else BF16_TOL)


@pytest.mark.parametrize("dt", ["tf32", "bf16"])
def test_deterministic_split_tiles_are_bitwise_reproducible(hp, dt):
    """Small blocks split their tiles' point chunks over CTAs.  With
    hp_op_set_deterministic the parts are summed in part order: repeated
    applies (plain and graph) give the same bits, and the result matches the
    atomic form to FP32 rounding and the oracle within the form's bound."""
    mesh = inputs.slab_mesh(2, 2, 4, (2, 4), order_seed=3, curved_rule="x_half")
    co, po = oracle_ops.layout(mesh)
    uh = inputs.random_coefficients(71, co)
    dtype = {"tf32": hp.HP_TF32, "bf16": hp.HP_BF16}[dt]
    h = hp.hp_mesh_create(mesh, 0)
    try:
        op = hp.hp_op_create(h, hp.HP_HELMHOLTZ, hp.HP_STRAT_ELEMAT, dtype)
        x = torch.tensor(uh, device="cuda:0", dtype=torch.float32)
        ys = []
        hp.hp_op_set_deterministic(op, True)
        for graph in (False, False, True, True):
            y = torch.full((len(uh),), float("nan"), device="cuda:0", dtype=torch.float32)
            (hp.hp_op_apply_graph if graph else hp.hp_op_apply)(op, 1.0, x, y)
            hp.hp_op_sync(op)
            ys.append(y.cpu().numpy())
        hp.hp_op_set_deterministic(op, False)
        ya = torch.zeros(len(uh), device="cuda:0", dtype=torch.float32)
        hp.hp_op_apply(op, 1.0, x, ya)
        hp.hp_op_sync(op)
        hp.hp_op_destroy(op)
    finally:
        hp.hp_mesh_destroy(h)
    for y in ys[1:]:
        assert np.array_equal(y.view(np.int32), ys[0].view(np.int32))
    ref = oracle_ops.apply("helmholtz", mesh, uh.astype(np.float32).astype(np.float64), 1.0)
    tol = TF32_TOL if dt == "tf32" else BF16_TOL
    assert rel_err(ys[0].astype(np.float64), ref) <= tol
    assert np.abs(ys[0] - ya.cpu().numpy()).max() <= 1e-5 * np.abs(ref).max()


@pytest.mark.parametrize("shape,P,curved", [(2, 8, True), (1, 7, False), (2, 8, False), (0, 6, True), (1, 8, False),
                                            (0, 7, True)])
def test_bf16_past_256_modes(hp, shape, P, curved):
    """BF16 blocks past 256 modes: the backward tiles are streamed; up to 320
    modes (pyramid P8: 285, prism P7: 288) the output takes two MMAs
    (N = 256 and N_P - 256), past 320 (hex P6: 343, prism P8: 405, hex P7:
    512) a tile's output modes are split into two work items of at most 320
    that each recompute the forward.  Blocks past 320 modes start on FP32 sum
    factorisation and are moved to the form here.  Many tiles, sampled
    elements against the oracle, per-output bound on a small mesh of the same
    block."""
    mesh = inputs.replicated_mesh(shape, P, 2000 + 13, curved=curved)
    co, _ = oracle_ops.layout(mesh)
    x = inputs.random_coefficients(91, co)
    y, strat = run_tc(hp, mesh, "helmholtz", x, 1.0, hp.HP_BF16, force=True)
    assert strat.tolist() == [hp.HP_STRAT_ELEMAT]
    rng = np.random.default_rng(5)
    sample = np.unique(np.concatenate([rng.choice(mesh["n_elem"], 30, replace=False), [0, 127, 128, 2012]]))
    x32 = x.astype(np.float32).astype(np.float64)
    ref = oracle_ops.apply("helmholtz", mesh, x32, 1.0, elems=sample)
    idx = np.concatenate([np.arange(co[e], co[e + 1]) for e in sample])
    assert rel_err(y[idx], ref[idx]) <= BF16_TOL
    small = inputs.replicated_mesh(shape, P, 37, curved=curved)
    cs, _ = oracle_ops.layout(small)
    xs = inputs.random_coefficients(92, cs)
    ys, _ = run_tc(hp, small, "helmholtz", xs, 1.0, hp.HP_BF16, force=True)
    xs32 = xs.astype(np.float32).astype(np.float64)
    refs = oracle_ops.apply("helmholtz", small, xs32, 1.0)
    from tests import roundoff
    bound = roundoff.tc_bound(small, xs32, 1.0, "helmholtz", BF16_U)
    assert (np.abs(ys - refs) <= bound).all(), np.max(np.abs(ys - refs) / bound)
