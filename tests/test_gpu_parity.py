"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle,
element by element, on seeded inputs.

Tolerances (relative, infinity norm over the whole output vector):
  FP64: 1e-12 (the operators' required agreement with the FP64 oracle).
  FP32: fp32_tol(P) below, 6e-8 * 40 * Q: the FP32 unit roundoff times the
        number of rounded terms per output (about six passes of Q each) and
        the growth of max|D| with Q.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import operators as oracle_ops  # noqa: E402
from paper_2604_04644_gb300 import inputs  # noqa: E402

OPS = {
    "mass": 0, "laplacian": 1, "helmholtz": 2, "bwd_trans": 3, "iproduct_wrt_base": 4,
    "phys_deriv": 5, "iproduct_wrt_deriv": 6,
}
FP64_TOL = 1e-12


def fp32_tol(P):
    # u_32 = 2^-24 ~ 6e-8; errors grow with the number of terms per output
    # (~ 6 Q passes) and with max|D| ~ Q^2/4 relative to the output scale
    Q = P + 2
    return 6e-8 * 40 * Q


@pytest.fixture(scope="module")
def hp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_04644_gb300 import hp as _hp
    return _hp


_MESH_CACHE = {}


def mixed_mesh(P, n=3):
    key = (P, n)
    if key not in _MESH_CACHE:
        _MESH_CACHE[key] = inputs.slab_mesh(n, n, 4, P, curved_rule="x_half")
    return _MESH_CACHE[key]


def rel_err(y, ref):
    return np.abs(y - ref).max() / max(np.abs(ref).max(), 1e-300)


def run_op(hp, mesh, opname, data, lam=1.0, dtype=0):
    h = hp.hp_mesh_create(mesh, 0)
    try:
        co, po, nc, nph = hp.hp_mesh_layout(h, mesh["n_elem"])
        op = hp.hp_op_create(h, OPS[opname], hp.HP_STRAT_SUMFAC, dtype)
        try:
            out_n = {"bwd_trans": nph, "phys_deriv": 3 * nph}.get(opname, nc)
            tdt = torch.float64 if dtype == hp.HP_FP64 else torch.float32
            x = torch.tensor(data, device="cuda:0", dtype=tdt)
            y = torch.full((out_n,), float("nan"), device="cuda:0", dtype=tdt)
            hp.hp_op_apply(op, lam, x, y)
            hp.hp_op_sync(op)
            return y.double().cpu().numpy()
        finally:
            hp.hp_op_destroy(op)
    finally:
        hp.hp_mesh_destroy(h)


def make_input(mesh, opname, seed):
    co, po = oracle_ops.layout(mesh)
    kind = oracle_ops.IN_KIND[opname]
    if kind == "coeff":
        return inputs.random_coefficients(seed, co)
    return inputs.random_phys(seed, po, 3 if kind == "phys3" else 1)


@pytest.mark.parametrize("P", [1, 2, 3, 4, 6, 8])
@pytest.mark.parametrize("opname", list(OPS))
def test_fp64_matches_oracle(hp, P, opname):
    mesh = mixed_mesh(P)
    x = make_input(mesh, opname, 100 + P)
    ref = oracle_ops.apply(opname, mesh, x, 1.7)
    y = run_op(hp, mesh, opname, x, 1.7)
    assert not np.isnan(y).any()
    assert rel_err(y, ref) <= FP64_TOL, rel_err(y, ref)


@pytest.mark.parametrize("P", [9, 10])
def test_fp64_helmholtz_high_order(hp, P):
    mesh = inputs.slab_mesh(1, 1, 4, P, curved_rule="x_half")
    x = make_input(mesh, "helmholtz", 7)
    ref = oracle_ops.apply("helmholtz", mesh, x, 1.0)
    assert rel_err(run_op(hp, mesh, "helmholtz", x, 1.0), ref) <= FP64_TOL


@pytest.mark.parametrize("P", [1, 2, 4, 6, 8])
@pytest.mark.parametrize("opname", ["mass", "helmholtz", "bwd_trans", "iproduct_wrt_deriv", "phys_deriv"])
def test_fp32_matches_oracle(hp, P, opname):
    mesh = mixed_mesh(P)
    x = make_input(mesh, opname, 200 + P)
    x32 = x.astype(np.float32).astype(np.float64)      # the FP32 path sees rounded inputs
    ref = oracle_ops.apply(opname, mesh, x32, 1.7)
    y = run_op(hp, mesh, opname, x, 1.7, dtype=hp.HP_FP32)
    err = rel_err(y, ref)
    assert err <= fp32_tol(P), (err, fp32_tol(P))
    if opname in ("mass", "helmholtz"):
        # per output: the first-order rounding bound of the FP32 passes
        from tests import roundoff
        bound = roundoff.sf32_bound(mesh, x32, 1.7, opname)
        assert (np.abs(y - ref) <= bound).all(), np.max(np.abs(y - ref) / bound)


@pytest.mark.parametrize("P", [2, 5])
def test_geometric_factors_match_oracle(hp, P):
    mesh = mixed_mesh(P, n=2)
    h = hp.hp_mesh_create(mesh, 0)
    try:
        co, po, nc, nph = hp.hp_mesh_layout(h, mesh["n_elem"])
        g7, g9 = hp.hp_geom_copy(h, nph, want_deriv=True)
    finally:
        hp.hp_mesh_destroy(h)
    six, nine = oracle_ops.geometric_factors(mesh)
    for e in range(mesh["n_elem"]):
        a = g7[po[e] * 7: po[e + 1] * 7].reshape(7, -1)
        b = g9[po[e] * 9: po[e + 1] * 9].reshape(9, -1)
        assert np.abs(a - six[e]).max() <= 1e-13 * np.abs(six[e]).max(), e
        assert np.abs(b - nine[e]).max() <= 1e-13 * np.abs(nine[e]).max(), e


def test_layout_matches_oracle(hp):
    mesh = mixed_mesh(3)
    h = hp.hp_mesh_create(mesh, 0)
    try:
        co, po, nc, nph = hp.hp_mesh_layout(h, mesh["n_elem"])
    finally:
        hp.hp_mesh_destroy(h)
    oc, op_ = oracle_ops.layout(mesh)
    np.testing.assert_array_equal(co, oc)
    np.testing.assert_array_equal(po, op_)


def test_single_element_each_shape(hp):
    for shape in range(4):
        for curved in (False, True):
            mesh = inputs.single_element_mesh(shape, 5, curved=curved)
            x = make_input(mesh, "helmholtz", 3)
            ref = oracle_ops.apply("helmholtz", mesh, x, 0.3)
            assert rel_err(run_op(hp, mesh, "helmholtz", x, 0.3), ref) <= FP64_TOL


def test_full_size_sampled(hp):
    """16^3-cell mixed curved mesh at P = 4 (the benchmark workload and launch
    configuration): 300 sampled elements against the oracle, element by element."""
    mesh = inputs.slab_mesh(16, 16, 16, 4, curved=True)
    co, po = oracle_ops.layout(mesh)
    x = inputs.random_coefficients(1002, co)
    y = run_op(hp, mesh, "helmholtz", x, 1.0)
    rng = np.random.default_rng(0)
    sample = np.sort(rng.choice(mesh["n_elem"], 300, replace=False))
    ref = oracle_ops.apply("helmholtz", mesh, x, 1.0, elems=sample)
    idx = np.concatenate([np.arange(co[e], co[e + 1]) for e in sample])
    assert rel_err(y[idx], ref[idx]) <= FP64_TOL
    # property at full size: H is symmetric, so x . H z == z . H x
    z = inputs.random_coefficients(77, co)
    yz = run_op(hp, mesh, "helmholtz", z, 1.0)
    assert abs(x @ yz - z @ y) <= 1e-12 * abs(x @ y)


def test_error_paths(hp):
    mesh = mixed_mesh(2, n=1)
    bad = dict(mesh, Q=mesh["Q"] + 1)
    with pytest.raises(hp.HpError) as ei:
        hp.hp_mesh_create(bad, 0)
    assert ei.value.status == hp.HP_ERR_UNSUPPORTED
    bad = dict(mesh, vert=mesh["vert"].copy())
    bad["vert"][0, 0] = 10 ** 9
    with pytest.raises(hp.HpError) as ei:
        hp.hp_mesh_create(bad, 0)
    assert ei.value.status == hp.HP_ERR_ARG
    bad = dict(mesh, xyz=mesh["xyz"].copy())
    hexv = mesh["vert"][0, 2]                      # a hex vertex that is not on the frame
    bad["xyz"][hexv] += 0.01
    with pytest.raises(hp.HpError) as ei:
        hp.hp_mesh_create(bad, 0)
    assert ei.value.status == hp.HP_ERR_GEOM
    bad = dict(mesh, P=np.full_like(mesh["P"], 11), Q=np.full_like(mesh["Q"], 13))
    with pytest.raises(hp.HpError) as ei:
        hp.hp_mesh_create(bad, 0)
    assert ei.value.status == hp.HP_ERR_UNSUPPORTED
    h = hp.hp_mesh_create(mesh, 0)
    try:
        op = hp.hp_op_create(h, hp.HP_MASS)
        x = torch.zeros(10, device="cuda:0", dtype=torch.float64)
        with pytest.raises(hp.HpError) as ei:
            hp.hp_op_apply(op, 1.0, x, x)
        assert ei.value.status == hp.HP_ERR_ARG
        hp.hp_op_destroy(op)
        with pytest.raises(hp.HpError) as ei:
            hp.hp_op_create(h, hp.HP_MASS, hp.HP_STRAT_SUMFAC, 7)
        assert ei.value.status == hp.HP_ERR_ARG
    finally:
        hp.hp_mesh_destroy(h)


@pytest.mark.parametrize("P", [2, 4, 5])
@pytest.mark.parametrize("curved", [False, True])
def test_fp64_on_conforming_mesh_orientations(hp, P, curved):
    """The conforming mesh's element orientations (vertices sorted by id, swaps
    for positive volume) against the oracle, Helmholtz and mass."""
    mesh = inputs.c0_slab_mesh(4, P, curved=curved)
    for opname in ("helmholtz", "mass"):
        x = make_input(mesh, opname, 500 + P)
        ref = oracle_ops.apply(opname, mesh, x, 1.0)
        y = run_op(hp, mesh, opname, x, 1.0)
        assert rel_err(y, ref) <= FP64_TOL, (opname, rel_err(y, ref))


@pytest.mark.parametrize("opname", ["mass", "helmholtz"])
def test_unit_cube_of_64_affine_hexes(hp, opname):
    """64 affine hexahedra (4x4x4 structured [0,1]^3), P = 4, Q = 6, lambda = 1,
    coefficients U[-1,1) from seed 1001: FP64 against the oracle at 1e-12, and
    the TF32 tensor-core form at 8 units of TF32 rounding."""
    mesh = inputs.hex_cube_mesh(4, 4)
    co, _ = oracle_ops.layout(mesh)
    x = inputs.random_coefficients(1001, co)
    ref = oracle_ops.apply(opname, mesh, x, 1.0)
    y = run_op(hp, mesh, opname, x, 1.0)
    assert rel_err(y, ref) <= FP64_TOL
    h = hp.hp_mesh_create(mesh, 0)
    try:
        op = hp.hp_op_create(h, OPS[opname], hp.HP_STRAT_ELEMAT, hp.HP_TF32)
        xt = torch.tensor(x, device="cuda:0", dtype=torch.float32)
        y32 = torch.full((len(x),), float("nan"), device="cuda:0", dtype=torch.float32)
        hp.hp_op_apply(op, 1.0, xt, y32)
        hp.hp_op_sync(op)
        hp.hp_op_destroy(op)
    finally:
        hp.hp_mesh_destroy(h)
    ref32 = oracle_ops.apply(opname, mesh, x.astype(np.float32).astype(np.float64), 1.0)
    assert rel_err(y32.double().cpu().numpy(), ref32) <= 8 * 2.0 ** -11


def test_apply_block_and_block_work(hp):
    """Launching every block in turn (hp_op_apply_block) gives hp_op_apply's
    result bit for bit; per-block work sums to the operator's; the executed
    FP64 operations are at most the collocated count; bad blocks are refused."""
    mesh = mixed_mesh(5)
    co, _ = oracle_ops.layout(mesh)
    x = make_input(mesh, "helmholtz", 31)
    h = hp.hp_mesh_create(mesh, 0)
    try:
        op = hp.hp_op_create(h, hp.HP_HELMHOLTZ)
        nb = len(set(zip(mesh["shape"].tolist(), mesh["P"].tolist(), mesh["curved"].tolist())))
        xt = torch.tensor(x, device="cuda:0")
        y1 = torch.full((len(x),), float("nan"), device="cuda:0", dtype=torch.float64)
        y2 = torch.full_like(y1, float("nan"))
        hp.hp_op_apply(op, 1.0, xt, y1)
        for b in range(nb):
            hp.hp_op_apply_block(op, b, 1.0, xt, y2)
        hp.hp_op_sync(op)
        assert torch.equal(y1, y2)
        tot = hp.hp_op_block_work(op, -1)
        parts = [hp.hp_op_block_work(op, b) for b in range(nb)]
        assert sum(p[0] for p in parts) == mesh["n_elem"] == tot[0]
        assert sum(p[1] for p in parts) == tot[1] == hp.hp_op_work(op)[0]
        assert abs(sum(p[2] for p in parts) - tot[2]) <= 1e-9 * tot[2]
        assert all(0 < p[3] <= p[2] for p in parts)
        with pytest.raises(hp.HpError) as ei:
            hp.hp_op_apply_block(op, nb, 1.0, xt, y2)
        assert ei.value.status == hp.HP_ERR_ARG
        hp.hp_op_destroy(op)
    finally:
        hp.hp_mesh_destroy(h)
