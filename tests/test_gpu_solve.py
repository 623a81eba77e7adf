"""Assembled Helmholtz solve on the GPU: gather/assembly maps, FP64 PCG and
mixed FP32 PCG + FP64 refinement against the oracle's independent
(null-space) solve, and spectral convergence to a manufactured solution."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import assembly, operators as oracle_ops  # noqa: E402
from paper_2604_04644_gb300 import inputs  # noqa: E402

LAM = 1.0


@pytest.fixture(scope="module")
def hp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_04644_gb300 import hp as _hp
    return _hp


_KAPPA = {}


def assembled_kappa(hp, pr, mesh):
    """Spectral condition number of the assembled, Dirichlet-masked lambda M + L
    of `mesh`: the oracle's explicit element matrices summed through the C0 map
    (signed gather, bit-exact against the oracle's null space elsewhere), the
    extreme eigenvalues by Lanczos (the smallest by shift-invert at 0)."""
    key = id(mesh)
    if key in _KAPPA:
        return _KAPPA[key]
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    gid, sign, bnd = hp.hp_c0_maps(pr.c0, pr.nc)
    co = pr.co
    rows, cols, vals = [], [], []
    nv = (8, 6, 5, 4)
    keys = {}
    for e in range(mesh["n_elem"]):
        keys.setdefault((int(mesh["shape"][e]), int(mesh["P"][e]), int(mesh["curved"][e])), []).append(e)
    for (s, P, cv), els in keys.items():
        X = mesh["xyz"][mesh["vert"][els][:, :nv[s]]]
        M, L = oracle_ops.element_matrices(s, P, P + 2, X, bool(cv), mesh["deformation"], mesh.get("geometry", 0))
        for t, e in enumerate(els):
            idx = gid[co[e]:co[e + 1]]
            sg = sign[co[e]:co[e + 1]].astype(np.float64)
            K = (LAM * M[t] + L[t]) * sg[:, None] * sg[None, :]
            rows.append(np.repeat(idx, len(idx)))
            cols.append(np.tile(idx, len(idx)))
            vals.append(K.ravel())
    ng = len(bnd)
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(ng, ng)).tocsc()
    free = np.nonzero(bnd == 0)[0]
    A = A[free][:, free]
    lmax = spla.eigsh(A, 1, which="LA", return_eigenvectors=False)[0]
    lmin = spla.eigsh(A, 1, sigma=0.0, which="LM", return_eigenvectors=False)[0]
    _KAPPA[key] = float(lmax / lmin)
    return _KAPPA[key]


def u_exact(x, y, z):
    return np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)


def f_rhs(x, y, z):
    return (3 * np.pi ** 2 + LAM) * u_exact(x, y, z)


class Problem:
    """Mesh, C0 map and right-hand side assembled with the library's kernels."""

    def __init__(self, hp, mesh):
        self.hp, self.mesh = hp, mesh
        self.h = hp.hp_mesh_create(mesh, 0)
        self.co, self.po, self.nc, self.nph = hp.hp_mesh_layout(self.h, mesh["n_elem"])
        self.c0 = hp.hp_c0_create(self.h)
        self.ng, self.nb = hp.hp_c0_info(self.c0)
        xyz = torch.empty(3 * self.nph, device="cuda:0", dtype=torch.float64)
        hp.hp_mesh_points(self.h, xyz)
        x, y, z = xyz.view(3, -1)
        f = (3 * np.pi ** 2 + LAM) * torch.sin(np.pi * x) * torch.sin(np.pi * y) * torch.sin(np.pi * z)
        self.xyz = xyz
        ip = hp.hp_op_create(self.h, hp.HP_IPRODUCT_WRT_BASE)
        bl = torch.empty(self.nc, device="cuda:0", dtype=torch.float64)
        hp.hp_op_apply(ip, 1.0, f.contiguous(), bl)
        hp.hp_op_destroy(ip)
        self.b = torch.empty(self.ng, device="cuda:0", dtype=torch.float64)
        hp.hp_c0_assemble(self.c0, bl, self.b, True)
        self.bwd = hp.hp_op_create(self.h, hp.HP_BWDTRANS)

    def values(self, xg):
        """Solution values at the quadrature points from a global vector."""
        loc = torch.empty(self.nc, device="cuda:0", dtype=torch.float64)
        self.hp.hp_c0_gather(self.c0, xg, loc)
        out = torch.empty(self.nph, device="cuda:0", dtype=torch.float64)
        self.hp.hp_op_apply(self.bwd, 1.0, loc, out)
        torch.cuda.synchronize()
        return out.cpu().numpy()

    def close(self):
        self.hp.hp_op_destroy(self.bwd)
        self.hp.hp_c0_destroy(self.c0)
        self.hp.hp_mesh_destroy(self.h)


def test_gather_and_assembly_match_host_maps(hp):
    mesh = inputs.c0_slab_mesh(4, 3, curved=True)
    pr = Problem(hp, mesh)
    try:
        gid, sign, bnd = hp.hp_c0_maps(pr.c0, pr.nc)
        gid2, sign2, bnd2, ng2 = hp.hp_c0_map_host(mesh, pr.nc)
        assert ng2 == pr.ng and np.array_equal(gid, gid2) and np.array_equal(sign, sign2) and np.array_equal(bnd, bnd2)
        rng = np.random.default_rng(0)
        g = rng.uniform(-1, 1, pr.ng)
        loc = torch.empty(pr.nc, device="cuda:0", dtype=torch.float64)
        hp.hp_c0_gather(pr.c0, torch.tensor(g, device="cuda:0"), loc)
        np.testing.assert_array_equal(loc.cpu().numpy(), sign * g[gid])      # integer map: exact
        l = rng.uniform(-1, 1, pr.nc)
        out = torch.empty(pr.ng, device="cuda:0", dtype=torch.float64)
        hp.hp_c0_assemble(pr.c0, torch.tensor(l, device="cuda:0"), out, False)
        ref = np.zeros(pr.ng)
        np.add.at(ref, gid, sign * l)
        np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=0, atol=1e-14)
        hp.hp_c0_assemble(pr.c0, torch.tensor(l, device="cuda:0"), out, True)
        assert (out.cpu().numpy()[bnd > 0] == 0).all()
    finally:
        pr.close()


@pytest.mark.parametrize("mixed", [0, 1, 2, 3])
def test_solve_matches_oracle(hp, mixed):
    """FP64 PCG (0), FP32 inner PCG (1), TF32 (2) and BF16 (3) tensor-core
    inner PCG, the mixed ones with FP64 refinement, all to the same FP64
    residual."""
    mesh = inputs.c0_slab_mesh(8, 3, curved=True, nx=1, ny=1)
    pr = Problem(hp, mesh)
    try:
        x = torch.zeros(pr.ng, device="cuda:0", dtype=torch.float64)
        rc, stats = hp.hp_solve(pr.c0, LAM, pr.b, x, tol=1e-12, mixed=mixed,
                                inner_tol={2: 1e-3, 3: 1e-2}.get(mixed, 1e-4))
        assert rc == hp.HP_OK and stats["rel_residual"] <= 1e-12, stats
        vals = pr.values(x)
        ul = assembly.solve(mesh, LAM, f_rhs)
        ref = oracle_ops.apply("bwd_trans", mesh, ul)
        assert np.abs(vals - ref).max() <= 1e-9 * np.abs(ref).max()
    finally:
        pr.close()


def test_manufactured_convergence_and_mixed_equals_fp64(hp):
    errs = []
    for P in (2, 3, 4, 5):
        mesh = inputs.c0_slab_mesh(4, P, curved=False)
        pr = Problem(hp, mesh)
        try:
            x64 = torch.zeros(pr.ng, device="cuda:0", dtype=torch.float64)
            rc, s64 = hp.hp_solve(pr.c0, LAM, pr.b, x64, tol=1e-10)
            assert rc == hp.HP_OK, (P, s64, hp.hp_last_error())
            xm = torch.zeros_like(x64)
            rc, sm = hp.hp_solve(pr.c0, LAM, pr.b, xm, tol=1e-10, mixed=True, inner_tol=1e-4)
            assert rc == hp.HP_OK and sm["refinements"] >= 1, (P, sm, hp.hp_last_error())
            v64 = pr.values(x64)
            vm = pr.values(xm)
            assert np.abs(v64 - vm).max() <= 1e-8 * np.abs(v64).max()
            pts = pr.xyz.view(3, -1).cpu().numpy()
            errs.append(np.abs(v64 - u_exact(*pts)).max())
        finally:
            pr.close()
    for a, b in zip(errs, errs[1:]):
        assert b < a / 2.5, errs


def test_solver_argument_checks(hp):
    mesh = inputs.c0_slab_mesh(4, 2, curved=False)
    pr = Problem(hp, mesh)
    try:
        x = torch.zeros(pr.ng, device="cuda:0", dtype=torch.float64)
        with pytest.raises(hp.HpError):
            hp.hp_solve(pr.c0, LAM, pr.b, x, tol=-1.0)
        rc, st = hp.hp_solve(pr.c0, LAM, pr.b, x, tol=1e-14, max_iter=2)
        assert rc == hp.HP_ERR_NOT_CONVERGED and st["iterations"] == 2
    finally:
        pr.close()


@pytest.mark.parametrize("P", [2, 4, 5])
def test_jacobi_diagonal_matches_unit_vector_applies(hp, P):
    """diag(A) from the element-diagonal kernel = assembled diagonals of the
    sum-factorised Helmholtz operator applied to unit vectors, one mode per
    element at a time."""
    mesh = inputs.c0_slab_mesh(4, P, curved=True)
    pr = Problem(hp, mesh)
    try:
        d = torch.empty(pr.ng, device="cuda:0", dtype=torch.float64)
        hp.hp_c0_diagonal(pr.c0, LAM, d)
        dl = torch.empty(pr.nc, device="cuda:0", dtype=torch.float64)
        hp.hp_c0_diagonal(pr.c0, LAM, dl, local=True)
        op = hp.hp_op_create(pr.h, hp.HP_HELMHOLTZ)
        co = pr.co
        npm = np.diff(co)
        loc = torch.zeros(pr.nc, device="cuda:0", dtype=torch.float64)
        outl = torch.empty_like(loc)
        dloc = np.zeros(pr.nc)
        for m in range(npm.max()):
            sel = co[:-1][npm > m] + m
            loc.zero_()
            loc[torch.tensor(sel, device="cuda:0")] = 1.0
            hp.hp_op_apply(op, LAM, loc, outl)
            dloc[sel] = outl.cpu().numpy()[sel]
        hp.hp_op_destroy(op)
        assert np.abs(dl.cpu().numpy() - dloc).max() <= 1e-12 * np.abs(dloc).max()
        gid, sign, bnd = hp.hp_c0_maps(pr.c0, pr.nc)
        ref = np.zeros(pr.ng)
        np.add.at(ref, gid, dloc)          # sign^2 = 1
        got = d.cpu().numpy()
        assert got[bnd == 0].min() > 0
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), np.argmax(np.abs(got - ref))
    finally:
        pr.close()


@pytest.mark.parametrize("mixed", [0, 1, 3])
def test_solve_is_deterministic(hp, mixed):
    """The CG loop's reductions use a fixed grid and sum in a fixed order, and
    alpha / beta stay on the device; the solve's tensor-core operator adds the
    partial outputs of split tiles in a fixed order (hp_op_set_deterministic).
    Two solves from the same start give the same iterates bit for bit and the
    same statistics, with the FP64, FP32 and BF16 tensor-core inner operators."""
    mesh = inputs.c0_slab_mesh(4, 4, curved=True)
    pr = Problem(hp, mesh)
    try:
        xs, st = [], []
        for _ in range(2):
            x = torch.zeros(pr.ng, device="cuda:0", dtype=torch.float64)
            rc, stats = hp.hp_solve(pr.c0, LAM, pr.b, x, tol=1e-11, mixed=mixed, inner_tol=1e-2 if mixed == 3 else 1e-4)
            assert rc == hp.HP_OK, stats
            xs.append(x.cpu().numpy())
            st.append(stats)
        assert st[0]["rel_residual"] <= 1e-11 and st[1]["rel_residual"] <= 1e-11
        assert np.array_equal(xs[0], xs[1])
        assert st[0] == st[1]
    finally:
        pr.close()


@pytest.mark.parametrize("mixed", [0, 1, 3])
def test_scheduled_solve_matches_plain_solve(hp, mixed):
    """schedule = 1 (graph-aware strategy choice of the solve's operators, stored
    matrices included) reaches the same tolerance and, within the bound the two
    residuals fix, the same solution as the default operators: both satisfy
    ||b - A x_i|| <= tol ||b||, so ||x_1 - x_2|| <= 2 tol kappa(A) ||x|| in the
    2-norm, with kappa(A) computed on this mesh (assembled_kappa); a later
    solve with schedule = 0 goes back to the default operators."""
    mesh = inputs.c0_slab_mesh(4, 4, curved=True)
    pr = Problem(hp, mesh)
    try:
        kw = dict(mixed=mixed, inner_tol={0: 1e-5, 1: 1e-4, 3: 1e-2}[mixed])
        xp = torch.zeros(pr.ng, device="cuda:0", dtype=torch.float64)
        rc, st = hp.hp_solve(pr.c0, LAM, pr.b, xp, tol=1e-11, **kw)
        assert rc == hp.HP_OK and st["rel_residual"] <= 1e-11
        xs = torch.zeros(pr.ng, device="cuda:0", dtype=torch.float64)
        rc, st = hp.hp_solve(pr.c0, LAM, pr.b, xs, tol=1e-11, schedule=True, **kw)
        assert rc == hp.HP_OK and st["rel_residual"] <= 1e-11
        kappa = assembled_kappa(hp, pr, mesh)
        assert float((xs - xp).norm() / xp.norm()) <= 2 * 1e-11 * kappa, kappa
        xq = torch.zeros(pr.ng, device="cuda:0", dtype=torch.float64)
        rc, st = hp.hp_solve(pr.c0, LAM, pr.b, xq, tol=1e-11, **kw)
        assert rc == hp.HP_OK
        if mixed == 0:
            assert torch.equal(xq, xp)      # the default FP64 operator again: the same iterates bit for bit
    finally:
        pr.close()
