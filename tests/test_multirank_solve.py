"""Multi-GPU layout on the host (no GPU): cost-balanced element partitions,
the halo plan of the assembled solve and exact dot products.

The pins: the exact dot product equals the rational-arithmetic sum rounded
once (fractions.Fraction), for any order and split of the terms; every
partition covers the elements and balances their cost; the halo sum of any
partition gives the one-rank assembly (copies added in local order from 0)
bit for bit; and a conjugate-gradient solve on two gloo ranks takes exactly
the iterates of the one-rank solve."""
import os
import socket
import sys
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2604_04644_gb300 import hp, inputs  # noqa: E402


def _bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.int64)


def _exact(x, y):
    return float(sum((Fraction(a) * Fraction(b) for a, b in zip(x.tolist(), y.tolist())), Fraction(0)))


def test_exact_dot_equals_rational_sum():
    rng = np.random.default_rng(3)
    for trial in range(20):
        n = int(rng.integers(1, 400))
        x = rng.standard_normal(n) * 2.0 ** rng.integers(-60, 60, n)
        y = rng.standard_normal(n) * 2.0 ** rng.integers(-60, 60, n)
        if trial % 3 == 0:                       # heavy cancellation: the exact sum is tiny
            x = np.concatenate([x, -x])
            y = np.concatenate([y, y * (1 + 2.0 ** -40)])
        got = hp.hp_xacc_round(hp.hp_xdot_acc(x, y))
        assert got == _exact(x, y)
    # extreme exponents: products near the top of the range and subnormal ones
    x = np.array([2.0 ** 500, -2.0 ** 500, 3.0, 2.0 ** -1074, 5e-324, 1e-310])
    y = np.array([2.0 ** 500, 2.0 ** 500, 2.0 ** -1000, 1.0, 3.0, 0.5])
    assert hp.hp_xacc_round(hp.hp_xdot_acc(x, y)) == _exact(x, y)


def test_exact_dot_is_independent_of_order_and_split():
    rng = np.random.default_rng(5)
    x = rng.standard_normal(5000) * 2.0 ** rng.integers(-30, 30, 5000)
    y = rng.standard_normal(5000)
    whole = hp.hp_xacc_round(hp.hp_xdot_acc(x, y))
    perm = rng.permutation(5000)
    assert hp.hp_xacc_round(hp.hp_xdot_acc(x[perm], y[perm])) == whole
    cuts = np.sort(rng.choice(np.arange(1, 5000), 6, replace=False))
    parts = [hp.hp_xdot_acc(a, b) for a, b in zip(np.split(x, cuts), np.split(y, cuts))]
    assert hp.hp_xacc_round(np.sum(parts, axis=0)) == whole      # the all-reduce is an integer sum
    assert whole == _exact(x, y)


@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("nparts", [1, 2, 3, 5])
def test_partition_covers_and_balances(method, nparts):
    mesh = inputs.slab_mesh(4, 4, 4, (1, 5), order_seed=3, curved_rule="x_half")
    cost = np.array([(P + 1) ** 3 * (1 + s) for s, P in zip(mesh["shape"].tolist(), mesh["P"].tolist())], float)
    part = hp.hp_partition(mesh, nparts, method, cost)
    assert part.min() >= 0 and part.max() == nparts - 1
    loads = np.bincount(part, weights=cost, minlength=nparts)
    assert np.abs(loads - cost.sum() / nparts).max() <= cost.max() + 1e-9
    assert np.array_equal(part, hp.hp_partition(mesh, nparts, method, cost))     # deterministic
    if method == 0:
        # ranges of the block order: along the blocks (first appearance, user
        # order inside), part ids never decrease
        keys = list(zip(mesh["shape"].tolist(), mesh["P"].tolist(), mesh["curved"].tolist()))
        first = {}
        for k in keys:
            first.setdefault(k, len(first))
        order = sorted(range(len(keys)), key=lambda e: (first[keys[e]], e))
        assert (np.diff(part[order]) >= 0).all()


def _c0_problem(n=4, P=2):
    mesh = inputs.c0_slab_mesh(n, P, curved=False)
    co = np.concatenate([[0], np.cumsum([[(P + 1) ** 3, (P + 1) ** 2 * (P + 2) // 2,
                                          (P + 1) * (P + 2) * (2 * P + 3) // 6,
                                          (P + 1) * (P + 2) * (P + 3) // 6][s] for s in mesh["shape"].tolist()])])
    gid, sign, bnd, ng = hp.hp_c0_map_host(mesh, int(co[-1]))
    return mesh, co, gid, sign, bnd, ng


def _one_rank_assembly(gid, sign, local, ng):
    out = np.zeros(ng)
    for i in range(len(gid)):             # copies of each DOF in local order, from 0 (hp_c0_assemble's order)
        out[gid[i]] += local[i] if sign[i] > 0 else -local[i]
    return out


@pytest.mark.parametrize("nparts", [1, 2, 3, 4])
def test_halo_sum_equals_one_rank_assembly(nparts):
    mesh, co, gid, sign, bnd, ng = _c0_problem()
    rng = np.random.default_rng(nparts)
    local = rng.standard_normal(len(gid)) * 2.0 ** rng.integers(-20, 20, len(gid))
    ref = _one_rank_assembly(gid, sign, local, ng)
    part = hp.hp_partition(mesh, nparts, 1)
    plans = [hp.Halo(gid, sign, co, ng, part, nparts, r) for r in range(nparts)]
    # each rank's local vector is its elements' coefficients, in user order
    loc = [local[p.local_index] for p in plans]
    send = [p.reduce_pack(l) for p, l in zip(plans, loc)]
    off = [np.concatenate([[0], np.cumsum(p.reduce_send)]) for p in plans]
    owned = []
    for r, p in enumerate(plans):
        recv = np.concatenate([send[q][off[q][r]:off[q][r + 1]] for q in range(nparts)])
        assert len(recv) == p.reduce_recv.sum()
        owned.append(p.reduce_sum(loc[r], recv))
        assert np.array_equal(_bits(owned[-1]), _bits(ref[p.owned_gid]))
    # every global DOF has exactly one owner
    assert np.array_equal(np.sort(np.concatenate([p.owned_gid for p in plans])), np.arange(ng))
    bsend = [p.bcast_pack(o) for p, o in zip(plans, owned)]
    boff = [np.concatenate([[0], np.cumsum(p.bcast_send)]) for p in plans]
    for r, p in enumerate(plans):
        recv = np.concatenate([bsend[q][boff[q][r]:boff[q][r + 1]] for q in range(nparts)])
        touched = p.bcast_unpack(owned[r], recv)
        assert np.array_equal(_bits(touched), _bits(ref[p.touched_gid]))
        # the gather of the touched values is the local part of A u
        assert np.array_equal(p.gather(touched), np.where(sign[p.local_index] > 0, 1.0, -1.0) *
                              ref[gid[p.local_index]])
    if nparts > 1:
        assert sum(p.reduce_send.sum() for p in plans) > 0      # the parts do share interface DOFs


# ------------------------------------------------------------------ two gloo ranks

def _element_matrices(mesh, co, seed=7):
    """A symmetric positive definite dense matrix per element (seeded): the
    stand-in element operator of the CG test (the exchange does not depend on
    what the element operator computes)."""
    rng = np.random.default_rng(seed)
    mats = []
    for e in range(mesh["n_elem"]):
        m = int(co[e + 1] - co[e])
        a = rng.standard_normal((m, m))
        mats.append(a @ a.T / m + np.eye(m))
    return mats


def _cg(plan, mats, co, part, rank, b_local_full, bnd, steps, comm):
    """Jacobi-free CG on the assembled sum of the element matrices, homogeneous
    Dirichlet DOFs masked; owned vectors on this rank, touched copies for the
    gather.  comm(kind, send_buf, counts_send, counts_recv) exchanges per-peer
    segments; allreduce(acc) sums exact-dot accumulators.  Returns the owned
    iterate and the residual norms squared."""
    exchange, allreduce = comm
    elems = np.nonzero(part == rank)[0]
    owned_bnd = bnd[plan.owned_gid].astype(bool)

    def apply(p_touched):
        lp = plan.gather(p_touched)
        ly = np.empty_like(lp)
        o = 0
        for e in elems:
            m = int(co[e + 1] - co[e])
            ly[o:o + m] = (mats[e] * lp[o:o + m][None, :]).sum(axis=1)
            o += m
        recv = exchange(plan.reduce_pack(ly), plan.reduce_send, plan.reduce_recv)
        q = plan.reduce_sum(ly, recv)
        q[owned_bnd] = 0.0
        return q

    def bcast(v):
        return plan.bcast_unpack(v, exchange(plan.bcast_pack(v), plan.bcast_send, plan.bcast_recv))

    def dot(a, c):
        return hp.hp_xacc_round(allreduce(hp.hp_xdot_acc(a, c)))

    lb = b_local_full[plan.local_index]
    b = plan.reduce_sum(lb, exchange(plan.reduce_pack(lb), plan.reduce_send, plan.reduce_recv))
    b[owned_bnd] = 0.0
    x = np.zeros(plan.n_owned)
    r = b.copy()
    p = r.copy()
    rr = dot(r, r)
    hist = [rr]
    for _ in range(steps):
        q = apply(bcast(p))
        alpha = rr / dot(p, q)
        x += alpha * p
        r -= alpha * q
        rr_new = dot(r, r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        hist.append(rr)
    return x, hist


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_2604_04644_gb300 import hp as hpm
    dist.init_process_group("gloo")

    def exchange(send, cs, cr):
        so = np.concatenate([[0], np.cumsum(cs)])
        ro = np.concatenate([[0], np.cumsum(cr)])
        recv = torch.zeros(int(ro[-1]), dtype=torch.float64)
        st = torch.from_numpy(np.ascontiguousarray(send))
        reqs = []
        for q in range(world):
            if q == rank:
                continue
            if cs[q]:
                reqs.append(dist.isend(st[so[q]:so[q + 1]].clone(), q))
            if cr[q]:
                reqs.append(dist.irecv(recv[ro[q]:ro[q + 1]], q))
        for rq in reqs:
            rq.wait()
        return recv.numpy()

    def allreduce(acc):
        t = torch.from_numpy(np.ascontiguousarray(acc, dtype=np.int64)).clone()
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return t.numpy()

    mesh, co, gid, sign, bnd, ng = _c0_problem(4, 2)
    mats = _element_matrices(mesh, co)
    b_local = np.random.default_rng(11).standard_normal(len(gid))
    part = hpm.hp_partition(mesh, world, 1)
    plan = hpm.Halo(gid, sign, co, ng, part, world, rank)
    x, hist = _cg(plan, mats, co, part, rank, b_local, bnd, 40, (exchange, allreduce))
    np.savez(os.path.join(out_dir, "rank%d.npz" % rank), x=x, gid=plan.owned_gid, hist=np.array(hist))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_cg_takes_the_one_rank_iterates(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    # the same solve on one rank, in this process
    mesh, co, gid, sign, bnd, ng = _c0_problem(4, 2)
    mats = _element_matrices(mesh, co)
    b_local = np.random.default_rng(11).standard_normal(len(gid))
    part = np.zeros(mesh["n_elem"], dtype=np.int32)
    plan = hp.Halo(gid, sign, co, ng, part, 1, 0)
    x1, hist1 = _cg(plan, mats, co, part, 0, b_local, bnd, 40,
                    (lambda send, cs, cr: np.zeros(0), lambda acc: acc))
    assert hist1[-1] < 1e-4 * hist1[0]                 # the one-rank CG converges
    xs = np.zeros(ng)
    for r in range(world):
        d = np.load(tmp_path / ("rank%d.npz" % r))
        assert np.array_equal(_bits(d["hist"]), _bits(np.array(hist1)))   # same residuals, bit for bit
        xs[d["gid"]] = d["x"]
    assert np.array_equal(_bits(xs), _bits(x1[np.argsort(plan.owned_gid)]))
