"""Learned strategy cost model (not in the paper).

The paper chooses an implementation strategy by a fixed rule (StdMat for the
mass operator, sum factorisation for Helmholtz, Sec. 4).  Here a small MLP
(5 block features -> 64 -> 64 -> 3 predicted log10 run times of
{sum-factorised, elemental matrix, hybrid}) is trained on timings that the
library generates itself, by the library's own forward/backward/Adam kernels
(hp_mlp_*), and then schedules each block of an operator (hp_op_schedule).
Exhaustive measurement (hp_op_schedule_exhaustive) is the fallback and the
judge of its mispredictions.

Features (hp_op_block_features): shape/3, P/10, curved, log10(elements)/6,
dtype/2.  One network per operator kind.  For a TF32 operator the three
outputs are FP32 sum factorisation, the tensor-core elemental matrix, and
hybrid (not built for TF32: its target is a 10x penalty on the sum-factorised
time, as is the tensor-core entry of blocks over 256 modes; both schedulers
skip strategies that are not built).
"""
import statistics

import numpy as np

from . import hp, inputs

STRATS = (hp.HP_STRAT_SUMFAC, hp.HP_STRAT_ELEMAT, hp.HP_STRAT_HYBRID)
STRAT_NAMES = ("sumfac", "elemat", "hybrid")


def _time(op, x, y, lam, stream, flush, reps):
    import torch
    ts = []
    for r in range(reps + 1):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        hp.hp_op_apply(op, lam, x, y, stream)
        b.record(stream)
        b.synchronize()
        if r:
            ts.append(a.elapsed_time(b))
    hp.hp_op_sync(op, stream)
    return statistics.median(ts)


def generate_timings(device=0, kind=hp.HP_HELMHOLTZ, shapes=(0, 1, 2, 3), orders=range(1, 11), curved=(0, 1),
                     sizes=(100, 1000, 10000, 100000, 1000000), dtypes=(hp.HP_FP64, hp.HP_FP32, hp.HP_TF32),
                     budget_ms=40.0, reps=2, measured_max=100000, log=None):
    """Time every strategy on single-block meshes of the grid.  A strategy whose
    time, extrapolated linearly from the next smaller size, would exceed
    `budget_ms` is not run, nor is any size above `measured_max` elements (at
    10^5 elements every block already fills the GPU many times over, so time is
    linear in the element count); their extrapolated times are used (flagged in
    `meta`).  Returns (X [N,5] float32 features, T [N,3] float32 log10(ms),
    meta list)."""
    import torch
    dev = "cuda:%d" % device
    stream = torch.cuda.current_stream(device)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    X, T, meta = [], [], []
    for shape in shapes:
        for P in orders:
            for cv in curved:
                prev = {}
                for n in sizes:
                    measured = n <= measured_max
                    if measured:
                        mesh = inputs.replicated_mesh(shape, P, n, curved=bool(cv))
                        h = hp.hp_mesh_create(mesh, device)
                        co, po, nc, nph = hp.hp_mesh_layout(h, n)
                        uh = inputs.random_coefficients(11, co)
                    for dt in dtypes:
                        feats = np.array([shape / 3.0, P / 10.0, float(cv), np.log10(n) / 6.0,
                                          (0 if dt == hp.HP_FP64 else dt) / 2.0], dtype=np.float32)
                        op = None
                        if measured:
                            tdt = torch.float64 if dt == hp.HP_FP64 else torch.float32
                            op = hp.hp_op_create(h, kind, hp.HP_STRAT_ELEMAT if dt == hp.HP_TF32 else hp.HP_STRAT_SUMFAC,
                                                 dt)
                            x = torch.tensor(uh, device=dev, dtype=tdt)
                            y = torch.empty(nc, device=dev, dtype=tdt)
                            feats = hp.hp_op_block_features(op, 1)[0]
                            built = hp.hp_op_strategies(op, 1)[0]      # TF32: ELEMAT where the tensor core takes it
                        times, extrap, avail = [], [], []
                        for k, st in enumerate(STRATS):
                            key = (dt, k)
                            ok = not (dt == hp.HP_TF32 and (k == 2 or (k == 1 and prev.get((dt, "tc")) is False)))
                            if measured and dt == hp.HP_TF32 and k == 1:
                                ok = built == hp.HP_STRAT_ELEMAT
                                prev[(dt, "tc")] = ok
                            if not ok:
                                times.append(None)
                                extrap.append(False)
                                avail.append(False)
                                continue
                            est = prev[key][1] * n / prev[key][0] if key in prev else 0.0
                            if est > budget_ms or not measured:
                                t = est
                                extrap.append(True)
                            else:
                                hp.hp_op_strategies(op, 1, [st])
                                t = _time(op, x, y, 1.0, stream, flush, reps)
                                extrap.append(False)
                            prev[key] = (n, t)
                            times.append(t)
                            avail.append(True)
                        if op is not None:
                            hp.hp_op_destroy(op)
                        # strategies that are not built: 10x the sum-factorised time
                        times = [t if a else 10.0 * times[0] for t, a in zip(times, avail)]
                        X.append(feats)
                        T.append(np.log10(np.maximum(times, 1e-4)))
                        meta.append(dict(shape=shape, P=P, curved=cv, n=n, dtype=dt, ms=times, extrapolated=extrap,
                                         built=avail))
                        if log:
                            log(meta[-1])
                    if measured:
                        hp.hp_mesh_destroy(h)
    return np.array(X, dtype=np.float32), np.array(T, dtype=np.float32), meta


def train(X, T, device=0, hidden=64, steps=4000, lr=3e-3, seed=7, decay_at=(0.6, 0.85)):
    """Full-batch Adam on the GPU with the library's kernels; returns (mlp, loss history)."""
    import torch
    dev = "cuda:%d" % device
    mlp = hp.hp_mlp_create(5, hidden, 3, seed, device)
    xt = torch.tensor(X, device=dev, dtype=torch.float32).contiguous()
    tt = torch.tensor(T, device=dev, dtype=torch.float32).contiguous()
    loss = torch.zeros(1, device=dev, dtype=torch.float32)
    hist = []
    for i in range(steps):
        rate = lr * (0.3 if i >= decay_at[0] * steps else 1.0) * (0.3 if i >= decay_at[1] * steps else 1.0)
        hp.hp_mlp_adam_step(mlp, xt, tt, len(X), rate, loss)
        if i % 200 == 0 or i == steps - 1:
            hist.append((i, float(loss.item())))
    return mlp, hist


def predict(mlp, X, device=0):
    import torch
    dev = "cuda:%d" % device
    xt = torch.tensor(X, device=dev, dtype=torch.float32).contiguous()
    y = torch.empty((len(X), 3), device=dev, dtype=torch.float32)
    hp.hp_mlp_forward(mlp, xt, len(X), y)
    torch.cuda.synchronize(device)
    return y.cpu().numpy()


def evaluate_schedules(mlp, mesh, kind, dtype=hp.HP_FP64, device=0, reps=5):
    """Apply time of one operator on `mesh` under three schedules: the paper's
    rule (elemental matrix for mass, sum factorisation otherwise), the MLP
    schedule, and the exhaustive-search schedule."""
    import torch
    dev = "cuda:%d" % device
    stream = torch.cuda.current_stream(device)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    h = hp.hp_mesh_create(mesh, device)
    co, po, nc, nph = hp.hp_mesh_layout(h, mesh["n_elem"])
    tdt = torch.float64 if dtype == hp.HP_FP64 else torch.float32
    x = torch.tensor(inputs.random_coefficients(21, co), device=dev, dtype=tdt)
    y = torch.empty(nc, device=dev, dtype=tdt)
    op = hp.hp_op_create(h, kind, hp.HP_STRAT_ELEMAT if dtype == hp.HP_TF32 else hp.HP_STRAT_SUMFAC, dtype)
    nb = len(set(zip(mesh["shape"].tolist(), mesh["P"].tolist(), mesh["curved"].tolist())))
    out = {"blocks": nb}
    if dtype == hp.HP_TF32:
        # no rule in the paper for the tensor cores: the baseline is "tensor core wherever it is built"
        out["rule"] = "tensor core where built (N_P <= 256), FP32 sum factorisation elsewhere"
    else:
        rule = hp.HP_STRAT_ELEMAT if kind == hp.HP_MASS else hp.HP_STRAT_SUMFAC
        hp.hp_op_strategies(op, nb, [rule] * nb)
        out["rule"] = "elemental matrix for mass, sum factorisation otherwise"
    out["rule_ms"] = _time(op, x, y, 1.0, stream, flush, reps)
    hp.hp_op_schedule(op, mlp)
    mlp_choice = hp.hp_op_strategies(op, nb)
    out["mlp_ms"] = _time(op, x, y, 1.0, stream, flush, reps)
    times = hp.hp_op_schedule_exhaustive(op, 1.0, x, y, nb)
    best = hp.hp_op_strategies(op, nb)
    out["exhaustive_ms"] = _time(op, x, y, 1.0, stream, flush, reps)
    sumfac_only = np.array([t[0] for t in times]).sum()
    times = np.where(times >= 1e29, np.inf, times)        # strategies that are not built
    out["mispredicted_blocks"] = int((mlp_choice != best).sum())
    out["mispredicted_cost_ms"] = float(sum(times[i][mlp_choice[i]] - times[i][best[i]] for i in range(nb)))
    out["choices_mlp"] = np.bincount(mlp_choice, minlength=3).tolist()
    out["choices_exhaustive"] = np.bincount(best, minlength=3).tolist()
    out["sum_of_block_times_sumfac_ms"] = float(sumfac_only)
    hp.hp_op_destroy(op)
    hp.hp_mesh_destroy(h)
    return out
