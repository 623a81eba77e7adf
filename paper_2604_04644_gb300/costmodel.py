"""Learned strategy cost model (not in the paper).

The paper chooses an implementation strategy by a fixed rule (StdMat for the
mass operator, sum factorisation for Helmholtz, Sec. 4).  Here a small MLP
predicts, for every block of an operator, the log10 run time of each
strategy the library builds, and the schedule takes the argmin
(hp_op_schedule_mlp).  The network is trained on timings the library
generates itself, by the library's own forward/backward/Adam kernels
(hp_mlp_*).  Exhaustive measurement is the fallback and the check on its
mispredictions: per block alone (hp_op_schedule_exhaustive) or on the time of
the whole concurrent graph (hp_op_schedule_graph).

Inputs (6): the block features of hp_op_block_features (shape/3, P/10,
curved, log10(elements)/6, dtype/2) and the launch mode: 0 when the blocks
run one after another (hp_op_apply), 1 when they run as the concurrent graph
of hp_op_apply_graph.
Outputs (4): log10 ms of sum factorisation, elemental matrix, hybrid and
stored per-element matrices.  For a TF32 / BF16 operator output 0 is its FP32
sum factorisation, output 1 its tensor-core elemental matrix and output 2 its
tensor-core hybrid.  A strategy
that is not built for a block gets the target 10x its sum-factorised time;
the schedulers never choose it.

Targets of the two launch modes.  Alone (mode 0): the block's own kernel
time.  Concurrent (mode 1): in the graph, blocks that do not fill the GPU
overlap with others, so a block costs its share of the GPU's throughput
rather than its latency: its per-element time on a block large enough to
fill the GPU (`n_sat` elements, the largest timed size) times its element
count.  One grid of single-block timings gives both.
"""
import statistics

import numpy as np

from . import hp, inputs

STRATS = (hp.HP_STRAT_SUMFAC, hp.HP_STRAT_ELEMAT, hp.HP_STRAT_HYBRID, hp.HP_STRAT_MATRIX)
STRAT_NAMES = ("sumfac", "elemat", "hybrid", "matrix")
N_IN, N_OUT = 6, 4
_TC = (hp.HP_TF32, hp.HP_BF16)


def n_modes(shape, P):
    """Modes per element of the modified C0 basis (Sec. 2.3): hex (P+1)^3,
    prism (P+1)^2 (P+2)/2, pyramid (P+1)(P+2)(2P+3)/6, tet (P+1)(P+2)(P+3)/6."""
    return ((P + 1) ** 3, (P + 1) ** 2 * (P + 2) // 2, (P + 1) * (P + 2) * (2 * P + 3) // 6,
            (P + 1) * (P + 2) * (P + 3) // 6)[shape]


def _built(dtype, kind, shape, P, k):
    """Strategy column k is built for a block of (shape, P) of this operator."""
    npm = n_modes(shape, P)
    if dtype in _TC:
        return (k == 0 or (k == 1 and npm <= (512 if dtype == hp.HP_BF16 else 256))
                or (k == 2 and npm <= (512 if dtype == hp.HP_BF16 else 352)))
    if k == 3:
        return kind in (hp.HP_MASS, hp.HP_LAPLACIAN, hp.HP_HELMHOLTZ) and npm <= 256
    return True


def _time_apply(op, x, y, lam, stream, flush, reps, graph=False):
    """Median device time (ms) of hp_op_apply (or hp_op_apply_graph), L2
    flushed before every launch, outside the events; one untimed warm-up."""
    import torch
    fn = hp.hp_op_apply_graph if graph else hp.hp_op_apply
    ts = []
    for r in range(reps + 1):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn(op, lam, x, y, stream)
        b.record(stream)
        b.synchronize()
        if r:
            ts.append(a.elapsed_time(b))
    hp.hp_op_sync(op, stream)
    return statistics.median(ts)


def generate_timings(device=0, kind=hp.HP_HELMHOLTZ, shapes=(0, 1, 2, 3), orders=range(1, 11), curved=(0, 1),
                     sizes=(128, 1024, 8192, 65536), dtypes=(hp.HP_FP64, hp.HP_FP32, hp.HP_BF16),
                     budget_ms=40.0, reps=2, log=None):
    """Time every built strategy on single-block meshes of the grid (each
    block launched alone).  A strategy whose time, extrapolated linearly from
    the next smaller size, would exceed `budget_ms` is not run; the
    extrapolated time is used and flagged.  Returns a list of records
    dict(shape, P, curved, n, dtype, ms[4] (None: not built), extrapolated[4])."""
    import torch
    dev = "cuda:%d" % device
    stream = torch.cuda.current_stream(device)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    recs = []
    for shape in shapes:
        for P in orders:
            for cv in curved:
                prev = {}
                for n in sizes:
                    mesh = inputs.replicated_mesh(shape, P, n, curved=bool(cv))
                    h = hp.hp_mesh_create(mesh, device)
                    co, po, nc, nph = hp.hp_mesh_layout(h, n)
                    uh = inputs.random_coefficients(11, co)
                    for dt in dtypes:
                        tdt = torch.float64 if dt == hp.HP_FP64 else torch.float32
                        op = hp.hp_op_create(h, kind, hp.HP_STRAT_ELEMAT if dt in _TC else hp.HP_STRAT_SUMFAC, dt)
                        x = torch.tensor(uh, device=dev, dtype=tdt)
                        y = torch.empty(nc, device=dev, dtype=tdt)
                        ms, ex = [None] * 4, [False] * 4
                        for k, st in enumerate(STRATS):
                            if not _built(dt, kind, shape, P, k):
                                continue
                            key = (dt, k)
                            est = prev[key][1] * n / prev[key][0] if key in prev else 0.0
                            if est > budget_ms:
                                t, ex[k] = est, True
                            else:
                                hp.hp_op_strategies(op, 1, [st])
                                t = _time_apply(op, x, y, 1.0, stream, flush, reps)
                            prev[key] = (n, t)
                            ms[k] = t
                        hp.hp_op_destroy(op)
                        recs.append(dict(shape=shape, P=P, curved=cv, n=n, dtype=dt, ms=ms, extrapolated=ex))
                        if log:
                            log(recs[-1])
                    hp.hp_mesh_destroy(h)
    return recs


def training_set(recs):
    """(X [N, 6], T [N, 4] log10 ms) with one sample per record and launch
    mode.  Mode 1 targets: per-element time at the largest timed size of the
    same (shape, P, curved, dtype) times the element count (for blocks at
    least that large, their own time)."""
    big = {}
    for r in recs:
        key = (r["shape"], r["P"], r["curved"], r["dtype"])
        if key not in big or r["n"] > big[key]["n"]:
            big[key] = r
    X, T = [], []
    for r in recs:
        f = [r["shape"] / 3.0, r["P"] / 10.0, float(r["curved"]), np.log10(r["n"]) / 6.0,
             (0 if r["dtype"] == hp.HP_FP64 else r["dtype"]) / 2.0]
        b = big[(r["shape"], r["P"], r["curved"], r["dtype"])]
        for mode in (0, 1):
            ms = []
            for k in range(N_OUT):
                if r["ms"][k] is None:
                    ms.append(None)
                elif mode == 0 or r["n"] >= b["n"]:
                    ms.append(r["ms"][k])
                else:
                    ms.append(b["ms"][k] * r["n"] / b["n"])
            ms = [t if t is not None else 10.0 * ms[0] for t in ms]
            X.append(f + [float(mode)])
            T.append(np.log10(np.maximum(ms, 1e-4)))
    return np.array(X, dtype=np.float32), np.array(T, dtype=np.float32)


def train(X, T, device=0, hidden=64, steps=4000, lr=3e-3, seed=7, decay_at=(0.6, 0.85)):
    """Full-batch Adam on the GPU with the library's kernels; returns (mlp, loss history)."""
    import torch
    dev = "cuda:%d" % device
    mlp = hp.hp_mlp_create(X.shape[1], hidden, T.shape[1], seed, device)
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
    n_out = hp.hp_mlp_info(mlp)[2]
    xt = torch.tensor(X, device=dev, dtype=torch.float32).contiguous()
    y = torch.empty((len(X), n_out), device=dev, dtype=torch.float32)
    hp.hp_mlp_forward(mlp, xt, len(X), y)
    torch.cuda.synchronize(device)
    return y.cpu().numpy()


def rule_strategy(kind, dtype):
    """The paper's fixed rule (Sec. 4): the elemental matrix (StdMat) for the
    mass operator, sum factorisation otherwise.  The paper has no tensor-core
    form; for TF32 / BF16 the baseline is the tensor core wherever it is built."""
    if dtype in _TC:
        return hp.HP_STRAT_ELEMAT
    return hp.HP_STRAT_ELEMAT if kind == hp.HP_MASS else hp.HP_STRAT_SUMFAC


def evaluate_schedules(mlp, mesh, kind, dtype=hp.HP_FP64, device=0, reps=7, graph=True, search=True):
    """Apply time (ms, median, L2 flushed) of one operator on `mesh`, launched
    as the concurrent graph (graph=True) or block after block, under: the
    paper's rule; the MLP schedule for that launch mode; each block's fastest
    strategy timed alone (hp_op_schedule_exhaustive); and, for graph launches,
    the search on the whole graph's time (hp_op_schedule_graph, from the
    rule's strategies) when `search`."""
    import torch
    dev = "cuda:%d" % device
    stream = torch.cuda.current_stream(device)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    h = hp.hp_mesh_create(mesh, device)
    co, po, nc, nph = hp.hp_mesh_layout(h, mesh["n_elem"])
    tdt = torch.float64 if dtype == hp.HP_FP64 else torch.float32
    x = torch.tensor(inputs.random_coefficients(21, co), device=dev, dtype=tdt)
    y = torch.empty(nc, device=dev, dtype=tdt)
    op = hp.hp_op_create(h, kind, hp.HP_STRAT_ELEMAT if dtype in _TC else hp.HP_STRAT_SUMFAC, dtype)
    nb = len(set(zip(mesh["shape"].tolist(), mesh["P"].tolist(), mesh["curved"].tolist())))
    default = hp.hp_op_strategies(op, nb)
    rule = rule_strategy(kind, dtype)
    rule_choice = np.where(default == hp.HP_STRAT_SUMFAC, hp.HP_STRAT_SUMFAC, rule) if dtype in _TC \
        else np.full(nb, rule, dtype=np.int32)
    out = {"blocks": nb, "launch": "graph" if graph else "per_block"}

    def timed():
        return _time_apply(op, x, y, 1.0, stream, flush, reps, graph=graph)

    def hist(st):
        return {n: int((st == v).sum()) for n, v in zip(STRAT_NAMES, STRATS) if (st == v).any()}

    hp.hp_op_strategies(op, nb, rule_choice)
    out["rule_ms"] = timed()
    hp.hp_op_schedule_mlp(op, mlp, 1 if graph else 0)
    mlp_choice = hp.hp_op_strategies(op, nb)
    out["mlp_ms"] = timed()
    out["choices_mlp"] = hist(mlp_choice)
    times = hp.hp_op_schedule_exhaustive(op, 1.0, x, y, nb)
    alone = hp.hp_op_strategies(op, nb)
    out["exhaustive_alone_ms"] = timed()
    out["choices_exhaustive_alone"] = hist(alone)
    out["mispredicted_vs_alone"] = int((mlp_choice != alone).sum())
    if graph and search:
        hp.hp_op_strategies(op, nb, rule_choice)
        hp.hp_op_schedule_graph(op, 1.0, x, y, 5, 2)
        gs = hp.hp_op_strategies(op, nb)
        out["graph_search_ms"] = timed()
        out["choices_graph_search"] = hist(gs)
        out["mispredicted_vs_graph_search"] = int((mlp_choice != gs).sum())
    best = min(v for k, v in out.items() if k.endswith("_ms") and k != "mlp_ms")
    out["mlp_over_best_searched"] = round(out["mlp_ms"] / min(best, out["exhaustive_alone_ms"]), 4)
    out["rule_over_mlp"] = round(out["rule_ms"] / out["mlp_ms"], 4)
    out["sum_of_block_times_alone_ms"] = float(np.where(times < 1e29, times, np.inf).min(axis=1).sum())
    hp.hp_op_destroy(op)
    hp.hp_mesh_destroy(h)
    return out
