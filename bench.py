"""Benchmark: Helmholtz apply throughput (GDOF/s) on the mixed curved mesh.

Workload: the unit cube in 16^3 cells, four slabs (hexes, prisms, pyramids,
tetrahedra; 15 360 elements), all curved by x_i += 0.05 sin(pi x_j) sin(pi x_k),
orders P = 1..8 with Q = P + 2, lambda = 1, coefficients U[-1,1) (seed 1002).
One step = one Helmholtz apply of the whole mesh at each order (8 applies).
GDOF/s = output elemental DOFs / seconds / 1e9 (the paper's BK metric).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--dtype f64|f32]

Under torchrun (N > 1) the mesh's elements are split over the ranks by
predicted cost (hp_partition), each rank applying its part on its own GPU
(strong scaling: the total work is fixed; the element-local operator needs no
data-path collective); time is the max over ranks, value the DOFs of all ranks
over that time.

Besides the timed step, rank 0 of a one-GPU run adds (unless --no-extra):
per shape/order GDOF/s, the 192 000-element p-adaptive batched apply (FP64 and
the reduced-precision graph forms), a strategy table, the FP32 / TF32 / BF16
forms of the bench mesh with their error against FP64, and the time to solution
of the assembled Helmholtz problem on ~1M elements (FP64 PCG against the
mixed-precision forms, --no-solve skips it).  The p-adaptive forms include the
FP64 and FP32 graph-scheduled applies, whose per-block strategy may be the
stored element matrix.

Other modes (instead of the timed step): --solve (time to solution alone, with
the graph-scheduled solves), --block-table (FP32 / TF32 / BF16 per large
block), --collocation-study (collocated vs non-collocated FP64 sum
factorisation on regular blocks, the paper's collocation study),
--matrix-study (stored H^e vs sum factorisation), --costmodel,
--profile-case NAME (one small case for a profiler capture).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Helmholtz apply GDOF/s per shape/order, % HBM/FP roofline, vs plain FP64 form"
ORDERS = list(range(1, 9))
CELLS = 16
FP64_PEAK_TFLOPS = 1.25     # GB300 FP64 (vector and tensor) nominal rate, profiling recipe table
SHAPES = ("hex", "prism", "pyr", "tet")
# modes per element of each shape at order P (the modified C0 basis, Sec. 2.3)
N_MODES = (lambda P: (P + 1) ** 3, lambda P: (P + 1) ** 2 * (P + 2) // 2,
           lambda P: (P + 1) * (P + 2) * (2 * P + 3) // 6, lambda P: (P + 1) * (P + 2) * (P + 3) // 6)
# DRAM bytes (read + write) of one launch, measured by ncu on this workload
# for the kernel named; a kernel whose code changed after the measurement is
# left out (its traffic reads null)
MEASURED_TRAFFIC = {"sf_kernel<pyr,P8,f64>": 372196352,           # profiles/sf_kernel_pyr_P8_fp64.md
                    "tc_emat_kernel<tet,P8,bf16>": 99582720,      # profiles/tc_emat_kernel_tet_P8_bf16_mixed16.md
                    "tc_emat_kernel<pyr,P7,bf16>": 75540224,      # profiles/tc_emat_kernel_pyr_P7_bf16_mixed16.md
                    "tc_emat_kernel<prism,P7,bf16>": 27841280,    # profiles/tc_emat_kernel_pyr_P7_bf16_mixed16.md
                    "tc_emat_kernel<pyr,P8,bf16>": 106597376,     # profiles/tc_emat_kernel_pyr_P8_bf16_mixed16.md
                    "sf_kernel<pyr,P8,f32>": 185804800}          # profiles/sf_kernel_pyr_P8_fp32_mixed16.md


# small, fixed cases for ncu captures (a few hundred MB on the device):
# name -> (shape, P, elements, strategy, dtype)
PROFILE_CASES = {
    "tc_tet8": (3, 8, 19456, "ELEMAT", "TF32"),
    "tc16_tet8": (3, 8, 19456, "ELEMAT", "BF16"),
    "tc16_hex4": (0, 4, 65536, "ELEMAT", "BF16"),
    "sf32_hex4": (0, 4, 65536, "SUMFAC", "FP32"),
    "sf32_tet4": (3, 4, 65536, "SUMFAC", "FP32"),
    # shape -1: the bench mesh itself (16^3 mixed curved cells) at order P
    "mesh16_bf16_P8": (-1, 8, 0, "ELEMAT", "BF16"),
    "mesh16_bf16_P4": (-1, 4, 0, "ELEMAT", "BF16"),
    "mesh16_bf16_P7": (-1, 7, 0, "ELEMAT", "BF16"),
}


def hp_block_work(op, block):
    from paper_2604_04644_gb300 import hp
    return hp.hp_op_block_work(op, block)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--oracle-sample", type=float, default=None, help=argparse.SUPPRESS)
    p.add_argument("--dtype", default="f64", choices=["f64", "f32"])
    p.add_argument("--no-table", action="store_true", help="skip the per-shape/order table")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--costmodel", action="store_true",
                   help="run the learned cost-model pipeline (timings, GPU training, held-out schedules) instead")
    p.add_argument("--solve", action="store_true",
                   help="assembled Helmholtz solve (time to 1e-10): FP64 PCG vs mixed FP32 PCG + FP64 refinement")
    p.add_argument("--no-extra", action="store_true",
                   help="skip the p-adaptive, strategy, precision and time-to-solution measurements")
    p.add_argument("--no-solve", action="store_true", help="skip the time-to-solution measurement (64^3 cells)")
    p.add_argument("--block-table", action="store_true",
                   help="GDOF/s of FP32 sum factorisation and the TF32 / BF16 tensor-core operator on large "
                        "single-shape blocks instead")
    p.add_argument("--reduced-q", action="store_true",
                   help="GDOF/s of the BF16 / TF32 tensor-core Helmholtz operator with the full and the reduced "
                        "quadrature rule on large collapsed-shape blocks instead")
    p.add_argument("--two-d", action="store_true",
                   help="GDOF/s of the two-dimensional quadrilateral / triangle Helmholtz operator (FP64, FP32) "
                        "instead")
    p.add_argument("--collocation-study", action="store_true",
                   help="GDOF/s of the collocated and the non-collocated FP64 sum-factorised Helmholtz on "
                        "regular (affine) single-shape blocks, P = 1..8, instead")
    p.add_argument("--matrix-study", action="store_true",
                   help="GDOF/s of the stored-matrix strategy (per-element dense H^e) against sum factorisation, "
                        "FP64 and FP32, curved single-shape blocks, P = 1..5, instead")
    p.add_argument("--profile-case", default=None, choices=sorted(PROFILE_CASES),
                   help="run one small case for a profiler capture instead (tc_tet8 / tc16_tet8: TF32 / BF16 "
                        "tensor-core Helmholtz, 19 456 curved tets, P = 8; tc16_hex4: BF16, 65 536 curved hexes, P = 4; sf32_hex4 / sf32_tet4: FP32 sum "
                        "factorisation, 65 536 curved hexes / tets, P = 4; three applies)")
    p.add_argument("--orders", default=None, help="comma-separated orders (default 1..8); for profiling runs")
    p.add_argument("--cells", type=int, default=None, help="cells per direction (default 16); for profiling runs")
    a = p.parse_args()
    global ORDERS, CELLS
    if a.orders:
        ORDERS = [int(x) for x in a.orders.split(",")]
    if a.cells:
        CELLS = a.cells
    return a


def dist_init(args, backend=None):
    """One process per GPU (torchrun environment); NCCL for the GPU arm, gloo
    for the CPU reference arm (and for the host-path tests)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if backend is None:
            backend = "nccl" if args.impl == "gb300" else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(world, x, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def split_scaling_value(world, dofs_local, ms_step, device=None):
    """Whole-job throughput of a workload split over the ranks (strong
    scaling: the total is fixed): the DOFs of all ranks over the slowest
    rank's step time.  Returns (max-over-ranks ms per step, total GDOF/s)."""
    ms_max = max_over_ranks(world, ms_step, device=device)
    dofs = sum_over_ranks(world, float(dofs_local), device=device)
    return ms_max, dofs / (ms_max * 1e-3) / 1e9


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def build_workloads(dtype_name, device, world=1, rank=0):
    """One Helmholtz operator per order on the bench mesh.  With several ranks
    the mesh's elements are split into world parts balanced by predicted cost
    (hp_partition: ranges of the block order, cost = each element's collocated
    flops) and this rank builds its part only: the element-local operator
    needs no exchange between parts."""
    import torch
    from paper_2604_04644_gb300 import hp, inputs
    dt = hp.HP_FP64 if dtype_name == "f64" else hp.HP_FP32
    tdt = torch.float64 if dtype_name == "f64" else torch.float32
    work = []
    for P in ORDERS:
        mesh = inputs.slab_mesh(CELLS, CELLS, CELLS, P, curved=True)
        if world > 1:
            part = hp.hp_partition(mesh, world, 0)
            mesh = inputs.subset_mesh(mesh, np.nonzero(part == rank)[0])
        h = hp.hp_mesh_create(mesh, device)
        co, po, nc, nph = hp.hp_mesh_layout(h, mesh["n_elem"])
        op = hp.hp_op_create(h, hp.HP_HELMHOLTZ, hp.HP_STRAT_SUMFAC, dt)
        uh = inputs.random_coefficients(1002, co)
        x = torch.tensor(uh, device="cuda:%d" % device, dtype=tdt)
        y = torch.zeros(nc, device="cuda:%d" % device, dtype=tdt)
        dofs, flops, bytes_ = hp.hp_op_work(op)
        keys = []
        for k in zip(mesh["shape"].tolist(), mesh["curved"].tolist()):
            if k not in keys:
                keys.append(k)
        work.append(dict(P=P, mesh=mesh, h=h, op=op, x=x, y=y, uh=uh, nc=nc, dofs=dofs, flops=flops,
                         bytes=bytes_, nblocks=len(keys), block_shapes=[k[0] for k in keys]))
    return work


def time_applies(work, steps, warmup, device, world, flush):
    """Device time of each Helmholtz apply (CUDA events on the launch stream),
    L2 flushed before every apply (outside the events).  Each apply launches
    its blocks one by one (hp_op_apply_block, the same launches hp_op_apply
    makes) with an event between launches, so every kernel's duration is
    measured inside the timed region too.  Returns per-apply ms (steps,
    orders) and per-block ms (list over orders of (steps, blocks))."""
    import torch
    from paper_2604_04644_gb300 import hp
    stream = torch.cuda.current_stream(device)
    for _ in range(warmup):
        for w in work:
            flush.zero_()
            hp.hp_op_apply(w["op"], 1.0, w["x"], w["y"], stream)
    for w in work:
        hp.hp_op_sync(w["op"], stream)
    ev = [[[torch.cuda.Event(enable_timing=True) for _ in range(w["nblocks"] + 1)] for w in work]
          for _ in range(steps)]
    torch.cuda.synchronize(device)
    barrier(world)
    torch.cuda.synchronize(device)
    for s in range(steps):
        for i, w in enumerate(work):
            flush.zero_()
            for b in range(w["nblocks"]):
                ev[s][i][b].record(stream)
                hp.hp_op_apply_block(w["op"], b, 1.0, w["x"], w["y"], stream)
            ev[s][i][-1].record(stream)
    torch.cuda.synchronize(device)
    barrier(world)
    torch.cuda.synchronize(device)
    for w in work:
        hp.hp_op_sync(w["op"], stream)
    per = np.array([[ev[s][i][0].elapsed_time(ev[s][i][-1]) for i in range(len(work))] for s in range(steps)])
    blocks = [np.array([[ev[s][i][b].elapsed_time(ev[s][i][b + 1]) for b in range(w["nblocks"])]
                        for s in range(steps)]) for i, w in enumerate(work)]
    return per, blocks


def time_e2e(work, steps, device):
    """Same workload through the public API with host buffers: pinned host ->
    device copy of the coefficients, apply, device -> host copy of the result,
    all inside the timed region.  The copies run on their own streams (one per
    direction), so one order's copies overlap the other orders' applies; each
    copy in waits for the previous step's apply of its order to free the input,
    each apply for its input and for the previous step's copy out of its output."""
    import torch
    from paper_2604_04644_gb300 import hp
    comp = torch.cuda.current_stream(device)
    s_in, s_out = torch.cuda.Stream(device), torch.cuda.Stream(device)
    hx = [torch.tensor(w["uh"], dtype=w["x"].dtype).pin_memory() for w in work]
    hy = [torch.empty(w["nc"], dtype=w["y"].dtype).pin_memory() for w in work]
    h2d = sum(t.numel() * t.element_size() for t in hx)
    d2h = sum(t.numel() * t.element_size() for t in hy)
    in_done = [torch.cuda.Event() for _ in work]
    applied = [torch.cuda.Event() for _ in work]
    out_done = [torch.cuda.Event() for _ in work]
    torch.cuda.synchronize(device)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(comp)
    s_in.wait_stream(comp)
    s_out.wait_stream(comp)
    for step in range(steps):
        for i, w in enumerate(work):
            with torch.cuda.stream(s_in):
                if step > 0:
                    s_in.wait_event(applied[i])
                w["x"].copy_(hx[i], non_blocking=True)
                in_done[i].record(s_in)
            comp.wait_event(in_done[i])
            if step > 0:
                comp.wait_event(out_done[i])
            hp.hp_op_apply(w["op"], 1.0, w["x"], w["y"], comp)
            applied[i].record(comp)
            with torch.cuda.stream(s_out):
                s_out.wait_event(applied[i])
                hy[i].copy_(w["y"], non_blocking=True)
                out_done[i].record(s_out)
    comp.wait_stream(s_in)
    comp.wait_stream(s_out)
    t1.record(comp)
    torch.cuda.synchronize(device)
    ms = t0.elapsed_time(t1) / steps
    dofs = sum(w["dofs"] for w in work)
    return {"value": dofs / (ms * 1e-3) / 1e9, "unit": "GDOF/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": ms,
            "copies": "own streams per direction, overlapping the other orders' applies"}


def shape_order_table(dtype_name, device, reps=5):
    """Per shape and order GDOF/s on single-shape slabs of the same cells
    (outside the headline): curved elements, and beside them the same cells
    affine (per-element factors, the metric rebuilt at the points)."""
    import torch
    from paper_2604_04644_gb300 import hp, inputs
    dt = hp.HP_FP64 if dtype_name == "f64" else hp.HP_FP32
    tdt = torch.float64 if dtype_name == "f64" else torch.float32
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda:%d" % device)
    stream = torch.cuda.current_stream(device)
    out = {}
    names = ("hex", "prism", "pyr", "tet")
    for s in range(4):
        for P in ORDERS:
            row = {}
            for curved in (True, False):
                mesh = inputs.slab_mesh(CELLS, CELLS, 4, P, curved=curved, slabs=(s,) * 4)
                h = hp.hp_mesh_create(mesh, device)
                co, po, nc, nph = hp.hp_mesh_layout(h, mesh["n_elem"])
                op = hp.hp_op_create(h, hp.HP_HELMHOLTZ, hp.HP_STRAT_SUMFAC, dt)
                x = torch.tensor(inputs.random_coefficients(1002, co), device="cuda:%d" % device, dtype=tdt)
                y = torch.zeros(nc, device="cuda:%d" % device, dtype=tdt)
                dofs, flops, bytes_ = hp.hp_op_work(op)
                ts = []
                for r in range(reps + 2):
                    flush.zero_()
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    hp.hp_op_apply(op, 1.0, x, y, stream)
                    b.record(stream)
                    b.synchronize()
                    if r >= 2:
                        ts.append(a.elapsed_time(b))
                hp.hp_op_sync(op, stream)
                t = statistics.median(ts) * 1e-3
                if curved:
                    row.update({"gdofs": round(dofs / t / 1e9, 3), "elements": int(mesh["n_elem"]),
                                "tflops": round(flops / t / 1e12, 4), "gbs": round(bytes_ / t / 1e9, 1)})
                else:
                    row.update({"affine_gdofs": round(dofs / t / 1e9, 3), "affine_tflops": round(flops / t / 1e12, 4)})
                hp.hp_op_destroy(op)
                hp.hp_mesh_destroy(h)
            out["%s_P%d" % (names[s], P)] = row
    return out


def precision_forms(work64, device, reps=10):
    """The reduced-precision forms on the same mesh and coefficients as the FP64
    workload: FP32 sum factorisation and the TF32 / BF16 tensor-core
    elemental-matrix operator (blocks over 256 modes: FP32 sum factorisation),
    GDOF/s (L2 flushed between applies) launched as the concurrent graph of
    the blocks (hp_op_apply_graph, `gdofs`) and block after block
    (hp_op_apply, `gdofs_per_block`), and the relative error against the FP64
    result."""
    import torch
    from paper_2604_04644_gb300 import hp
    dev = "cuda:%d" % device
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    out = {}
    for w in work64:
        y64 = torch.zeros_like(w["y"])
        hp.hp_op_apply(w["op"], 1.0, w["x"], y64)
        x32 = w["x"].float()
        y32 = torch.zeros(w["nc"], device=dev, dtype=torch.float32)
        row = {}
        for name, strat, dt in (("fp32_sumfac", hp.HP_STRAT_SUMFAC, hp.HP_FP32),
                                ("tf32_tensor_core", hp.HP_STRAT_ELEMAT, hp.HP_TF32),
                                ("bf16_tensor_core", hp.HP_STRAT_ELEMAT, hp.HP_BF16)):
            op = hp.hp_op_create(w["h"], hp.HP_HELMHOLTZ, strat, dt)
            med = {}
            for launch, fn in (("graph", hp.hp_op_apply_graph), ("per_block", hp.hp_op_apply)):
                for _ in range(3):
                    fn(op, 1.0, x32, y32)
                ts = []
                for _ in range(reps):
                    flush.zero_()
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record()
                    fn(op, 1.0, x32, y32)
                    b.record()
                    torch.cuda.synchronize(dev)
                    ts.append(a.elapsed_time(b))
                med[launch] = statistics.median(ts)
            hp.hp_op_sync(op)
            err = float((y32.double() - y64).abs().max() / y64.abs().max())
            row[name] = {"gdofs": round(w["dofs"] / (med["graph"] * 1e-3) / 1e9, 3),
                         "gdofs_per_block": round(w["dofs"] / (med["per_block"] * 1e-3) / 1e9, 3),
                         "rel_err_vs_fp64": float("%.3g" % err)}
            hp.hp_op_destroy(op)
        out["P%d" % w["P"]] = row
    return out


def reduced_precision_roofline(work64, device, hbm_peak, hbm_src, dtype_name="bf16", reps=10):
    """HBM roofline of the reduced-precision (BF16 or TF32) tensor-core form on
    the same mesh and coefficients as the FP64 workload.  Every block launch of
    every order is timed alone (CUDA events on the launching stream, L2 flushed
    before each); `achieved` = the block's algorithmic bytes (hp_op_block_work:
    FP32 coefficients in and out, FP16 metric factors at every point, two FP32
    scales and an 8-byte offset per element) / its time.  Returns the entry of
    the launch with the largest time (the form's dominant kernel; blocks over
    256 modes run FP32 sum factorisation) and, beside it, that of the dominant
    tensor-core launch."""
    import torch
    from paper_2604_04644_gb300 import hp
    dev = "cuda:%d" % device
    dt = hp.HP_BF16 if dtype_name == "bf16" else hp.HP_TF32
    stream = torch.cuda.current_stream(device)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    rows = []
    for w in work64:
        op = hp.hp_op_create(w["h"], hp.HP_HELMHOLTZ, hp.HP_STRAT_ELEMAT, dt)
        strat = hp.hp_op_strategies(op, w["nblocks"])
        x32 = w["x"].float()
        y32 = torch.zeros(w["nc"], device=dev, dtype=torch.float32)
        for _ in range(3):
            hp.hp_op_apply(op, 1.0, x32, y32, stream)
        for b in range(w["nblocks"]):
            ts = []
            for _ in range(reps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                hp.hp_op_apply_block(op, b, 1.0, x32, y32, stream)
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            n_el, dofs, fl, fx, by = hp.hp_op_block_work(op, b)
            tc = int(strat[b]) == hp.HP_STRAT_ELEMAT
            if tc:
                name = "tc_emat_kernel<%s,P%d,%s>" % (SHAPES[w["block_shapes"][b]], w["P"], dtype_name)
            else:
                name = "sf_kernel<%s,P%d,f32>" % (SHAPES[w["block_shapes"][b]], w["P"])
            t = statistics.median(ts) * 1e-3
            rows.append({"kernel": name, "tensor_core": tc, "elements": int(n_el), "launch_ms": round(t * 1e3, 4),
                         "achieved": round(by / t / 1e9, 1), "algorithmic_bytes": int(by),
                         "gdofs": round(dofs / t / 1e9, 3)})
        hp.hp_op_sync(op, stream)
        hp.hp_op_destroy(op)

    def entry(r):
        return {"bound": "hbm", "kernel": r["kernel"], "elements": r["elements"], "launch_ms": r["launch_ms"],
                "achieved": r["achieved"], "peak": hbm_peak, "unit": "GB/s",
                "frac": round(r["achieved"] / hbm_peak, 4), "traffic": MEASURED_TRAFFIC.get(r["kernel"]),
                "algorithmic_bytes": r["algorithmic_bytes"], "gdofs": r["gdofs"],
                "peak_source": hbm_src + " copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
    dom = max(rows, key=lambda r: r["launch_ms"])
    out = entry(dom)
    tcs = [r for r in rows if r["tensor_core"]]
    if tcs:
        out["tensor_core_dominant"] = entry(max(tcs, key=lambda r: r["launch_ms"]))
    out["launches_per_step"] = len(rows)
    return out


def strategy_table(device, orders=(1, 2, 4, 6, 8), reps=3):
    """GDOF/s per shape and order of the three strategies (sum-factorised
    collocated, elemental matrix, hybrid) for the mass and Helmholtz operators
    in FP64, on single-shape 16x16x4-cell curved slabs (the paper's strategy
    comparison per shape/order, Sec. 4)."""
    import torch
    from paper_2604_04644_gb300 import hp, inputs
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda:%d" % device)
    stream = torch.cuda.current_stream(device)
    names = ("hex", "prism", "pyr", "tet")
    out = {}
    for s in range(4):
        for P in orders:
            mesh = inputs.slab_mesh(CELLS, CELLS, 4, P, curved=True, slabs=(s,) * 4)
            h = hp.hp_mesh_create(mesh, device)
            co, po, nc, nph = hp.hp_mesh_layout(h, mesh["n_elem"])
            x = torch.tensor(inputs.random_coefficients(1002, co), device="cuda:%d" % device)
            y = torch.zeros(nc, device="cuda:%d" % device, dtype=torch.float64)
            row = {}
            for opname, kind in (("mass", hp.HP_MASS), ("helmholtz", hp.HP_HELMHOLTZ)):
                for sname, strat in (("sumfac", hp.HP_STRAT_SUMFAC), ("elemat", hp.HP_STRAT_ELEMAT),
                                     ("hybrid", hp.HP_STRAT_HYBRID)):
                    op = hp.hp_op_create(h, kind, strat, hp.HP_FP64)
                    dofs, flops, _ = hp.hp_op_work(op)
                    ts = []
                    for r in range(reps + 1):
                        flush.zero_()
                        a = torch.cuda.Event(enable_timing=True)
                        b = torch.cuda.Event(enable_timing=True)
                        a.record(stream)
                        hp.hp_op_apply(op, 1.0, x, y, stream)
                        b.record(stream)
                        b.synchronize()
                        if r:
                            ts.append(a.elapsed_time(b))
                    hp.hp_op_sync(op, stream)
                    hp.hp_op_destroy(op)
                    t = statistics.median(ts) * 1e-3
                    row["%s_%s" % (opname, sname)] = round(dofs / t / 1e9, 4)
            out["%s_P%d" % (names[s], P)] = row
            hp.hp_mesh_destroy(h)
    return out


def padaptive(device, reps=10):
    """p-adaptive batched apply: 40x40x32 cells of the four-slab mesh (192 000
    elements), P ~ U{2..8} per element (seed 3), affine for x < 0.5 and curved
    otherwise, FP64 Helmholtz.  One launch per (shape, P, curved) block on one
    stream vs one CUDA-graph launch with the blocks as concurrent nodes, with
    default and autotuned tiles."""
    import torch
    from paper_2604_04644_gb300 import hp, inputs
    mesh = inputs.slab_mesh(40, 40, 32, (2, 8), order_seed=3, curved_rule="x_half")
    h = hp.hp_mesh_create(mesh, device)
    co, po, nc, nph = hp.hp_mesh_layout(h, mesh["n_elem"])
    op = hp.hp_op_create(h, hp.HP_HELMHOLTZ, hp.HP_STRAT_SUMFAC, hp.HP_FP64)
    x = torch.tensor(inputs.random_coefficients(1003, co), device="cuda:%d" % device)
    y = torch.zeros(nc, device="cuda:%d" % device, dtype=torch.float64)
    dofs, flops, bytes_ = hp.hp_op_work(op)
    stream = torch.cuda.current_stream(device)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda:%d" % device)
    nblocks = len(set(zip(mesh["shape"].tolist(), mesh["P"].tolist(), mesh["curved"].tolist())))

    def timed(fn):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        hp.hp_op_sync(op, stream)
        return statistics.median(ts)

    t_stream = timed(lambda: hp.hp_op_apply(op, 1.0, x, y, stream))
    t_graph = timed(lambda: hp.hp_op_apply_graph(op, 1.0, x, y, stream))
    y_blocks = y.clone()
    # one persistent launch over a device work list (all blocks), plain and graph-captured
    hp.hp_op_set_batching(op, 1)
    t_wl = timed(lambda: hp.hp_op_apply(op, 1.0, x, y, stream))
    t_wl_graph = timed(lambda: hp.hp_op_apply_graph(op, 1.0, x, y, stream))
    wl_bitwise = bool(torch.equal(y, y_blocks))
    hp.hp_op_set_batching(op, 0)
    hp.hp_op_tune(op, 1.0, x, y, stream)
    tiles = hp.hp_op_tiles(op, nblocks)
    t_tuned = timed(lambda: hp.hp_op_apply_graph(op, 1.0, x, y, stream))
    hp.hp_op_destroy(op)
    # reduced-precision forms of the same batched apply (graph launches), with
    # their error against the FP64 result: FP32 sum factorisation; TF32 on the
    # tensor cores (elemental matrices, FP32 sum factorisation for blocks over
    # 256 modes); TF32 with each block's strategy chosen by measurement
    y64 = y.clone()
    x32 = x.float()
    y32 = torch.zeros(nc, device="cuda:%d" % device, dtype=torch.float32)
    forms = {}
    # scheduled forms: "exhaustive" times every block alone; "graph" searches on
    # the time of the whole concurrent graph (coordinate descent over blocks)
    for name, strat, dt, sched in (("fp64_graph_scheduled", hp.HP_STRAT_SUMFAC, hp.HP_FP64, "graph"),
                                   ("fp32_sumfac", hp.HP_STRAT_SUMFAC, hp.HP_FP32, None),
                                   ("fp32_graph_scheduled", hp.HP_STRAT_SUMFAC, hp.HP_FP32, "graph"),
                                   ("tf32_tensor_core", hp.HP_STRAT_ELEMAT, hp.HP_TF32, None),
                                   ("tf32_scheduled", hp.HP_STRAT_ELEMAT, hp.HP_TF32, "exhaustive"),
                                   ("tf32_graph_scheduled", hp.HP_STRAT_ELEMAT, hp.HP_TF32, "graph"),
                                   ("bf16_tensor_core", hp.HP_STRAT_ELEMAT, hp.HP_BF16, None),
                                   ("bf16_graph_scheduled", hp.HP_STRAT_ELEMAT, hp.HP_BF16, "graph")):
        op = hp.hp_op_create(h, hp.HP_HELMHOLTZ, strat, dt)
        xi, yo = (x, y) if dt == hp.HP_FP64 else (x32, y32)
        if sched == "exhaustive":
            hp.hp_op_schedule_exhaustive(op, 1.0, xi, yo, nblocks, stream)
        elif sched == "graph":
            hp.hp_op_schedule_graph(op, 1.0, xi, yo, 5, 2 if dt in (hp.HP_TF32, hp.HP_BF16) else 1, stream)
        ms = timed(lambda: hp.hp_op_apply_graph(op, 1.0, xi, yo, stream))
        st = hp.hp_op_strategies(op, nblocks)
        err = float((yo.double() - y64).abs().max() / y64.abs().max())
        forms[name] = {"ms": round(ms, 4), "gdofs": round(dofs / (ms * 1e-3) / 1e9, 4),
                       "rel_err_vs_fp64": float("%.3g" % err),
                       "blocks_on_tensor_core": int((st == hp.HP_STRAT_ELEMAT).sum()) if dt in (hp.HP_TF32, hp.HP_BF16) else 0,
                       "strategy_histogram": {k: int((st == v).sum()) for k, v in
                                              (("sumfac", 0), ("elemat", 1), ("hybrid", 2), ("matrix", 4)) if (st == v).any()}}
        hp.hp_op_destroy(op)
    hp.hp_mesh_destroy(h)
    g = lambda ms: round(dofs / (ms * 1e-3) / 1e9, 4)
    return {"workload": "helmholtz_padaptive_40x40x32_P2-8_affine_curved_halves", "elements": int(mesh["n_elem"]),
            "reduced_precision_graph": forms,
            "dofs": int(dofs), "blocks": nblocks, "dtype": "f64",
            "per_block_launches": {"ms": round(t_stream, 4), "gdofs": g(t_stream)},
            "graph": {"ms": round(t_graph, 4), "gdofs": g(t_graph)},
            "persistent_worklist": {"ms": round(t_wl, 4), "gdofs": g(t_wl), "bitwise_equal_to_per_block": wl_bitwise},
            "persistent_worklist_graph": {"ms": round(t_wl_graph, 4), "gdofs": g(t_wl_graph)},
            "graph_autotuned": {"ms": round(t_tuned, 4), "gdofs": g(t_tuned),
                                "tiles_histogram": np.bincount(tiles, minlength=3).tolist()},
            "tflops_graph_autotuned": round(flops / (t_tuned * 1e-3) / 1e12, 4)}


def _oracle_sample(target_s):
    """Time the oracle (plain FP64 numpy definition) on a bounded sample of the
    workload: Helmholtz on a random subset of elements at each order, each
    subset grown until it takes about target_s / 32 s.  Returns (output DOFs,
    seconds, sample description)."""
    from oracle import operators as oracle_ops
    from paper_2604_04644_gb300 import inputs
    rng = np.random.default_rng(0)
    dofs = 0
    t_total = 0.0
    per = max(1, int(target_s / len(ORDERS) * 1.0))
    sample_desc = []
    for P in ORDERS:
        mesh = inputs.slab_mesh(CELLS, CELLS, CELLS, P, curved=True)
        co, po = oracle_ops.layout(mesh)
        uh = inputs.random_coefficients(1002, co)
        oracle_ops.apply("helmholtz", mesh, uh, 1.0, elems=[0])     # builds the reference tables (setup)
        n = 64
        while True:
            el = np.sort(rng.choice(mesh["n_elem"], min(n, mesh["n_elem"]), replace=False))
            t0 = time.perf_counter()
            oracle_ops.apply("helmholtz", mesh, uh, 1.0, elems=el)
            dt = time.perf_counter() - t0
            if dt > per / 4 or n >= mesh["n_elem"]:
                break
            n *= 4
        dofs += int(sum(co[e + 1] - co[e] for e in el))
        t_total += dt
        sample_desc.append("P%d:%d" % (P, len(el)))
    return dofs, t_total, sample_desc


def cpu_baseline(target_s=12.0, one_thread=True):
    """The oracle on the host cores, all of them (numpy's thread pool) and, in
    a child process whose BLAS / OpenMP pools are limited to one thread, one
    core; GDOF/s on a bounded sample of the workload (see _oracle_sample)."""
    nproc = os.cpu_count()
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        cores = nproc
    dofs, t_total, desc = _oracle_sample(target_s)
    out = {"value": dofs / t_total / 1e9, "unit": "GDOF/s", "cores": int(cores), "nproc": int(nproc or 0),
           "kind": "oracle",
           "sample": "Helmholtz on random element subsets of the 16^3 mixed curved mesh (" + ",".join(desc) +
                     "), %.1f s of CPU work" % t_total}
    if one_thread:
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
                   NUMEXPR_NUM_THREADS="1")
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", str(target_s)], env=env,
                           capture_output=True, text=True, timeout=600)
        try:
            d1, t1, desc1 = json.loads(r.stdout.strip().splitlines()[-1])
            out["one_thread"] = {"value": d1 / t1 / 1e9, "cores": 1, "seconds": round(t1, 2),
                                 "sample": ",".join(desc1)}
        except Exception:
            out["one_thread"] = {"error": (r.stderr or r.stdout)[-300:]}
    return out


def run_reference(args, world, rank):
    if rank != 0:
        return
    for _ in range(args.warmup):
        pass
    vals = []
    t0 = time.time()
    cb = None
    for _ in range(max(args.steps, 1)):
        cb = cpu_baseline(target_s=max(4.0, 60.0 / max(args.steps, 1)), one_thread=False)
        vals.append(cb["value"])
    v = statistics.median(vals)
    line = {"metric": METRIC, "value": v, "unit": "GDOF/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": (time.time() - t0) * 1e3 / max(args.steps, 1),
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "helmholtz_mixed_16cube_P1-8_curved", "cells": "16x16x16",
                       "orders": "1..8", "Q": "P+2", "lambda": 1.0, "l2": "n/a (CPU)"},
            "cpu_baseline": dict(cb, value=v),
            "e2e": {"value": v, "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_costmodel(local):
    """Learned strategy scheduling (--costmodel): timings over shape x P = 1..10
    x affine/curved x 128..65 536 elements x {FP64, FP32, BF16}, each strategy
    of each block timed alone by the library; one MLP per operator (6 inputs:
    block features and launch mode, 4 outputs: log times of sum factorisation,
    elemental matrix, hybrid, stored matrices) trained on the GPU by the
    library's kernels; evaluated on a held-out 16x16x32-cell mesh with
    P ~ U{3..9} and affine/curved halves, launched as the concurrent graph."""
    import torch
    from paper_2604_04644_gb300 import costmodel, hp, inputs
    torch.cuda.set_device(local)
    held = inputs.slab_mesh(16, 16, 32, (3, 9), order_seed=4, curved_rule="x_half")
    res = {}
    for name, kind in (("helmholtz", hp.HP_HELMHOLTZ), ("mass", hp.HP_MASS)):
        t0 = time.time()
        recs = costmodel.generate_timings(local, kind)
        t_gen = time.time() - t0
        X, T = costmodel.training_set(recs)
        t0 = time.time()
        mlp, hist = costmodel.train(X, T, local)
        t_train = time.time() - t0
        pred = costmodel.predict(mlp, X, local)
        row = {"samples": int(len(X)), "extrapolated_entries": int(sum(sum(r["extrapolated"]) for r in recs)),
               "timing_s": round(t_gen, 1), "train_s": round(t_train, 1),
               "train_loss_first_last": [hist[0][1], hist[-1][1]],
               "train_rmse_log10": float(np.sqrt(np.mean((pred - T) ** 2))),
               "train_argmin_accuracy": float(np.mean(pred.argmin(1) == T.argmin(1)))}
        for dn, dt in (("f64", hp.HP_FP64), ("f32", hp.HP_FP32), ("bf16", hp.HP_BF16)):
            row["held_out_%s" % dn] = costmodel.evaluate_schedules(mlp, held, kind, dt, local, graph=True)
        res[name] = row
        hp.hp_mlp_destroy(mlp)
    print(json.dumps({"costmodel": res, "held_out_mesh": {"cells": "16x16x32", "elements": int(held["n_elem"]),
                                                          "orders": "U{3..9}", "curved": "x >= 0.5"}}), flush=True)


def costmodel_summary(local):
    """Compact cost-model key of the default bench line: Helmholtz timings the
    library generates (four shapes, P = 1..8, affine / curved, 512 / 4 096 /
    32 768 elements, FP64 and BF16, each strategy of each block timed alone),
    the 6 -> 64 -> 64 -> 4 network trained on them by the library's kernels,
    and the graph-launch time of a held-out mesh (16x16x16 cells of the
    four-slab construction, P ~ U{1..8}, affine / curved halves) under the
    paper's rule, the network's schedule, each block's fastest strategy timed
    alone, and the search on the whole graph's time."""
    from paper_2604_04644_gb300 import costmodel, hp, inputs
    t0 = time.time()
    recs = costmodel.generate_timings(local, hp.HP_HELMHOLTZ, orders=range(1, 9), sizes=(512, 4096, 32768),
                                      dtypes=(hp.HP_FP64, hp.HP_BF16), budget_ms=20.0, reps=2)
    t_gen = time.time() - t0
    X, T = costmodel.training_set(recs)
    mlp, hist = costmodel.train(X, T, local)
    held = inputs.slab_mesh(16, 16, 16, (1, 8), order_seed=4, curved_rule="x_half")
    out = {"timing_s": round(t_gen, 1), "samples": int(len(X)),
           "train_loss_first_last": [round(hist[0][1], 5), round(hist[-1][1], 5)],
           "held_out": {"cells": "16x16x16", "elements": int(held["n_elem"]), "orders": "U{1..8}",
                        "curved": "x >= 0.5", "launch": "hp_op_apply_graph"}}
    keep = ("rule_ms", "mlp_ms", "exhaustive_alone_ms", "graph_search_ms", "choices_mlp",
            "choices_graph_search", "rule_over_mlp", "mlp_over_best_searched")
    try:
        for dn, dt in (("helmholtz_f64", hp.HP_FP64), ("helmholtz_bf16", hp.HP_BF16)):
            ev = costmodel.evaluate_schedules(mlp, held, hp.HP_HELMHOLTZ, dt, local, graph=True)
            out[dn] = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in ev.items() if k in keep}
    finally:
        hp.hp_mlp_destroy(mlp)
    return out


def run_solve(local, cells, order=4, lam=1.0, tol=1e-10, scheduled=False):
    """Time to solution of the C0-assembled Helmholtz problem on the conforming
    four-slab mesh (cells^3 cells + pyramid-to-tet transition layer, curved),
    P = order, f = (3 pi^2 + lambda) sin(pi x) sin(pi y) sin(pi z).  With
    `scheduled`, also the FP64, FP32-inner and BF16-inner solves with the
    operators' strategies chosen by the graph-aware schedule."""
    import torch
    from paper_2604_04644_gb300 import hp, inputs
    torch.cuda.set_device(local)
    dev = "cuda:%d" % local
    t0 = time.time()
    mesh = inputs.c0_slab_mesh(cells, order, curved=True)
    h = hp.hp_mesh_create(mesh, local)
    co, po, nc, nph = hp.hp_mesh_layout(h, mesh["n_elem"])
    t_mesh = time.time() - t0
    t0 = time.time()
    c0 = hp.hp_c0_create(h)
    ng, nb = hp.hp_c0_info(c0)
    t_c0 = time.time() - t0
    xyz = torch.empty(3 * nph, device=dev, dtype=torch.float64)
    hp.hp_mesh_points(h, xyz)
    x, y, z = xyz.view(3, -1)
    f = (3 * np.pi ** 2 + lam) * torch.sin(np.pi * x) * torch.sin(np.pi * y) * torch.sin(np.pi * z)
    del xyz, x, y, z
    ip = hp.hp_op_create(h, hp.HP_IPRODUCT_WRT_BASE)
    bl = torch.empty(nc, device=dev, dtype=torch.float64)
    hp.hp_op_apply(ip, 1.0, f.contiguous(), bl)
    hp.hp_op_destroy(ip)
    del f
    b = torch.empty(ng, device=dev, dtype=torch.float64)
    hp.hp_c0_assemble(c0, bl, b, True)
    del bl
    out = {"workload": "helmholtz_c0_solve_%dcube_P%d_curved" % (cells, order), "elements": int(mesh["n_elem"]),
           "local_dofs": int(nc), "global_dofs": int(ng), "dirichlet_dofs": int(nb), "tol": tol,
           "setup_s": {"mesh": round(t_mesh, 2), "c0_map": round(t_c0, 2)}}
    # warm-up (builds the Jacobi diagonal, operators and workspaces) then timed solves
    xw = torch.zeros(ng, device=dev, dtype=torch.float64)
    hp.hp_solve(c0, lam, b, xw, tol=1e-2, mixed=3, inner_tol=1e-1, max_refinements=1)
    hp.hp_solve(c0, lam, b, xw, tol=1e-2, mixed=2, inner_tol=1e-1, max_refinements=1)
    hp.hp_solve(c0, lam, b, xw, tol=1e-2, mixed=True, inner_tol=1e-1, max_refinements=1)
    hp.hp_solve(c0, lam, b, xw, tol=1e-2)
    sols = {}
    for name, kw in (("fp64_pcg", dict(mixed=False)), ("mixed_fp32_pcg_fp64_ir", dict(mixed=True, inner_tol=1e-4)),
                     ("mixed_tf32_tensor_core_pcg_fp64_ir", dict(mixed=2, inner_tol=1e-3)),
                     ("mixed_bf16_tensor_core_pcg_fp64_ir", dict(mixed=3, inner_tol=1e-2))):
        xs = torch.zeros(ng, device=dev, dtype=torch.float64)
        torch.cuda.synchronize(dev)
        t0 = time.time()
        rc, st = hp.hp_solve(c0, lam, b, xs, tol=tol, **kw)
        torch.cuda.synchronize(dev)
        dt = time.time() - t0
        out[name] = dict(st, seconds=round(dt, 4), status=hp.hp_status_str(rc))
        if rc:
            out[name]["error"] = hp.hp_last_error()
        sols[name] = xs
    # the same solves with the operators' per-block strategies chosen by the
    # graph-aware schedule (stored matrices included); the first solve of each
    # kind schedules (its time is reported as setup), the second is timed
    sched_setup = {}
    sched_forms = (("fp64_pcg_scheduled", dict(mixed=False)),
                   ("mixed_fp32_pcg_fp64_ir_scheduled", dict(mixed=True, inner_tol=1e-4)),
                   ("mixed_bf16_tensor_core_pcg_fp64_ir_scheduled", dict(mixed=3, inner_tol=1e-2)))
    for name, kw in sched_forms if scheduled else ():
        torch.cuda.synchronize(dev)
        t0 = time.time()
        hp.hp_solve(c0, lam, b, xw, tol=1e-2, max_refinements=1, schedule=True,
                    **dict(kw, inner_tol=1e-1) if kw["mixed"] else kw)
        torch.cuda.synchronize(dev)
        sched_setup[name] = round(time.time() - t0, 2)
        xs = torch.zeros(ng, device=dev, dtype=torch.float64)
        torch.cuda.synchronize(dev)
        t0 = time.time()
        rc, st = hp.hp_solve(c0, lam, b, xs, tol=tol, schedule=True, **kw)
        torch.cuda.synchronize(dev)
        dt = time.time() - t0
        out[name] = dict(st, seconds=round(dt, 4), status=hp.hp_status_str(rc))
        if rc:
            out[name]["error"] = hp.hp_last_error()
        sols[name] = xs
    if scheduled:
        out["setup_s"]["schedule_first_solve"] = sched_setup
    for name, tag in (("mixed_fp32_pcg_fp64_ir", "mixed"), ("mixed_tf32_tensor_core_pcg_fp64_ir", "tf32_tc"),
                      ("mixed_bf16_tensor_core_pcg_fp64_ir", "bf16_tc"), ("fp64_pcg_scheduled", "fp64_scheduled"),
                      ("mixed_fp32_pcg_fp64_ir_scheduled", "mixed_scheduled"),
                      ("mixed_bf16_tensor_core_pcg_fp64_ir_scheduled", "bf16_tc_scheduled")):
        if name not in sols:
            continue
        d = sols["fp64_pcg"] - sols[name]
        out["rel_diff_%s_vs_fp64" % tag] = float(d.norm() / sols["fp64_pcg"].norm())
        out["speedup_%s_vs_fp64" % tag] = round(out["fp64_pcg"]["seconds"] / out[name]["seconds"], 3)
    hp.hp_c0_destroy(c0)
    hp.hp_mesh_destroy(h)
    return out


# large single-shape blocks of the per-block precision table: (shape, P, elements)
BLOCK_TABLE = [(3, 2, 65536), (3, 4, 65536), (3, 6, 32768), (3, 8, 32768), (2, 4, 65536), (2, 6, 32768),
               (1, 4, 65536), (0, 4, 65536), (0, 5, 32768), (0, 6, 16384), (0, 7, 16384)]


def run_block_table(local, reps=10):
    """Helmholtz GDOF/s of FP32 sum factorisation and of the TF32 / BF16
    tensor-core elemental matrix and hybrid on large single-shape blocks,
    curved and affine (L2 flushed before every apply; median of `reps`), one
    JSON line per block; null where the form is not built for the block."""
    import torch
    from paper_2604_04644_gb300 import hp, inputs
    torch.cuda.set_device(local)
    dev = "cuda:%d" % local
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    for shape, P, n in BLOCK_TABLE:
        for curved in (True, False):
            mesh = inputs.replicated_mesh(shape, P, n, curved=curved)
            h = hp.hp_mesh_create(mesh, local)
            co, po, nc, nph = hp.hp_mesh_layout(h, mesh["n_elem"])
            x = torch.tensor(inputs.random_coefficients(5, co), device=dev, dtype=torch.float32)
            y = torch.zeros(nc, device=dev, dtype=torch.float32)
            line = {"shape": SHAPES[shape], "P": P, "curved": curved, "elements": n}
            for name, strat, dt in (("fp32_sumfac", hp.HP_STRAT_SUMFAC, hp.HP_FP32),
                                    ("tf32_tensor_core", hp.HP_STRAT_ELEMAT, hp.HP_TF32),
                                    ("bf16_tensor_core", hp.HP_STRAT_ELEMAT, hp.HP_BF16),
                                    ("tf32_tc_hybrid", hp.HP_STRAT_HYBRID, hp.HP_TF32),
                                    ("bf16_tc_hybrid", hp.HP_STRAT_HYBRID, hp.HP_BF16)):
                op = hp.hp_op_create(h, hp.HP_HELMHOLTZ, strat, dt)
                try:   # the form itself, also where the operator starts the block on another one
                    hp.hp_op_strategies(op, 1, [strat])
                except hp.HpError:   # not built for this block
                    hp.hp_op_destroy(op)
                    line[name] = None
                    continue
                for _ in range(3):
                    hp.hp_op_apply(op, 1.0, x, y)
                ts = []
                for _ in range(reps):
                    flush.zero_()
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record()
                    hp.hp_op_apply(op, 1.0, x, y)
                    b.record()
                    b.synchronize()
                    ts.append(a.elapsed_time(b))
                hp.hp_op_sync(op)
                line[name] = round(nc / (statistics.median(ts) * 1e-3) / 1e9, 2)
                hp.hp_op_destroy(op)
            hp.hp_mesh_destroy(h)
            print(json.dumps({"block_table": line}), flush=True)


# collapsed-shape blocks of the reduced-rule study: (shape, P, elements)
REDUCED_Q = [(3, 2, 65536), (3, 4, 65536), (3, 6, 32768), (3, 8, 32768), (2, 4, 65536), (2, 6, 32768),
             (1, 4, 65536), (1, 6, 32768)]


def run_reduced_q(local, reps=10):
    """The reduced quadrature rule (Q - 1 points in the collapsed directions)
    against the full one: Helmholtz GDOF/s of the BF16 and TF32 tensor-core
    elemental-matrix operator on large curved single-shape blocks (L2 flushed
    before every apply; median of `reps`), the points per element of each rule
    and the relative difference of the two FP64 elemental-matrix results (the
    quadrature error the reduced rule adds on curved elements)."""
    import torch
    from paper_2604_04644_gb300 import hp, inputs
    torch.cuda.set_device(local)
    dev = "cuda:%d" % local
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    for shape, P, n in REDUCED_Q:
        line = {"shape": SHAPES[shape], "P": P, "elements": n}
        ys = {}
        for rq in (0, 1):
            mesh = inputs.replicated_mesh(shape, P, n, curved=True)
            mesh["quadrature"] = rq
            h = hp.hp_mesh_create(mesh, local)
            co, po, nc, nph = hp.hp_mesh_layout(h, mesh["n_elem"])
            line["points_" + ("reduced" if rq else "full")] = int(po[1] - po[0])
            x = torch.tensor(inputs.random_coefficients(5, co), device=dev, dtype=torch.float64)
            y = torch.zeros(nc, device=dev, dtype=torch.float64)
            op = hp.hp_op_create(h, hp.HP_HELMHOLTZ, hp.HP_STRAT_ELEMAT, hp.HP_FP64)
            hp.hp_op_apply(op, 1.0, x, y)
            hp.hp_op_sync(op)
            ys[rq] = y.clone()
            hp.hp_op_destroy(op)
            x32, y32 = x.float(), torch.zeros(nc, device=dev, dtype=torch.float32)
            for name, dt in (("bf16", hp.HP_BF16), ("tf32", hp.HP_TF32)):
                op = hp.hp_op_create(h, hp.HP_HELMHOLTZ, hp.HP_STRAT_ELEMAT, dt)
                for _ in range(3):
                    hp.hp_op_apply(op, 1.0, x32, y32)
                ts = []
                for _ in range(reps):
                    flush.zero_()
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record()
                    hp.hp_op_apply(op, 1.0, x32, y32)
                    b.record()
                    b.synchronize()
                    ts.append(a.elapsed_time(b))
                hp.hp_op_sync(op)
                line["%s_%s" % (name, "reduced" if rq else "full")] = round(nc / (statistics.median(ts) * 1e-3) / 1e9, 2)
                hp.hp_op_destroy(op)
            hp.hp_mesh_destroy(h)
        line["rel_diff_fp64"] = float("%.3g" % float((ys[1] - ys[0]).abs().max() / ys[0].abs().max()))
        print(json.dumps({"reduced_q": line}), flush=True)


# two-dimensional blocks: (cells, P, cells per side of the unit square)
TWO_D = [("quad", 2, 500), ("quad", 4, 400), ("quad", 8, 250), ("tri", 2, 400), ("tri", 4, 300), ("tri", 8, 200)]


def run_two_d(local, reps=10):
    """The paper's two-dimensional formulation (Sec. 2.2) on this GPU:
    Helmholtz GDOF/s of the collocated sum factorisation on curved
    quadrilateral / triangle meshes of the unit square, FP64 and FP32 (L2
    flushed before every apply; median of `reps`), with the FP64 rate against
    the measured FP64 FMA peak (flops: the passes the kernel runs, FMA = 2)."""
    import torch
    from paper_2604_04644_gb300 import hp, inputs
    torch.cuda.set_device(local)
    dev = "cuda:%d" % local
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    for cells, P, nx in TWO_D:
        mesh = inputs.square_mesh_2d(nx, nx, P, cells=cells, curved=True)
        h = hp.hp_mesh2d_create(mesh, local)
        co, po = hp.hp_mesh2d_layout(h, mesh["n_elem"])
        n, Q = P + 1, P + 2
        rows = n * n if cells == "quad" else (2 * n + sum(P - f for f in range(1, P)))
        # FMAs per element: eta_2 / eta_1 passes of B and B^T, two collocation
        # derivatives and their transposes, the metric (5) and the mass term (2)
        fma = 2 * (rows * Q + n * Q * Q) + 4 * Q * Q * Q + 7 * Q * Q
        line = {"shape": cells, "P": P, "elements": int(mesh["n_elem"]), "dofs": int(co[-1])}
        for name, dt, tdt in (("fp64", hp.HP_FP64, torch.float64), ("fp32", hp.HP_FP32, torch.float32)):
            x = torch.rand(int(co[-1]), device=dev, dtype=tdt)
            y = torch.empty_like(x)
            for _ in range(3):
                hp.hp_op2d_apply(h, hp.HP_HELMHOLTZ, dt, 1.0, x, y)
            ts = []
            for _ in range(reps):
                flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record()
                hp.hp_op2d_apply(h, hp.HP_HELMHOLTZ, dt, 1.0, x, y)
                b.record()
                b.synchronize()
                ts.append(a.elapsed_time(b))
            ms = statistics.median(ts)
            line[name + "_gdofs"] = round(co[-1] / (ms * 1e-3) / 1e9, 2)
            line[name + "_tflops"] = round(2.0 * fma * mesh["n_elem"] / (ms * 1e-3) / 1e12, 3)
        hp.hp_mesh2d_destroy(h)
        print(json.dumps({"two_d": line}), flush=True)


def run_collocation_study(local, reps=10):
    """The paper's collocation study (Sec. 5) on this GPU: FP64 Helmholtz
    GDOF/s of the collocated sum factorisation (derivatives by collocation at
    the points) and of the non-collocated form (derivatives by sum
    factorisation with the derivative tables), on regular (affine) single-shape
    blocks of about six million DOFs, P = 1..8 (L2 flushed before every apply;
    median of `reps`), one JSON line per (shape, P)."""
    import torch
    from paper_2604_04644_gb300 import hp, inputs
    torch.cuda.set_device(local)
    dev = "cuda:%d" % local
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    for shape in range(4):
        for P in range(1, 9):
            n = min(200000, max(4096, int(6e6 / N_MODES[shape](P))))
            mesh = inputs.replicated_mesh(shape, P, n, curved=False)
            h = hp.hp_mesh_create(mesh, local)
            co, po, nc, nph = hp.hp_mesh_layout(h, mesh["n_elem"])
            x = torch.tensor(inputs.random_coefficients(5, co), device=dev, dtype=torch.float64)
            y = torch.zeros(nc, device=dev, dtype=torch.float64)
            line = {"shape": SHAPES[shape], "P": P, "elements": int(mesh["n_elem"]), "dofs": int(nc)}
            op = hp.hp_op_create(h, hp.HP_HELMHOLTZ, hp.HP_STRAT_SUMFAC, hp.HP_FP64)
            for name, coll in (("collocated", True), ("noncollocated", False)):
                hp.hp_op_set_collocated(op, coll)
                for _ in range(3):
                    hp.hp_op_apply(op, 1.0, x, y)
                ts = []
                for _ in range(reps):
                    flush.zero_()
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record()
                    hp.hp_op_apply(op, 1.0, x, y)
                    b.record()
                    b.synchronize()
                    ts.append(a.elapsed_time(b))
                hp.hp_op_sync(op)
                line[name] = round(nc / (statistics.median(ts) * 1e-3) / 1e9, 3)
            line["collocated_over_noncollocated"] = round(line["collocated"] / line["noncollocated"], 3)
            hp.hp_op_destroy(op)
            hp.hp_mesh_destroy(h)
            print(json.dumps({"collocation_study": line}), flush=True)


def run_matrix_study(local, reps=10):
    """Matrix-based (stored per-element dense H^e, HP_STRAT_MATRIX) against
    matrix-free sum factorisation: Helmholtz GDOF/s in FP64 and FP32 on curved
    single-shape blocks of about four million DOFs and at least 256 MB of FP32
    stored matrices and vectors, P = 1..5 (blocks of at most
    256 modes), with the build time, the stored bytes and the stored-matrix
    apply's HBM rate against the measured copy bandwidth (L2 flushed before
    every apply; median of `reps`). One JSON line per (shape, P)."""
    import torch
    from paper_2604_04644_gb300 import hp, inputs
    torch.cuda.set_device(local)
    dev = "cuda:%d" % local
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    try:
        hbm_peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except (OSError, KeyError, ValueError):
        hbm_peak = 6800.0
    def timed(op, x, y):
        for _ in range(3):
            hp.hp_op_apply(op, 1.0, x, y)
        ts = []
        for _ in range(reps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            hp.hp_op_apply(op, 1.0, x, y)
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        hp.hp_op_sync(op)
        return statistics.median(ts) * 1e-3
    for shape in range(4):
        for P in range(1, 6):
            NP = N_MODES[shape](P)
            if NP > 256:
                continue
            # about four million DOFs, and at least 256 MB (twice L2) of stored
            # FP32 matrices, coefficients and offsets, at most four million elements
            n = min(4000000, max(4096, int(4e6 / NP), int(256e6 / (4 * NP * NP + 8 * NP + 8))))
            mesh = inputs.replicated_mesh(shape, P, n, curved=True)
            h = hp.hp_mesh_create(mesh, local)
            co, po, nc, nph = hp.hp_mesh_layout(h, mesh["n_elem"])
            ne = int(mesh["n_elem"])
            line = {"shape": SHAPES[shape], "P": P, "modes": NP, "elements": ne, "dofs": int(nc)}
            xs = inputs.random_coefficients(5, co)
            for dname, dt, tdt, vs in (("f64", hp.HP_FP64, torch.float64, 8), ("f32", hp.HP_FP32, torch.float32, 4)):
                x = torch.tensor(xs, device=dev, dtype=tdt)
                y = torch.zeros(nc, device=dev, dtype=tdt)
                op = hp.hp_op_create(h, hp.HP_HELMHOLTZ, hp.HP_STRAT_SUMFAC, dt)
                line["sumfac_" + dname] = round(nc / timed(op, x, y) / 1e9, 3)
                hp.hp_op_destroy(op)
                op = hp.hp_op_create(h, hp.HP_HELMHOLTZ, hp.HP_STRAT_MATRIX, dt)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                hp.hp_op_apply(op, 1.0, x, y)           # builds the stored matrices
                hp.hp_op_sync(op)
                line["build_s_" + dname] = round(time.perf_counter() - t0, 3)
                t = timed(op, x, y)
                line["matrix_" + dname] = round(nc / t / 1e9, 3)
                algo = ne * (NP * NP * vs + 2 * NP * vs + 8)          # stored H^e, in, out, offsets
                line["matrix_gbs_" + dname] = round(algo / t / 1e9, 1)
                line["matrix_hbm_frac_" + dname] = round(algo / t / 1e9 / hbm_peak, 3)
                line["stored_gb_" + dname] = round(ne * NP * NP * vs / 1e9, 3)
                hp.hp_op_destroy(op)
            hp.hp_mesh_destroy(h)
            print(json.dumps({"matrix_study": line}), flush=True)


def run_profile_case(name, local):
    """One block of curved elements (or the bench mesh at one order), three
    Helmholtz applies (the capture takes one)."""
    import torch
    from paper_2604_04644_gb300 import hp, inputs
    torch.cuda.set_device(local)
    shape, P, n, strat, dt = PROFILE_CASES[name]
    if shape < 0:
        mesh = inputs.slab_mesh(CELLS, CELLS, CELLS, P, curved=True)
    else:
        mesh = inputs.replicated_mesh(shape, P, n, curved=True)
    h = hp.hp_mesh_create(mesh, local)
    co, po, nc, nph = hp.hp_mesh_layout(h, mesh["n_elem"])
    x = torch.tensor(inputs.random_coefficients(5, co), device="cuda:%d" % local, dtype=torch.float32)
    y = torch.zeros(nc, device="cuda:%d" % local, dtype=torch.float32)
    op = hp.hp_op_create(h, hp.HP_HELMHOLTZ, getattr(hp, "HP_STRAT_" + strat), getattr(hp, "HP_" + dt))
    for _ in range(3):
        hp.hp_op_apply(op, 1.0, x, y)
    hp.hp_op_sync(op)
    hp.hp_op_destroy(op)
    hp.hp_mesh_destroy(h)
    print(json.dumps({"profile_case": name, "elements": int(mesh["n_elem"]), "ok": True}), flush=True)


def main():
    args = parse()
    if args.oracle_sample is not None:     # the one-thread leg of cpu_baseline (a child process)
        print(json.dumps(_oracle_sample(args.oracle_sample)), flush=True)
        return
    world, rank, local = dist_init(args)
    if args.profile_case:
        if rank == 0:
            run_profile_case(args.profile_case, local)
        return
    if args.block_table:
        if rank == 0:
            run_block_table(local)
        return
    if args.two_d:
        if rank == 0:
            run_two_d(local)
        return
    if args.reduced_q:
        if rank == 0:
            run_reduced_q(local)
        return
    if args.collocation_study:
        if rank == 0:
            run_collocation_study(local)
        return
    if args.matrix_study:
        if rank == 0:
            run_matrix_study(local)
        return
    if args.solve:
        if rank == 0:
            print(json.dumps({"solve": run_solve(local, args.cells or 64, scheduled=True)}), flush=True)
        return
    if args.costmodel:
        if rank == 0:
            run_costmodel(local)
        return
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import torch
    from paper_2604_04644_gb300 import hp
    torch.cuda.set_device(local)
    work = build_workloads(args.dtype, local, world, rank)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda:%d" % local)  # 256 MiB > L2
    with ClockSampler(local) as clk:
        per, per_block = time_applies(work, args.steps, args.warmup, local, world, flush)
        fp64_peak, fp64_peak_ms = (hp.hp_peak_fp64(local) if args.dtype == "f64" else (None, None))
    dofs_step = sum(w["dofs"] for w in work)
    flops_step = sum(w["flops"] for w in work)
    bytes_step = sum(w["bytes"] for w in work)
    ms_step, value = split_scaling_value(world, dofs_step, float(per.sum(axis=1).mean()),
                                         device="cuda:%d" % local)
    e2e = time_e2e(work, max(2, args.steps // 2), local)
    if world > 1:   # the whole job: all ranks' DOFs and bytes over the slowest rank's time
        e2e["ms_per_step"] = max_over_ranks(world, e2e["ms_per_step"], device="cuda:%d" % local)
        e2e["value"] = sum_over_ranks(world, float(dofs_step), device="cuda:%d" % local) / \
            (e2e["ms_per_step"] * 1e-3) / 1e9
        for k in ("h2d_bytes_per_step", "d2h_bytes_per_step"):
            e2e[k] = int(sum_over_ranks(world, float(e2e[k]), device="cuda:%d" % local))
    launches = args.steps * sum(w["nblocks"] for w in work)
    per_order = {}
    for i, w in enumerate(work):
        t = float(per[:, i].mean()) * 1e-3
        per_order["P%d" % w["P"]] = {"gdofs": round(w["dofs"] / t / 1e9, 3),
                                     "tflops": round(w["flops"] / t / 1e12, 4),
                                     "gbs": round(w["bytes"] / t / 1e9, 1)}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        hbm_peak, hbm_src = peaks["hbm_gbs"], "measured"
    except Exception:
        hbm_peak, hbm_src = 6800.0, "fallback"
    achieved_tf = flops_step / (ms_step * 1e-3) / 1e12
    achieved_gbs = bytes_step / (ms_step * 1e-3) / 1e9
    # the dominant kernel: the block launch with the largest share of the timed region
    dom = max(((i, b) for i, w in enumerate(work) for b in range(w["nblocks"])),
              key=lambda ib: per_block[ib[0]][:, ib[1]].sum())
    wd = work[dom[0]]
    n_el, _, fl_dom, fx_dom, by_dom = hp_block_work(wd["op"], dom[1])
    t_dom = float(per_block[dom[0]][:, dom[1]].mean()) * 1e-3
    share = float(per_block[dom[0]][:, dom[1]].sum() / per.sum())
    name = "sf_kernel<%s,P%d,%s>" % (SHAPES[wd["block_shapes"][dom[1]]], wd["P"], args.dtype)
    traffic = MEASURED_TRAFFIC.get(name)
    if args.dtype == "f64":
        # the collocated algorithm's flop count (hp_op_block_work `flops`) over
        # the kernel's event time, against the FP64 FMA rate measured on this
        # GPU by the library's own FMA-loop kernel; the operations the kernel
        # actually issues (fewer: even-odd eta1 pass, compact index sets) and the
        # nominal rate are reported beside
        a_tf = fl_dom / t_dom / 1e12
        issued_tf = fx_dom / t_dom / 1e12
        peak = fp64_peak if fp64_peak else FP64_PEAK_TFLOPS
        roof = {"bound": "alu", "kernel": name, "elements": int(n_el), "launch_ms": round(t_dom * 1e3, 4),
                "share_of_timed": round(share, 4), "achieved": round(a_tf, 4), "peak": round(peak, 4),
                "unit": "TFLOP/s", "frac": round(a_tf / peak, 4),
                "flops_counted": "collocated sum-factorisation algorithm (FMA = 2) per launch: %d" % int(fl_dom),
                "issued_tflops": round(issued_tf, 4), "issued_frac": round(issued_tf / peak, 4),
                "issued_flops_per_launch": int(fx_dom),
                "frac_of_nominal": round(a_tf / FP64_PEAK_TFLOPS, 4),
                "traffic": traffic, "algorithmic_bytes": int(by_dom),
                "peak_source": ("measured: hp_peak_fp64 FMA-loop kernel on this GPU, right after the timed region "
                                "(%.4f ms); nominal 1.25 TFLOP/s" % fp64_peak_ms) if fp64_peak else
                               "FP64 nominal 1.25 TFLOP/s (recipe unit table)",
                "step_achieved_tflops": round(achieved_tf, 4),
                "step_hbm_gbs": round(achieved_gbs, 1), "step_hbm_frac_of_measured": round(achieved_gbs / hbm_peak, 4)}
    else:
        a_gbs = by_dom / t_dom / 1e9
        roof = {"bound": "hbm", "kernel": name, "elements": int(n_el), "launch_ms": round(t_dom * 1e3, 4),
                "share_of_timed": round(share, 4), "achieved": round(a_gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(a_gbs / hbm_peak, 4), "traffic": traffic, "algorithmic_bytes": int(by_dom),
                "peak_source": hbm_src + " copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if hbm_src == "measured" else hbm_src,
                "step_achieved_gbs": round(achieved_gbs, 1)}
    table = None
    if rank == 0 and not args.no_table:
        table = shape_order_table(args.dtype, local)
    batched = None
    strategies = None
    forms = None
    roof_bf16 = None
    cost = None
    if rank == 0 and not args.no_extra:
        batched = padaptive(local)
        strategies = strategy_table(local)
        if args.dtype == "f64":
            forms = precision_forms(work, local)
            roof_bf16 = reduced_precision_roofline(work, local, hbm_peak, hbm_src)
        cost = costmodel_summary(local)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline()
    # time to solution of the assembled problem (64^3 cells, ~1M elements, P = 4):
    # FP64 PCG against the mixed-precision forms, on one GPU only
    solve = None
    if rank == 0 and world == 1 and not args.no_extra and not args.no_solve:
        solve = run_solve(local, 64, scheduled=True)
    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 4), "unit": "GDOF/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": args.dtype,
                "data": "synthetic",
                "config": {"workload": "helmholtz_mixed_%dcube_P%s_curved" % (CELLS, "-".join(map(str, ORDERS))),
                           "cells": "%dx%dx%d" % (CELLS, CELLS, CELLS), "elements": int(work[0]["mesh"]["n_elem"]), "orders": ",".join(map(str, ORDERS)), "Q": "P+2",
                           "lambda": 1.0, "strategy": "sumfac_collocated",
                           "l2": "flushed (256 MiB write) before every apply, outside the timed events"},
                "roofline": roof, "roofline_bf16": roof_bf16, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": clk.summary(), "per_order": per_order, "per_shape_order": table,
                "p_adaptive": batched, "strategies_gdofs_f64": strategies, "precision_forms": forms, "costmodel": cost,
                "time_to_solution": solve}
        print(json.dumps(line), flush=True)
    for w in work:
        from paper_2604_04644_gb300 import hp
        hp.hp_op_destroy(w["op"])
        hp.hp_mesh_destroy(w["h"])
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
