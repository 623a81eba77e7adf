"""The bench's multi-rank host path on CPU: two gloo ranks (one process each,
as torchrun would start them), the barrier, the max-over-ranks step time and
the whole-job throughput of the split workload (all ranks' DOFs over the
slowest rank's time); the reference arm does its work on rank 0 only."""
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist

    class A:
        impl = "gb300"
    w, r, local = bench.dist_init(A, backend="gloo")
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    ms_local = [3.0, 5.0, 4.0, 2.0][rank]
    ms_max, value = bench.split_scaling_value(w, [2.0e6, 1.0e6, 3.0e6, 4.0e6][rank], ms_local)
    # the reference arm: rank 0 alone prints; the others return at once
    import io
    import contextlib
    buf = io.StringIO()

    class R:
        warmup, steps, gpus = 0, 1, world
    if rank != 0:
        with contextlib.redirect_stdout(buf):
            bench.run_reference(R, w, r)
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump({"ms_max": ms_max, "value": value, "ref_out": buf.getvalue()}, f)
    bench.barrier(w)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_split_scaling_host_path(tmp_path, world):
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(world)]
    slowest = max([3.0, 5.0, 4.0, 2.0][:world])
    for r in res:
        assert r["ms_max"] == slowest                       # every rank sees the slowest rank's time
        assert r["value"] == pytest.approx(sum([2.0e6, 1.0e6, 3.0e6, 4.0e6][:world]) / (slowest * 1e-3) / 1e9)
    assert all(r["ref_out"] == "" for r in res[1:])          # non-zero ranks: no reference work


def test_single_rank_value_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    ms, v = bench.split_scaling_value(1, 1.0e9, 10.0)
    assert ms == 10.0 and v == pytest.approx(100.0)


def _part_main(rank, world, port, out_dir):
    """The bench's per-rank workload: each rank builds its part of the bench
    mesh (hp_partition, ranges of the block order) without a GPU."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank))
    sys.path.insert(0, ROOT)
    import numpy as np
    from paper_2604_04644_gb300 import hp, inputs
    mesh = inputs.slab_mesh(4, 4, 4, 3, curved=True)
    part = hp.hp_partition(mesh, world, 0)
    mine = np.nonzero(part == rank)[0]
    np.save(os.path.join(out_dir, "part%d.npy" % rank), mine)


def test_bench_split_covers_the_mesh_once(tmp_path):
    world = 2
    mp.start_processes(_part_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    import numpy as np
    parts = [np.load(tmp_path / ("part%d.npy" % r)) for r in range(world)]
    allp = np.sort(np.concatenate(parts))
    assert np.array_equal(allp, np.arange(len(allp))) and all(len(p) > 0 for p in parts)
