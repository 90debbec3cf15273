"""The multi-rank path of bench.py on CPU with 2 gloo ranks: every rank gets its
own seeded batch (weak scaling, nothing exchanged in the data path), the job
time is the slowest rank's, and the job value counts all ranks' work."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    import bench
    w = bench.workload("ellipses2x32", rank)
    ms = bench.reduce_max(10.0 + 5.0 * rank, world, "cpu")
    val = bench.job_value(w.batch * w.voxels * w.T, world, ms)
    digest = float(np.asarray(w.I0, np.float64).sum() + 3.0 * np.asarray(w.J, np.float64).sum())
    gathered = [None] * world
    dist.all_gather_object(gathered, (rank, ms, val, digest))
    if rank == 0:
        out.put(gathered)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_the_batch_and_take_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res = sorted(res)
    assert [r[0] for r in res] == [0, 1]
    assert all(r[1] == 15.0 for r in res)  # max over ranks
    voxel_steps = 2 * 32 * 32 * 3
    assert all(abs(r[2] - 2 * voxel_steps / 15.0e-3) < 1e-6 * r[2] for r in res)
    assert res[0][3] != res[1][3]  # each rank registers its own instances
