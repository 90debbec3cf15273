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


# ------------------------------------------------- one job split across ranks

def test_partition_assigns_every_instance_once_and_balances_voxel_steps():
    import itertools
    import sys
    sys.path.insert(0, ROOT)
    import phantoms
    from paper_2106_08817_gb300 import partition as pt
    # the 64 uneven pairs: each instance's voxel-steps
    work = [w.batch * w.voxels * w.T for w in phantoms.mixed_pairs()]
    for n in (1, 2, 3, 4, 8):
        shares = pt.partition(work, n)
        flat = sorted(i for s in shares for i in s)
        assert flat == list(range(len(work)))  # each instance exactly once
        assert shares == pt.partition(work, n)  # the same split on every rank
        loads = [pt.load_of(work, s) for s in shares]
        mean = sum(work) / n
        assert max(loads) <= mean + max(work)  # list scheduling
        assert max(loads) / mean < 1.15  # 64 pairs spread well over up to 8 ranks
    # Graham's bound for largest-first scheduling against the brute-force optimum
    r = np.random.default_rng(5)
    for _ in range(30):
        m = int(r.integers(4, 9))
        w = [float(x) for x in r.integers(1, 100, size=m)]
        for n in (2, 3):
            got = max(pt.load_of(w, s) for s in pt.partition(w, n))
            opt = min(max(sum(w[i] for i in range(m) if a[i] == k) for k in range(n))
                      for a in itertools.product(range(n), repeat=m))
            assert got <= (4.0 / 3.0 - 1.0 / (3 * n)) * opt + 1e-9
    with pytest.raises(ValueError):
        pt.partition([1.0], 0)


def _gather_worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    from paper_2106_08817_gb300 import partition as pt
    work = [float((7 * i) % 11 + 1) for i in range(13)]
    mine = pt.rank_share(work, world, rank)
    # a per-instance "cost" only the owning rank computes
    vals = [[float(i), float(i * i), float(rank)] for i in mine]
    allv = pt.gather_in_order(mine, vals, len(work))
    bad = None
    try:
        pt.gather_in_order(mine[:1] if rank == 0 else mine, vals[:1] if rank == 0 else vals,
                           len(work))
    except ValueError as e:
        bad = str(e)
    if rank == 0:
        out.put((allv, mine, bad))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_split_one_job_and_gather_costs_in_instance_order():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gather_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    allv, mine0, bad = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [v[0] for v in allv] == [float(i) for i in range(13)]  # instance order
    assert all(v[1] == v[0] ** 2 for v in allv)
    owners = [int(v[2]) for v in allv]
    assert set(owners) == {0, 1} and [i for i in range(13) if owners[i] == 0] == mine0
    assert bad is not None and "not gathered" in bad  # a dropped instance is an error
