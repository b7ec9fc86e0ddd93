"""World-size-2 gloo test of the multi-GPU partition (CPU only): the shards
cover the pair list exactly once, their estimated costs balance, and the
max-over-ranks timing reduction used by the benchmark works over the
process group."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1701_06588_gb300 import shard, workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sh, pa, pb = W.make("c2_200k_l4_k8", n=5000)
    a, b, lo = shard.shard_pairs(sh["l"], sh["nprim"], pa, pb, rank, world)
    cost = float(shard.pair_costs(sh["l"], sh["nprim"], a, b).sum())
    t = torch.tensor([cost, float(len(a)), float(lo)], dtype=torch.float64)
    out = [torch.zeros(3, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(out, t)
    mx = torch.tensor([float(rank + 1)], dtype=torch.float64)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    if rank == 0:
        q.put(([o.tolist() for o in out], float(mx.item())))
    dist.barrier()
    dist.destroy_process_group()


def test_shards_cover_and_balance_over_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res, mx = q.get(timeout=300)
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    costs = [r[0] for r in res]
    counts_ = [int(r[1]) for r in res]
    starts = [int(r[2]) for r in res]
    assert sum(counts_) == 5000 and starts == [0, counts_[0]]
    assert max(costs) / min(costs) < 1.02
    assert mx == float(world)


def test_shard_bounds_edge_cases():
    assert list(shard.shard_bounds(np.array([]), 3)) == [0, 0, 0, 0]
    b = shard.shard_bounds(np.ones(10), 4)
    assert b[0] == 0 and b[-1] == 10 and np.all(np.diff(b) >= 0)
    b = shard.shard_bounds(np.array([100.0, 1, 1, 1]), 2)
    assert list(b) == [0, 1, 4]


def _bench_worker(rank, world, port, q):
    """The benchmark's own partition (bench.rank_workload) on one gloo rank."""
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    full, pa, pb = W.make(bench.WORKLOAD, n=4000)
    sh, a, b, lo, job_units = bench.rank_workload(full, pa, pb, rank, world)
    # the slice's shells are the original shells of pairs lo .. lo + len(a)
    ref = np.arange(lo, lo + len(a))
    same = (np.array_equal(sh["l"][a], full["l"][pa[ref]]) and np.array_equal(sh["l"][b], full["l"][pb[ref]]) and
            np.array_equal(sh["nprim"][a], full["nprim"][pa[ref]]) and
            np.allclose(sh["centers"][sh["center_of"][b]], full["centers"][full["center_of"][pb[ref]]]))
    cost = float(shard.pair_costs(sh["l"], sh["nprim"], a, b).sum())
    t = torch.tensor([cost, float(len(a)), float(lo), float(job_units), float(same)], dtype=torch.float64)
    out = [torch.zeros(5, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(out, t)
    if rank == 0:
        q.put([o.tolist() for o in out])
    dist.barrier()
    dist.destroy_process_group()


def test_bench_partition_over_gloo():
    """bench.py --gpus 2: each rank evaluates its cost-balanced slice of the one
    pair list; the slices tile the list, carry the right shells, and the job's
    units are the whole list's."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_bench_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = q.get(timeout=300)
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    costs = [r[0] for r in res]
    counts_ = [int(r[1]) for r in res]
    starts = [int(r[2]) for r in res]
    assert sum(counts_) == 4000 and starts == [0, counts_[0]]
    assert all(int(r[3]) == 4000 * len(bench.OPS) for r in res)
    assert all(r[4] == 1.0 for r in res)
    assert max(costs) / min(costs) < 1.05
