"""The multi-process path on CPU (gloo, world size 2): the method shards into
independent units (geometries of a batch, or frequencies) with no exchange, so
each rank works on its share and the job's rate is the units of all ranks over
the slowest rank's time.  Checked: the shards cover every unit exactly once and
balance uneven sizes (largest first to the least-loaded rank); the aggregation
gives every rank the same whole-job rate."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    units = list(range(11))
    mine = bench.shard(units, rank, world)
    # rank r "processed" its units in 1 + r seconds
    rate, tmax = bench.aggregate(1.0 + rank, float(len(mine)), dist)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    out.put((rank, rate, tmax, gathered))
    dist.barrier()
    dist.destroy_process_group()


def test_shards_and_aggregate_over_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, tmax, gathered in res:
        assert tmax == 2.0                              # the slowest rank's time
        assert rate == 11 / 2.0                         # all units over it
        flat = sorted(u for part in gathered for u in part)
        assert flat == list(range(11))                  # every unit once
        assert abs(len(gathered[0]) - len(gathered[1])) <= 1


def test_shard_balances_uneven_units():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    sizes = [60, 5, 50, 8, 40, 12, 30, 20]              # uneven geometries, largest first
    parts = [bench.shard(sizes, r, 2, sizes=sizes) for r in range(2)]
    assert sorted(parts[0] + parts[1]) == sorted(sizes)
    assert abs(sum(parts[0]) - sum(parts[1])) <= max(sizes) // 6   # 115 vs 110 here
    # without sizes: every other unit
    assert bench.shard(sizes, 1, 2) == sizes[1::2]
