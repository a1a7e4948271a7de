"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): replicas take
disjoint shares of independent work, the job time is the slowest rank's and
the throughput counts every rank's work.  No GPU is involved."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    items = list(range(11))
    mine = bench.shard(items, rank, world)
    my_ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
    mx = bench.allreduce_max(my_ms, world)
    count = torch.tensor([len(mine)], dtype=torch.int64)
    dist.all_reduce(count)
    bench.barrier(world)
    q.put((rank, mine, mx, int(count.item()), bench.job_throughput(5, world, mx)))
    dist.destroy_process_group()


def test_two_rank_replicas_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    shards = [o[1] for o in out]
    assert sorted(shards[0] + shards[1]) == list(range(11)) and not set(shards[0]) & set(shards[1])
    assert all(o[2] == 150.0 for o in out)          # slowest rank's time
    assert all(o[3] == 11 for o in out)             # every item processed once
    assert all(abs(o[4] - 2 * 5 / 0.150) < 1e-9 for o in out)
