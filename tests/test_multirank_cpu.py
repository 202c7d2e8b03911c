"""N > 1 host logic on CPU ranks (gloo, world size 2): the batched workload is sharded
over ranks with no data-path collective (weak scaling), and the step time is the maximum
over ranks.  The single-system solve does not shard (replicas only)."""
import importlib.util
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _bench()
    mine = b.shard_systems(512, rank, world)
    t = b.max_over_ranks(1.0 + rank, dist)
    q.put((rank, mine, t))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_partition_single_rank():
    b = _bench()
    assert b.shard_systems(7, 0, 1) == list(range(7))
    parts = [b.shard_systems(10, r, 3) for r in range(3)]
    assert sorted(sum(parts, [])) == list(range(10))
    assert max(map(len, parts)) - min(map(len, parts)) <= 1
    assert b.max_over_ranks(2.5) == 2.5


def test_two_cpu_ranks_shard_and_max():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out.sort()
    shares = [o[1] for o in out]
    assert sorted(shares[0] + shares[1]) == list(range(512))   # every system exactly once
    assert not set(shares[0]) & set(shares[1])
    assert all(o[2] == 2.0 for o in out)                        # slowest rank's time on every rank
