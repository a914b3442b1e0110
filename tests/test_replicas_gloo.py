"""Multi-process replica logic on CPU: gloo, world size 2, 127.0.0.1."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1208_2675_gb300 import replicas


def test_partition_is_complete_disjoint_and_balanced():
    costs = [replicas.chain_cost(n, 10 ** 7) for n in range(20, 300, 7)]
    for world in (1, 2, 3, 8):
        parts = replicas.partition_by_cost(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) <= 4 / 3 * max(sum(costs) / world, max(costs)) + 1e-6


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, costs, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = replicas.partition_by_cost(costs, world)[rank]
    load = sum(costs[i] for i in mine)
    got = [None] * world
    dist.all_gather_object(got, mine)
    worst = replicas.max_over_ranks(load, dist)
    sid = [None] * world
    dist.all_gather_object(sid, replicas.stream_id_for(rank, 100))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got, worst, sid))


def test_two_ranks_agree_on_partition_time_and_streams():
    costs = [replicas.chain_cost(n, i) for n, i in [(30, 10 ** 6), (300, 10 ** 8), (100, 10 ** 7),
                                                     (50, 10 ** 7), (600, 10 ** 6), (80, 10 ** 8)]]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, costs, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    parts = res[0][1]
    assert res[1][1] == parts
    assert sorted(parts[0] + parts[1]) == list(range(len(costs)))
    loads = [sum(costs[i] for i in p) for p in parts]
    assert res[0][2] == res[1][2] == pytest.approx(max(loads))
    assert res[0][3] == [100, 101]
