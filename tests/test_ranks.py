"""Multi-GPU host logic on the CPU: two gloo ranks (no GPU), the way bench.py runs N > 1."""
import os
import socket

import pytest
import torch
import torch.distributed as td
import torch.multiprocessing as mp

from paper_2204_03139_gb300.ranks import max_over_ranks, rank_seed, shard_by_cost


def test_shard_by_cost_covers_every_item_once_and_balances():
    costs = [90, 10, 40, 40, 30, 30, 20, 5, 5, 1]
    for world in (1, 2, 3, 4):
        sh = shard_by_cost(costs, world)
        flat = sorted(i for s in sh for i in s)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in s) for s in sh]
        # longest-processing-time bound: no rank exceeds the mean by more than the largest item
        assert max(loads) <= sum(costs) / world + max(costs)
    assert shard_by_cost([], 3) == [[], [], []]


def test_rank_seeds_differ_and_rank0_keeps_the_base():
    assert rank_seed(7, 0) == 7
    assert len({rank_seed(7, r) for r in range(8)}) == 8


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        td.barrier()
        local = 1.5 + rank  # this rank's time
        m = max_over_ranks(local, td)
        # the whole-job value: units of all ranks / the slowest rank's time
        units = 100.0
        value = world * units / m
        sh = shard_by_cost([5, 4, 3, 3, 2, 1], world)[rank]
        q.put((rank, m, value, sh))
        td.barrier()
    finally:
        td.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_take_the_max_time_and_split_the_work():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, q), nprocs=world, join=True,
                       start_method="spawn")
    res = sorted(q.get(timeout=30) for _ in range(world))
    assert [r[1] for r in res] == [2.5, 2.5]            # max over ranks on every rank
    assert all(abs(r[2] - 2 * 100 / 2.5) < 1e-12 for r in res)
    items = sorted(i for r in res for i in r[3])
    assert items == list(range(6))                       # each trajectory on exactly one rank
