"""The bench's multi-rank path (one process per GPU, weak scaling, max over
ranks) exercised with two gloo ranks on the CPU.  Systems are independent
units, so ranks exchange nothing but the barrier and the timing reduction."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 50.0 * rank           # rank 1 is the slow one
        got = bench.max_over_ranks(ms, world, torch.device("cpu"))
        dist.barrier()
        # the workload once per rank: the job's work is world times a rank's
        rate = bench.whole_job_rate(bench.flops_equiv(2000) * 14 * world, got)
        q.put((rank, got, rate))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_weak_rate_with_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [r[1] for r in res] == [150.0, 150.0]     # both ranks see the slowest time
    expect = bench_rate = (2.0 / 3.0 * 2000 ** 3 + 2.0 * 2000 ** 2) * 14 * 2 / 0.150 / 1e12
    assert res[0][2] == pytest.approx(expect) and res[1][2] == pytest.approx(bench_rate)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.whole_job_rate(1e12, 1000.0) == pytest.approx(1.0)


def _lpt_rank(rank, world, port, costs, q):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = bench.lpt_partition(costs, world)[rank]   # computed locally, no exchange
        got = [None] * world
        dist.all_gather_object(got, mine)                # the test's check only
        q.put((rank, mine, got))
    finally:
        dist.destroy_process_group()


def test_lpt_partition_two_gloo_ranks_solve_every_system_once():
    """The batched workload's systems (n uniform in [32, 512]) sharded by LPT
    on n^3 over two ranks: each rank derives its share alone, the shares are
    disjoint and cover every system, and the loads differ by at most the
    largest single system."""
    from synth import batched_systems
    systems = batched_systems(512, seed=0)
    costs = [float(n) ** 3 for (n, _, _) in systems]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_lpt_rank, args=(r, 2, port, costs, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    shares = [r[1] for r in res]
    assert res[0][2] == res[1][2] == shares            # both ranks agree on the partition
    flat = sorted(i for sh in shares for i in sh)
    assert flat == list(range(len(systems)))           # every system exactly once
    loads = [sum(costs[i] for i in sh) for sh in shares]
    assert abs(loads[0] - loads[1]) <= max(costs)


def test_lpt_partition_properties():
    import bench
    assert bench.lpt_partition([5.0, 1.0, 4.0, 3.0, 3.0], 2) == [[0, 4], [1, 2, 3]]
    assert bench.lpt_partition([1.0, 2.0], 1) == [[0, 1]]
    assert bench.lpt_partition([], 3) == [[], [], []]
    parts = bench.lpt_partition([7.0] * 9, 4)
    assert sorted(len(p) for p in parts) == [2, 2, 2, 3]
