"""The N > 1 path of bench.py on CPU: two gloo ranks (replicas, no collective
on the data path; the slowest rank's time defines the whole-job rate)."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    local_ms = [12.5, 20.0][rank]
    ms = bench.max_over_ranks(local_ms)
    rate = bench.job_rate(96, 10, world, ms)
    # each rank builds the same replica workload
    from paper_2510_10070_gb300 import workloads as W

    case = W.batch_96()
    sig = (len(case.boxes), sum(b.cells for b in case.boxes), round(float(sum(case.times)), 12))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, rate, sig))


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, ms, rate, sig in out:
        assert ms == 20.0
        assert rate == pytest.approx(2 * 96 * 10 / 0.020)
    assert out[0][3] == out[1][3]


def test_single_rank_is_unchanged():
    import bench

    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.job_rate(96, 4, 1, 2.0) == pytest.approx(96 * 4 / 0.002)
