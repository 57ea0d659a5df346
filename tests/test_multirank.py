"""The N > 1 path of bench.py on CPU: two gloo ranks run bench.py's own timed
region (replicas: every rank solves its own copy of the 96-box batch, no
collective on the data path) with the solve replaced by a stub whose time
differs per rank.  The slowest rank's time defines the whole-job rate, and
rank 0 prints the contract's JSON line."""

import argparse
import json
import os
import socket
import time

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class _WallClock:
    def start(self):
        self.t0 = time.perf_counter()

    def stop(self):
        self.t1 = time.perf_counter()

    def ms(self):
        return (self.t1 - self.t0) * 1e3


def _rank(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    boxes = [b for b, _, _ in bench.batch_specs()]  # each rank's replica of the workload
    calls = []

    def step():  # stands in for sbp_solve_batched over the rank's boxes
        calls.append(1)
        time.sleep(0.002 * (rank + 1))

    ms = bench.replica_timing(step, dist.barrier, steps=5, warmup=3, clock=_WallClock())
    value = bench.job_rate(len(boxes), 5, world, ms)
    line = None
    if rank == 0:
        args = argparse.Namespace(steps=5, warmup=3)
        config = {"workload": "batch96", "boxes": len(boxes), "parallelism": f"replicas x{world}"}
        line = json.dumps(bench.result_line(args, world, value, ms / 5, "f32", config))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, len(calls), value, len(boxes), line))


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, ms0, calls0, v0, n0, line), (_, ms1, calls1, v1, n1, _) = out
    assert ms0 == ms1                # both ranks report the MAX over ranks
    assert ms0 >= 5 * 4.0            # rank 1's five steps of 4 ms bound it
    assert calls0 == calls1 == 8     # 3 warm-up + exactly 5 timed steps
    assert n0 == n1 == 96
    assert v0 == pytest.approx(2 * 96 * 5 / (ms0 / 1e3))
    rec = json.loads(line)
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config"):
        assert key in rec
    assert rec["n_gpus"] == 2 and rec["scaling"] == "weak" and rec["steps"] == 5
    assert rec["value"] == pytest.approx(v0)
    assert rec["config"]["parallelism"] == "replicas x2"


def test_single_rank_is_unchanged():
    import bench

    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.job_rate(96, 4, 1, 2.0) == pytest.approx(96 * 4 / 0.002)
    clock = _WallClock()
    calls = []
    ms = bench.replica_timing(lambda: calls.append(1), lambda: None, steps=4, warmup=3, clock=clock)
    assert len(calls) == 7 and ms == clock.ms()


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    # under torchrun the reference arm's other ranks exit without work
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    t0 = time.perf_counter()
    assert bench.main(["--impl", "reference", "--gpus", "2", "--steps", "3", "--warmup", "3"]) is None
    assert time.perf_counter() - t0 < 5.0
