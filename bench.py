#!/usr/bin/env python
"""Throughput of the shearing-box VGF-HybridBC Poisson solver on GB300.

    python bench.py [--gpus N --steps K --warmup W] [--workload batch96|box256|box256_f64]
                    [--impl ours|reference] [--no-cpu-baseline] [--no-side]

A step is one pass of the whole method over one batch of synthetic input:
by default the 96-box FP32 batch (32× 64³, 32× 128²×64, 16× 192²×96,
16× 256²×128, each box with its own shear time and q), solved through
sbp_solve_batched.  Inputs (931 MB) are larger than L2, so no flush is
needed between steps.  Under torchrun every rank solves its own copy of the
batch (weak scaling, no collective on the data path); rank 0 prints one JSON
line with the whole-job rate.

Beside the rate the line states, per result, the error against FP64
references (the FP64 GPU solve of every box, and the FP64 oracle where it
is quick): relative L2, relative L2 without the plane means, and the
max-norm error relative to ‖Φ‖∞.  `single_box` holds single-box rows of the
other configurations (256×256×128 at t = 0, 1.3, 5; 512×512×256; the
1024×1024×512 clumpy disc), FP32 and FP64, each with its B_alg roofline
fraction.  `cpu_baseline` times the FP64 oracle on the host cores: one
process per core, each solving one box of the batch's size classes.

--impl reference times that oracle alone, on the same workload, metric and
unit: every step runs one process per host core on boxes of one size class
of the batch, the classes taken in proportion to their counts.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Poisson solves/s and Gcells/s on 1 GB300 (FP32 & batched vs FP64) at stated rel-L2; % HBM peak"
HBM_PEAK_FALLBACK = 6800.0
L2_FLUSH_BYTES = 256 << 20  # larger than the 126 MB L2


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": HBM_PEAK_FALLBACK}, "fallback"


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def batch_specs():
    """The 96 boxes of the batch as (box, seed, t) with σ = 0.7."""
    from paper_2510_10070_gb300 import workloads as W

    case = W.batch_96()
    return [(b, s, float(t)) for b, s, t in zip(case.boxes, case.seeds, case.times)]


def build_workload(name):
    import numpy as np

    from paper_2510_10070_gb300 import workloads as W

    if name == "batch96":
        specs = batch_specs()
        rhos = [W.lognormal_disc(b, seed=s, sigma=0.7, dtype=np.float32) for b, s, _ in specs]
        return [b for b, _, _ in specs], rhos, [t for _, _, t in specs], 1
    if name in ("box256", "box256_f64"):
        box = W.BOX_256
        rho = W.lognormal_disc(box, seed=2, sigma=0.5)
        dt = 0 if name == "box256_f64" else 1
        return [box], [rho if dt == 0 else rho.astype(np.float32)], [1.3], dt
    raise SystemExit(f"unknown workload {name}")


def shape_of(box):
    return (box.nx, box.ny, box.nz)


def alg_bytes(box, rb):
    """B_alg of one solve: read ρ, write φ, and the half spectrum written by
    the forward passes, read and written by the z pass and read by the
    inverse passes (three-sweep model)."""
    N = box.nx * box.ny * box.nz
    H = (box.nx // 2 + 1) * box.ny * box.nz
    return 2 * N * rb + 8 * H * rb


def middle_pass_bytes(box, rb):
    """Algorithmic bytes of one launch of the middle pass (or of the five-pass
    z pass): read and write the half spectrum."""
    H = (box.nx // 2 + 1) * box.ny * box.nz
    return 2 * 2 * H * rb


def oracle_cost(box):
    """Multiply-add count of the oracle's direct sums (only for a class whose
    boxes were not timed at all)."""
    nx, ny, nz = box.nx, box.ny, box.nz
    return (2 * nz * ny * nx * (nx + ny) + nx * ny * (2 * nz) * (2 * nz - 1) + nx * ny * nz * nz)


def recorded_traffic(kernel_name):
    """DRAM bytes (read + write) per launch of the dominant kernel from the
    committed ncu record, or None when the record is for another kernel or
    the kernel sources changed since it was taken."""
    import hashlib

    try:
        with open(os.path.join(ROOT, "profiles", "dominant_kernel_traffic.json")) as f:
            rec = json.load(f)
        h = hashlib.sha256()
        for name in rec.get("sources", []):
            with open(os.path.join(ROOT, "paper_2510_10070_gb300", "csrc", name), "rb") as f:
                h.update(f.read())
    except (OSError, ValueError):
        return None, None
    if rec.get("source_sha256") != h.hexdigest() or rec.get("kernel") != kernel_name:
        return None, None
    return rec["dram_bytes_read"] + rec["dram_bytes_write"], rec


# ---------------------------------------------------------------------------
# accuracy
# ---------------------------------------------------------------------------

def errors(got, want):
    """(rel-L2, rel-L2 without the plane means, max-norm relative to ‖Φ‖∞) of
    got against want, on the device (torch tensors [nz, ny, nx])."""
    import torch

    g = got.double()
    w = want.double()
    d = g - w
    e1 = (torch.linalg.vector_norm(d) / torch.linalg.vector_norm(w)).item()
    dm = d - d.mean(dim=(-2, -1), keepdim=True)
    wm = w - w.mean(dim=(-2, -1), keepdim=True)
    e2 = (torch.linalg.vector_norm(dm) / torch.linalg.vector_norm(wm)).item()
    e3 = (d.abs().max() / w.abs().max()).item()
    return {"rel_l2": e1, "rel_l2_no_plane_means": e2, "max_rel": e3}


def worst(errs):
    return {k: max(e[k] for e in errs) for k in errs[0]} if errs else None


# ---------------------------------------------------------------------------
# multi-rank timing (replicas: every rank solves its own copy of the batch)
# ---------------------------------------------------------------------------

def max_over_ranks(ms, device=None):
    """The slowest rank's time; each rank passes its own (1 rank: unchanged)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, steps, world, ms_max):
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return world * units_per_rank * steps / (ms_max / 1e3)


class CudaClock:
    """Device time of the work enqueued on `stream` between start() and stop()."""

    def __init__(self, stream):
        import torch

        self.stream = stream
        self.a = torch.cuda.Event(enable_timing=True)
        self.b = torch.cuda.Event(enable_timing=True)

    def start(self):
        self.a.record(self.stream)

    def stop(self):
        self.b.record(self.stream)

    def ms(self):
        return self.a.elapsed_time(self.b)


def replica_timing(step, sync, steps, warmup, clock, device=None, during=None):
    """The timed region every rank runs: `warmup` untimed steps, then exactly
    `steps` steps on `clock`, with `sync` (barrier over the ranks and the
    device) on both sides; returns the slowest rank's milliseconds.  `during`
    is a context manager held around the timed steps (the clock sampler)."""
    import contextlib

    for _ in range(warmup):
        step()
    sync()
    with (during if during is not None else contextlib.nullcontext()):
        sync()
        clock.start()
        for _ in range(steps):
            step()
        clock.stop()
        sync()
    return max_over_ranks(clock.ms(), device=device)


def result_line(args, world, value, ms_per_step, dtype, config, **extra):
    """The JSON line rank 0 prints (keys of the driver's contract first)."""
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": config}
    line.update(extra)
    return line


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle: one process per host core (spawned), each solving whole boxes
# ---------------------------------------------------------------------------

def _oracle_init():
    # one BLAS thread per process: the processes, not BLAS, use the cores
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"


def _oracle_job(spec):
    """Solve one box with the FP64 oracle; returns (wall s, CPU s, Φ or None)."""
    import numpy as np

    import oracle as O
    from paper_2510_10070_gb300 import workloads as W

    b = W.Box(*spec["box"])
    if spec["kind"] == "array":  # the density itself, built by the caller
        rho = np.asarray(spec["rho"], dtype=np.float64)
    elif spec["kind"] == "noisy":
        rho = W.noisy_gaussian(b, seed=spec["seed"])
    else:
        rho = W.lognormal_disc(b, seed=spec["seed"], sigma=spec["sigma"])
        if spec.get("down"):
            rho = W.downsample(rho, *spec["down"])
            b = W.Box(rho.shape[2], rho.shape[1], rho.shape[0], b.Lx, b.Ly, b.Lz, q=b.q, Omega=b.Omega, G=b.G)
    if spec.get("f32"):
        rho = rho.astype(np.float32).astype(np.float64)
    p = O.SolveParams(b.Lx, b.Ly, b.Lz, q=b.q, Omega=b.Omega, G=b.G)
    c0, t0 = time.process_time(), time.perf_counter()
    phi = O.solve(rho, p, spec["t"])
    wall, cpu = time.perf_counter() - t0, time.process_time() - c0
    return wall, cpu, (phi if spec.get("keep") else None)


def box_tuple(b):
    return (b.nx, b.ny, b.nz, b.Lx, b.Ly, b.Lz, b.q, b.Omega, b.G)


class OraclePool:
    """`cores` spawned worker processes (spawn: safe beside a CUDA context)."""

    def __init__(self, cores):
        import multiprocessing as mp

        self.cores = cores
        self.pool = mp.get_context("spawn").Pool(cores, initializer=_oracle_init)

    def run(self, specs):
        """Run the specs concurrently, one per process; returns (the longest
        solve, [(wall, cpu, phi)]).  Each process builds its input before its
        clock starts, so the longest solve is the time in which every core
        solved one box."""
        out = self.pool.map(_oracle_job, specs, chunksize=1)
        return max(o[0] for o in out), out

    def close(self):
        self.pool.close()
        self.pool.join()


def class_specs(specs, shape, count):
    """`count` boxes of the batch's class `shape` (cycling through the class)."""
    cls = [s for s in specs if shape_of(s[0]) == shape]
    out = []
    for i in range(count):
        b, seed, t = cls[i % len(cls)]
        out.append({"kind": "lognormal", "box": box_tuple(b), "seed": seed, "sigma": 0.7, "t": t})
    return out


def batch_classes(boxes):
    counts = {}
    for b in boxes:
        counts[shape_of(b)] = counts.get(shape_of(b), 0) + 1
    return counts


def batch_rate_from_classes(boxes, class_rate):
    """Solves/s of the whole batch from per-class rates (boxes/s with every
    core busy): n_boxes / Σ_c n_c / rate_c."""
    counts = batch_classes(boxes)
    secs = sum(n / class_rate[c] for c, n in counts.items())
    return len(boxes) / secs


def cpu_batch_baseline(pool, boxes, extra_256=None):
    """One round per size class of the batch: `cores` processes each solve a
    box of that class at once.  Returns (solves/s of the batch, details).
    extra_256 replaces one 256×256×128 job (same cost) and is returned too."""
    specs = batch_specs()
    cores = pool.cores
    rates, details, kept = {}, {}, None
    for shape in sorted(batch_classes(boxes), key=lambda s: s[0] * s[1] * s[2]):
        jobs = class_specs(specs, shape, cores)
        if extra_256 is not None and shape == (256, 256, 128):
            jobs[0] = extra_256
        wall, out = pool.run(jobs)
        rates[shape] = cores / wall
        cpu = sum(o[1] for o in out)
        details["x".join(map(str, shape))] = {"boxes": cores, "longest_solve_s": wall, "solves_per_s": cores / wall,
                                              "mean_box_s": statistics.mean(o[0] for o in out),
                                              "cores_busy": cpu / wall}
        if extra_256 is not None and shape == (256, 256, 128):
            kept = out[0]
    return batch_rate_from_classes(boxes, rates), details, kept


# ---------------------------------------------------------------------------
# GPU helpers
# ---------------------------------------------------------------------------

def event_time_ms(fn, stream, reps, warm=3, flush=None):
    """Mean ms per call of fn, with CUDA events on `stream` after `warm`
    untimed calls.  With a flush buffer, L2 is overwritten before every call
    and each call is timed on its own."""
    import torch

    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    if flush is None:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps
    tot = 0.0
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        tot += a.elapsed_time(b)
    return tot / reps


def solve_row(box, ms, rb, peak):
    cells = box.nx * box.ny * box.nz
    gbs = alg_bytes(box, rb) / (ms / 1e3) / 1e9
    return {"ms_per_solve": ms, "solves_per_s": 1e3 / ms, "gcells_per_s": cells / (ms / 1e3) / 1e9,
            "alg_bytes": alg_bytes(box, rb), "alg_gbs": gbs, "hbm_frac": gbs / peak}


# ---------------------------------------------------------------------------
# reference arm: the oracle alone
# ---------------------------------------------------------------------------

def reference_arm(args):
    boxes, _, _, dt = build_workload(args.workload)
    cores = host_cores()
    pool = OraclePool(cores)
    specs = batch_specs()
    counts = batch_classes(boxes)
    shapes = sorted(counts, key=lambda s: s[0] * s[1] * s[2])
    # classes in proportion to their counts: 32:32:16:16 → [64³, 128², 64³, 128², 192², 256²]
    unit = min(counts.values())
    cycle = []
    for k in range(max(counts.values()) // unit):
        for s in shapes:
            if counts[s] // unit > k:
                cycle.append(s)
    for _ in range(args.warmup):
        pool.run(class_specs(specs, shapes[0], cores))
    times, per = [], {}
    for i in range(args.steps):
        shape = cycle[i % len(cycle)]
        wall, _ = pool.run(class_specs(specs, shape, cores))
        times.append(wall)
        per.setdefault(shape, []).append(cores / wall)
    pool.close()
    rate = {s: statistics.mean(v) for s, v in per.items()}
    missing = [s for s in shapes if s not in rate]
    if missing:  # fewer steps than classes: scale the slowest measured class by the oracle's cost
        ref = max(rate, key=lambda s: oracle_cost(next(b for b in boxes if shape_of(b) == s)))
        rb = next(b for b in boxes if shape_of(b) == ref)
        for s in missing:
            bs = next(b for b in boxes if shape_of(b) == s)
            rate[s] = rate[ref] * oracle_cost(rb) / oracle_cost(bs)
    value = batch_rate_from_classes(boxes, rate)
    cells = sum(b.cells for b in boxes)
    sample = (f"each step: {cores} processes (one per host core, spawned, one BLAS thread each) solved "
              f"{cores} boxes of one size class of the batch with the FP64 oracle; classes in proportion "
              f"to their counts ({' '.join('x'.join(map(str, s)) for s in cycle)}); batch rate = "
              f"{len(boxes)} / sum over classes of count / measured class rate"
              + (f"; classes {missing} not reached in {args.steps} steps, scaled by the oracle's operation count"
                 if missing else ""))
    config = {"workload": args.workload, "boxes": len(boxes), "cells_per_step": cells,
              "gcells_per_s": value * cells / len(boxes) / 1e9,
              "alg_bytes_per_step": sum(alg_bytes(b, 8) for b in boxes), "parallelism": f"{cores} host processes"}
    line = result_line(args, args.gpus, value, statistics.mean(times) * 1e3, "f64", config, impl="reference",
                       cpu_baseline={"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                                     "sample": sample},
                       e2e={"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                       class_rates={"x".join(map(str, s)): r for s, r in rate.items()})
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# main
# ---------------------------------------------------------------------------

def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="batch96", choices=["batch96", "box256", "box256_f64"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-side", action="store_true", help="skip the single-box rows of the other configs")
    args = ap.parse_args(argv)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.warmup < 3:
        raise SystemExit("--warmup must be at least 3")

    if args.impl == "reference":
        if rank == 0:
            reference_arm(args)
        return

    import numpy as np
    import torch

    from paper_2510_10070_gb300 import sbp
    from paper_2510_10070_gb300 import workloads as W

    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    boxes, rhos_np, times, dt = build_workload(args.workload)
    tdt = torch.float64 if dt == 0 else torch.float32
    rb = 8 if dt == 0 else 4
    plans = [sbp.Plan(b.nx, b.ny, b.nz, b.Lx, b.Ly, b.Lz, q=b.q, Omega=b.Omega, G=b.G, dtype=dt) for b in boxes]
    rhos = [torch.from_numpy(np.ascontiguousarray(r)).to(device=dev, dtype=tdt) for r in rhos_np]
    phis = [torch.empty_like(r) for r in rhos]
    stream = torch.cuda.current_stream()
    peaks, peak_src = measured_peaks()
    peak = peaks["hbm_gbs"]

    def step():
        sbp.solve_batched(plans, rhos, phis, times, stream=stream)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    clk = ClockSampler(local)
    ms = replica_timing(step, barrier, args.steps, args.warmup, CudaClock(stream), device=dev, during=clk)
    ms_per_step = ms / args.steps
    nbox = len(boxes)
    value = job_rate(nbox, args.steps, world, ms)
    cells = sum(b.cells for b in boxes)
    balg = sum(alg_bytes(b, rb) for b in boxes)
    launches_per_step, grouped_boxes = sbp.batch_info(plans, rhos, phis)

    # End to end: every step copies its inputs from pinned host memory, solves
    # through sbp_solve_batched and copies its results back.  All boxes sit in
    # one pinned host buffer and one device buffer per direction (each box at
    # a 256-byte aligned offset), so a step's copies are one transfer each way.
    # Three device buffer sets let step i+1's host-to-device copy and step
    # i-1's device-to-host copy run on their own streams while step i solves,
    # without the solve waiting for a copy-out two steps back; the events keep
    # every buffer's uses in order.  The host link, not the solve, bounds this
    # rate: copy engines and SM copy kernels both move 211 GB/s host to device
    # and 193 GB/s back on this part, about 340 GB/s with both directions busy.
    offs, total = [], 0
    for r in rhos:
        offs.append(total)
        total += (r.numel() + 63) // 64 * 64

    def views(flat):
        return [flat[o:o + r.numel()].view(r.shape) for o, r in zip(offs, rhos)]

    flat_in = torch.empty(total, dtype=tdt).pin_memory()
    flat_out = torch.empty(total, dtype=tdt).pin_memory()
    for hv, r in zip(views(flat_in), rhos):
        hv.copy_(r.cpu())
    h2d = sum(r.numel() * r.element_size() for r in rhos)
    NSET = 3
    dev_flat = [(torch.empty(total, dtype=tdt, device=dev), torch.empty(total, dtype=tdt, device=dev))
                for _ in range(NSET)]
    sets = [(views(fi), views(fo)) for fi, fo in dev_flat]
    s_in = torch.cuda.Stream(device=dev)
    s_out = torch.cuda.Stream(device=dev)
    ev_in = [torch.cuda.Event() for _ in range(NSET)]
    ev_done = [torch.cuda.Event() for _ in range(NSET)]
    ev_out = [torch.cuda.Event() for _ in range(NSET)]
    used = [False] * NSET

    def e2e_step(i):
        k = i % NSET
        r_set, f_set = sets[k]
        with torch.cuda.stream(s_in):
            if used[k]:
                s_in.wait_event(ev_done[k])  # the solve NSET steps back has read these inputs
            dev_flat[k][0].copy_(flat_in, non_blocking=True)
            ev_in[k].record(s_in)
        stream.wait_event(ev_in[k])
        if used[k]:
            stream.wait_event(ev_out[k])  # the copy-out NSET steps back has read these outputs
        sbp.solve_batched(plans, r_set, f_set, times, stream=stream)
        ev_done[k].record(stream)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_done[k])
            flat_out.copy_(dev_flat[k][1], non_blocking=True)
            ev_out[k].record(s_out)
        used[k] = True

    def e2e_drain():
        stream.wait_stream(s_in)
        stream.wait_stream(s_out)

    for i in range(2 * NSET):
        e2e_step(i)
    e2e_drain()
    barrier()
    e2e_steps = max(8, args.steps)
    s2, e2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s2.record(stream)
    s_in.wait_stream(stream)
    for i in range(e2e_steps):
        e2e_step(i)
    e2e_drain()
    e2.record(stream)
    barrier()
    e2e_value = job_rate(nbox, e2e_steps, world, max_over_ranks(s2.elapsed_time(e2), device=dev))
    del dev_flat, sets, flat_in, flat_out

    # ---- accuracy of the timed batch: every box against its FP64 GPU solve
    # (which the tests pin to the FP64 oracle at ≤ 1e-12), and the first box
    # against the oracle itself
    accuracy = None
    if args.workload == "batch96" and rank == 0:
        step()
        torch.cuda.synchronize()
        per_class, ref64 = {}, {}
        for i, b in enumerate(boxes):
            key = (shape_of(b), b.q)
            if key not in ref64:
                ref64[key] = sbp.Plan(b.nx, b.ny, b.nz, b.Lx, b.Ly, b.Lz, q=b.q, Omega=b.Omega, G=b.G, dtype=0)
            want = ref64[key].solve(rhos[i].double(), t=times[i], stream=stream)
            per_class.setdefault("x".join(map(str, shape_of(b))), []).append(errors(phis[i], want))
        for p in ref64.values():
            p.close()
        import oracle as O

        b0 = boxes[0]
        want0 = O.solve(np.asarray(rhos_np[0], dtype=np.float64), O.SolveParams(b0.Lx, b0.Ly, b0.Lz, q=b0.q),
                        times[0])
        accuracy = {"vs_fp64_gpu_worst_box": worst([e for v in per_class.values() for e in v]),
                    "vs_fp64_gpu_per_class": {k: worst(v) for k, v in per_class.items()},
                    "vs_oracle_box0_64x64x64": errors(phis[0], torch.from_numpy(want0).to(dev)),
                    "note": "FP32 batch output of the timed step; the FP64 GPU solves are pinned to the FP64 "
                            "oracle at <= 1e-12 rel-L2 by the test suite"}

    # ---- the same batch in FP64 through one batched call per step (the
    # precision of the accuracy reference), for the FP32/FP64 speed ratio
    batch_fp64 = None
    if args.workload == "batch96" and rank == 0 and not args.no_side:
        plans64 = [sbp.Plan(b.nx, b.ny, b.nz, b.Lx, b.Ly, b.Lz, q=b.q, Omega=b.Omega, G=b.G, dtype=0) for b in boxes]
        r64 = [r.double() for r in rhos]
        f64 = [torch.empty_like(r) for r in r64]
        m64 = event_time_ms(lambda: sbp.solve_batched(plans64, r64, f64, times, stream=stream), stream, 3)
        b64 = sum(alg_bytes(b, 8) for b in boxes)
        batch_fp64 = {"ms_per_step": m64, "solves_per_s": nbox / (m64 / 1e3),
                      "alg_gbs": b64 / (m64 / 1e3) / 1e9, "hbm_frac": b64 / (m64 / 1e3) / 1e9 / peak,
                      "fp32_over_fp64_speed": m64 / ms_per_step,
                      "fp32_vs_fp64_batch_worst_box": worst([errors(phis[i], f64[i]) for i in range(nbox)])}
        for p in plans64:
            p.close()
        del plans64, r64, f64

    # ---- dominant kernel: the middle sweep of the largest shape, launched for
    # all boxes of that shape at once as the batch graph runs it (the padded z
    # pass of one box where that shape runs five passes), timed alone with
    # CUDA events on the launching stream, L2 overwritten before every launch
    big = max(range(nbox), key=lambda i: boxes[i].cells)
    bp, bb = plans[big], boxes[big]
    big_shape = shape_of(bb)
    nbig = sum(1 for b in boxes if shape_of(b) == big_shape)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    grouped_dominant = False
    if args.workload == "batch96":
        try:
            sbp.batch_run_stage(plans, rhos, phis, big_shape, sbp.Stage.SWEEP_MIDDLE, stream=stream)
            grouped_dominant = True
        except sbp.SbpError:
            grouped_dominant = False
    if grouped_dominant:
        zname = f"k3_middle<{bb.nx}, {bb.ny}, {bb.nz}>"
        what = (f"middle sweep: second y stage, padded z pass with the Green's multiply, first inverse y stage; "
                f"one launch for the {nbig} boxes of this shape, as in the batch graph")
        zbytes = nbig * middle_pass_bytes(bb, rb)

        def launch():
            sbp.batch_run_stage(plans, rhos, phis, big_shape, sbp.Stage.SWEEP_MIDDLE, stream=stream)
    else:
        spec = bp.new_spectrum()
        bp.run_stage(sbp.Stage.X_FORWARD, rhos[big], spec, stream=stream)
        bp.run_stage(sbp.Stage.Y_FORWARD, spec, spec, stream=stream)
        bp.run_stage(sbp.Stage.GREEN_FILL, None, spec, t=times[big], stream=stream)
        zname = f"k_z_padded<{'float' if dt == 1 else 'double'}, {16 if dt == 1 else 8}, {bb.nz}>"
        what = "padded z pass of one box"
        zbytes = middle_pass_bytes(bb, rb)

        def launch():
            bp.run_stage(sbp.Stage.Z_CONVOLVE, spec, spec, stream=stream)
    z_ms = event_time_ms(launch, stream, 20, flush=flush)
    z_ms_warm = event_time_ms(launch, stream, 20)
    z_gbs = zbytes / (z_ms / 1e3) / 1e9
    traffic, rec = recorded_traffic(zname)
    roofline = {"bound": "hbm", "kernel": f"{zname} ({what}), {bb.nx}x{bb.ny}x{bb.nz}",
                "achieved": z_gbs, "peak": peak, "unit": "GB/s", "frac": z_gbs / peak,
                "traffic": traffic, "alg_bytes_per_launch": zbytes, "ms_per_launch": z_ms,
                "timing": "L2 overwritten (256 MiB) before each launch; CUDA events per launch on its stream",
                "warm_l2_ms_per_launch": z_ms_warm,
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                "traffic_note": (rec or {}).get("note"),
                "step_alg_gbs": balg / (ms_per_step / 1e3) / 1e9,
                "step_frac": balg / (ms_per_step / 1e3) / 1e9 / peak}
    del flush

    # ---- single-box rows of the other configurations, FP32 and FP64
    side = {}
    cpu_cfg = {}
    pool = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pool = OraclePool(host_cores())
    if args.workload == "batch96" and not args.no_side and rank == 0:
        flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

        def plan_for(b, d, opts=()):
            p = sbp.Plan(b.nx, b.ny, b.nz, b.Lx, b.Ly, b.Lz, q=b.q, Omega=b.Omega, G=b.G, dtype=d)
            for o, v in opts:
                p.set_option(o, v)
            return p

        def timed_solve(p, r, t, reps):
            out = torch.empty_like(r)
            ms_ = event_time_ms(lambda: p.solve(r, out, t=t, stream=stream), stream, reps)
            p.solve(r, out, t=t, stream=stream)
            return ms_, out

        # config 2: 256×256×128, lognormal σ = 0.5 (seed 2), t ∈ {0, 1.3, 5.0}
        b2 = W.BOX_256
        rho2 = torch.from_numpy(W.lognormal_disc(b2, seed=2, sigma=0.5)).to(dev)
        p64, p32 = plan_for(b2, 0), plan_for(b2, 1)
        out2 = {}
        for t in W.T_256:
            m64, o64 = timed_solve(p64, rho2, t, 5)
            m32, o32 = timed_solve(p32, rho2.float(), t, 20)
            out2[t] = (o64, o32)
            side[f"config2_256x256x128_t{t}"] = {
                "fp64": solve_row(b2, m64, 8, peak), "fp32": solve_row(b2, m32, 4, peak),
                "fp32_vs_fp64_gpu": errors(o32, o64), "fp32_over_fp64_speed": m64 / m32}
        # the oracle's full solve of config 2 at t = 1.3 (one of the CPU jobs)
        cfg2_spec = {"kind": "lognormal", "box": box_tuple(b2), "seed": 2, "sigma": 0.5, "t": 1.3, "keep": True}
        # config 3: 512×512×256, FP32 input (seed 3), t = 2.1; its 64³ copy against the oracle
        b3 = W.BOX_512
        rho3 = torch.from_numpy(W.lognormal_disc(b3, seed=3, sigma=0.5, dtype=np.float32)).to(dev)
        p64, p32 = plan_for(b3, 0), plan_for(b3, 1)
        m64, o64 = timed_solve(p64, rho3.double(), W.T_512, 3)
        m32, o32 = timed_solve(p32, rho3, W.T_512, 10)
        side["config3_512x512x256"] = {"fp64": solve_row(b3, m64, 8, peak), "fp32": solve_row(b3, m32, 4, peak),
                                       "fp32_vs_fp64_gpu": errors(o32, o64), "fp32_over_fp64_speed": m64 / m32}
        del p64, p32, o64, o32
        small = W.downsample(rho3.double().cpu().numpy(), 8, 8, 4)
        sb = W.Box(64, 64, 64, b3.Lx, b3.Ly, b3.Lz)
        import oracle as O

        want3 = torch.from_numpy(O.solve(small, O.SolveParams(sb.Lx, sb.Ly, sb.Lz), W.T_512)).to(dev)
        sd = torch.from_numpy(small).to(dev)
        q64, q32 = plan_for(sb, 0), plan_for(sb, 1)
        m64, o64 = timed_solve(q64, sd, W.T_512, 20)
        m32, o32 = timed_solve(q32, sd.float(), W.T_512, 50)
        side["config3_64x64x64_copy"] = {"fp64": solve_row(sb, m64, 8, peak), "fp32": solve_row(sb, m32, 4, peak),
                                         "fp64_vs_oracle": errors(o64, want3), "fp32_vs_oracle": errors(o32, want3)}
        # config 1: 32³ noisy Gaussian (seed 0), t = 0.7, against the oracle;
        # one box alone is launch-latency bound, so 256 such boxes in one
        # batched call are timed too
        b1 = W.BOX_32
        rho1 = W.noisy_gaussian(b1, seed=0)
        want1 = torch.from_numpy(O.solve(rho1, O.SolveParams(b1.Lx, b1.Ly, b1.Lz, q=b1.q, Omega=b1.Omega, G=b1.G),
                                         W.T_32)).to(dev)
        r1 = torch.from_numpy(rho1).to(dev)
        q64, q32 = plan_for(b1, 0), plan_for(b1, 1)
        m64, o64 = timed_solve(q64, r1, W.T_32, 50)
        m32, o32 = timed_solve(q32, r1.float(), W.T_32, 50)
        nb1 = 256
        qs = [plan_for(b1, 1) for _ in range(nb1)]
        rs = [r1.float().clone() for _ in range(nb1)]
        fs = [torch.empty_like(r) for r in rs]
        ts1 = [W.T_32] * nb1
        mb = event_time_ms(lambda: sbp.solve_batched(qs, rs, fs, ts1, stream=stream), stream, 20, flush=flush)
        side["config1_32x32x32"] = {"fp64": solve_row(b1, m64, 8, peak), "fp32": solve_row(b1, m32, 4, peak),
                                    "fp64_vs_oracle": errors(o64, want1), "fp32_vs_oracle": errors(o32, want1),
                                    f"fp32_batched_{nb1}": {"ms_per_call": mb, "solves_per_s": nb1 / (mb / 1e3),
                                                            "worst_vs_oracle": worst([errors(f, want1) for f in fs])}}
        for p in qs:
            p.close()
        del q64, q32, qs, rs, fs
        # config 5: 1024×1024×512 clumpy disc (float32 input), t = 3.3
        b5 = W.BOX_1024
        rho5 = W.clumpy_disc(b5, seed=5, device=dev, dtype=np.float32)
        p32 = plan_for(b5, 1)
        m32, o32 = timed_solve(p32, rho5, W.T_1024, 5)
        del p32
        p64 = plan_for(b5, 0)
        m64, o64 = timed_solve(p64, rho5.double(), W.T_1024, 2)
        del p64
        side["config5_1024x1024x512_clumpy"] = {"fp64": solve_row(b5, m64, 8, peak),
                                                "fp32": solve_row(b5, m32, 4, peak),
                                                "fp32_vs_fp64_gpu": errors(o32, o64),
                                                "fp32_over_fp64_speed": m64 / m32}
        del o32, o64, rho5
        # the "next" rows on the config-2 box at t = 1.3: the paper's α = 1.1
        # with 4·nz padding (Sect. 2.3), the physical frame (Sect. 2.1),
        # SASHA (Sect. 2.2), the force of Sect. 2.4's ghost rule
        O_ = sbp.Option
        for name, opts in (("alpha1.1_pad4", ((O_.TRUNCATION, 1.1),)), ("physical_frame", ((O_.FRAME, 1),)),
                           ("sasha", ((O_.METHOD, 2),))):
            q64, q32 = plan_for(b2, 0, opts), plan_for(b2, 1, opts)
            m64, o64 = timed_solve(q64, rho2, 1.3, 3)
            m32, o32 = timed_solve(q32, rho2.float(), 1.3, 20)
            side[f"config2_{name}"] = {"fp64": solve_row(b2, m64, 8, peak), "fp32": solve_row(b2, m32, 4, peak),
                                       "fp32_vs_fp64_gpu": errors(o32, o64)}
        g = torch.empty((3,) + tuple(rho2.shape), dtype=torch.float32, device=dev)
        phi2 = out2[1.3][1]
        pf = plan_for(b2, 1)
        mf = event_time_ms(lambda: pf.force(phi2, t=1.3, out=g, stream=stream), stream, 20, flush=flush)
        side["config2_force_fp32"] = {"ms_per_call": mf,
                                      "gb_per_s": 4 * phi2.numel() * 4 / (mf / 1e3) / 1e9}
        side["batch_fp32_vs_config2_fp64_cells_speedup"] = (cells / (ms_per_step / 1e3) / 1e9) / \
            side["config2_256x256x128_t1.3"]["fp64"]["gcells_per_s"]
        del flush

        # the CPU oracle on the host cores: config 1 (32³) and the 64³ copy of
        # config 3 with one process and with one per core; config 2 at t = 1.3
        # as one process (its answer also checks the GPU solves)
        if pool is not None:
            cores = pool.cores
            b1 = W.BOX_32
            cfg1 = {"kind": "noisy", "box": box_tuple(b1), "seed": 0, "t": W.T_32}
            cfg3 = {"kind": "array", "rho": small, "box": box_tuple(sb), "t": W.T_512}
            for name, spec, box in (("config1_32x32x32", cfg1, b1), ("config3_copy_64x64x64", cfg3, sb)):
                one = _run_single(spec)
                wall, _ = pool.run([spec] * cores)
                cpu_cfg[name] = {"one_process": {"solves_per_s": 1.0 / one[0], "cores": 1},
                                 "all_cores": {"solves_per_s": cores / wall, "cores": cores,
                                               "gcells_per_s": cores * box.cells / wall / 1e9}}
    # ---- the CPU baseline: the batch's size classes, one process per core
    cpu = None
    if pool is not None:
        extra = cfg2_spec if "cfg2_spec" in locals() else None
        rate, details, kept = cpu_batch_baseline(pool, boxes, extra_256=extra)
        pool.close()
        cores = pool.cores
        cpu = {"value": rate, "unit": "solves/s", "cores": cores, "kind": "oracle",
               "sample": f"one round per size class of the batch: {cores} spawned processes (one per host core, "
                         f"one BLAS thread each) each solved one box of that class with the FP64 oracle at the same "
                         f"time; class rate = {cores} / the round's longest solve; batch rate = {nbox} / sum over "
                         f"classes of count / class rate",
               "classes": details}
        if kept is not None:
            wall, cpu_s, phi_o = kept
            want2 = torch.from_numpy(phi_o).to(dev)
            cpu_cfg["config2_256x256x128_t1.3"] = {
                "one_process": {"solves_per_s": 1.0 / wall, "cores": 1,
                                "note": "one of the processes of the 256x256x128 round (the others busy)"},
                "all_cores": {"solves_per_s": details["256x256x128"]["solves_per_s"], "cores": cores,
                              "note": "the batch's 256x256x128 round: same size, same cost"}}
            o64, o32 = out2[1.3]
            side["config2_256x256x128_t1.3"]["fp64_vs_oracle"] = errors(o64, want2)
            side["config2_256x256x128_t1.3"]["fp32_vs_oracle"] = errors(o32, want2)
        if cpu_cfg:
            cpu["configs"] = cpu_cfg

    if rank == 0:
        config = {"workload": args.workload, "boxes": nbox, "cells_per_step": cells,
                  "gcells_per_s": world * cells * args.steps / (ms / 1e3) / 1e9,
                  "alg_bytes_per_step": balg, "l2": "inputs larger than L2 (no flush needed)"
                  if sum(r.numel() * r.element_size() for r in rhos) > 129e6 else "inputs smaller than L2",
                  "parallelism": f"replicas x{world}",
                  "schedule": {"boxes_in_grouped_sweeps": grouped_boxes,
                               "boxes_on_own_kernels": nbox - grouped_boxes,
                               "kernel_launches_per_step": launches_per_step}}
        line = result_line(args, world, value, ms_per_step, "f64" if dt == 0 else "f32", config,
                           roofline=roofline, cpu_baseline=cpu,
                           e2e={"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d,
                                "d2h_bytes_per_step": h2d},
                           gpu_launches=launches_per_step * args.steps,
                           clocks=clk.summary(), accuracy=accuracy, batch_fp64=batch_fp64, single_box=side)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def _run_single(spec):
    """One oracle solve in a fresh spawned process with one BLAS thread."""
    import multiprocessing as mp

    with mp.get_context("spawn").Pool(1, initializer=_oracle_init) as p:
        return p.map(_oracle_job, [spec])[0]


if __name__ == "__main__":
    main()
