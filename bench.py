#!/usr/bin/env python
"""Throughput of the shearing-box VGF-HybridBC Poisson solver on GB300.

    python bench.py [--gpus N --steps K --warmup W] [--workload batch96|box256|box256_f64]
                    [--impl ours|reference]

A step is one pass of the whole method over one batch of synthetic input:
by default the 96-box FP32 batch (32× 64³, 32× 128²×64, 16× 192²×96,
16× 256²×128, each box with its own shear time and q), solved through
sbp_solve_batched.  Inputs (931 MB) are larger than L2, so no flush is
needed between steps.  Under torchrun every rank solves its own copy of the
batch (weak scaling, no collective on the data path); rank 0 prints one JSON
line with the whole-job rate.

--impl reference times the FP64 CPU oracle (numpy) on the host cores on a
bounded sample of the same workload and extrapolates to the batch by the
oracle's operation count.
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


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": HBM_PEAK_FALLBACK}, "fallback"


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def build_workload(name):
    import numpy as np

    from paper_2510_10070_gb300 import workloads as W

    if name == "batch96":
        case = W.batch_96()
        boxes, times = case.boxes, [float(t) for t in case.times]
        rhos = [W.lognormal_disc(b, seed=s, sigma=0.7, dtype=np.float32) for b, s in zip(boxes, case.seeds)]
        return boxes, rhos, times, 1
    if name in ("box256", "box256_f64"):
        box = W.BOX_256
        rho = W.lognormal_disc(box, seed=2, sigma=0.5)
        dt = 0 if name == "box256_f64" else 1
        return [box], [rho if dt == 0 else rho.astype(np.float32)], [1.3], dt
    raise SystemExit(f"unknown workload {name}")


def recorded_traffic(kernel_name, key=None):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    record (or the record's field `key`), or None when the kernel sources
    changed since it was taken."""
    import hashlib

    try:
        with open(os.path.join(ROOT, "profiles", "z_pass_traffic.json")) as f:
            rec = json.load(f)
        h = hashlib.sha256()
        for name in ("sbp_kernels.cuh", "sbp_fft.cuh"):
            with open(os.path.join(ROOT, "paper_2510_10070_gb300", "csrc", name), "rb") as f:
                h.update(f.read())
    except (OSError, ValueError):
        return None
    if rec.get("source_sha256") != h.hexdigest() or rec.get("kernel") != kernel_name:
        return None
    if key is not None:
        return rec.get(key)
    return rec["dram_bytes_read"] + rec["dram_bytes_write"]


def issue_view(warp_instr, ms, dev, peaks):
    if not warp_instr:
        return None
    import torch

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = peaks.get("sm_max_mhz", 2070.0)
    peak = sms * 4 * mhz * 1e6 / 1e9  # G warp-instructions/s
    achieved = warp_instr / (ms / 1e3) / 1e9
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gwarp-instr/s", "frac": achieved / peak,
            "warp_instructions_per_launch": warp_instr, "peak_source": f"{sms} SMs x 4 schedulers x {mhz:.0f} MHz"}


def alg_bytes(box, rb):
    """B_alg of one solve: read ρ, write φ, and the half spectrum written by
    the forward passes, read and written by the z pass and read by the
    inverse passes (three-sweep model)."""
    N = box.nx * box.ny * box.nz
    H = (box.nx // 2 + 1) * box.ny * box.nz
    return 2 * N * rb + 8 * H * rb


def z_pass_bytes(box, rb):
    """Algorithmic bytes of one z-pass launch: read and write the half spectrum."""
    H = (box.nx // 2 + 1) * box.ny * box.nz
    return 2 * 2 * H * rb


def oracle_cost(box):
    """Multiply-add count of the oracle's direct sums (for extrapolation)."""
    nx, ny, nz = box.nx, box.ny, box.nz
    return (2 * nz * ny * nx * (nx + ny)      # forward + inverse horizontal DFTs
            + nx * ny * (2 * nz) * (2 * nz - 1)  # vertical kernel by direct sum
            + nx * ny * nz * nz)              # Toeplitz sums


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
# CPU oracle timing
# ---------------------------------------------------------------------------

def oracle_rate(boxes, rhos, times, budget_s=20.0):
    """Time the oracle on a bounded sample; return (solves/s, Gcells/s, sample text, cores)."""
    import numpy as np

    import oracle as O

    order = sorted(range(len(boxes)), key=lambda i: boxes[i].cells)
    seen, sample = set(), []
    for i in order:  # one box of each size class, smallest first
        key = (boxes[i].nx, boxes[i].ny, boxes[i].nz)
        if key not in seen:
            seen.add(key)
            sample.append(i)
    spent, per_cost = 0.0, []
    done = []
    for i in sample:
        b = boxes[i]
        est = (spent / sum(oracle_cost(boxes[j]) for j in done) * oracle_cost(b)) if done else 0.0
        if done and spent + est > budget_s:
            break
        p = O.SolveParams(b.Lx, b.Ly, b.Lz, q=b.q, Omega=b.Omega, G=b.G)
        t0 = time.perf_counter()
        O.solve(np.asarray(rhos[i], dtype=np.float64), p, times[i])
        dt = time.perf_counter() - t0
        spent += dt
        done.append(i)
        per_cost.append(dt / oracle_cost(b))
    sec_per_op = sum(per_cost) / len(per_cost)
    total = sum(sec_per_op * oracle_cost(b) for b in boxes)
    cells = sum(b.cells for b in boxes)
    names = ", ".join(f"{boxes[i].nx}x{boxes[i].ny}x{boxes[i].nz}" for i in done)
    text = (f"oracle solved one box of each of [{names}] ({spent:.1f} s); the rest of the "
            f"{len(boxes)}-box workload is extrapolated by the oracle's multiply-add count")
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count()
    return len(boxes) / total, cells / total / 1e9, text, cores, total


# ---------------------------------------------------------------------------
# main
# ---------------------------------------------------------------------------

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="batch96", choices=["batch96", "box256", "box256_f64"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.warmup < 3:
        raise SystemExit("--warmup must be at least 3")

    if args.impl == "reference":
        if rank != 0:
            return
        boxes, rhos, times, dt = build_workload(args.workload)
        vals = []
        for _ in range(args.warmup + args.steps):
            r, g, text, cores, tot = oracle_rate(boxes, rhos, times, budget_s=5.0)
            vals.append(r)
        v = statistics.median(vals[args.warmup:])
        gc = v * sum(b.cells for b in boxes) / len(boxes) / 1e9
        line = {"metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * len(boxes) / v, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
                "config": {"workload": args.workload, "boxes": len(boxes), "gcells_per_s": gc},
                "cpu_baseline": {"value": v, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": text},
                "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import numpy as np
    import torch

    from paper_2510_10070_gb300 import sbp

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

    def step():
        sbp.solve_batched(plans, rhos, phis, times, stream=stream)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        start.record(stream)
        for _ in range(args.steps):
            step()
        end.record(stream)
        barrier()
    ms = max_over_ranks(start.elapsed_time(end), device=dev)
    ms_per_step = ms / args.steps
    nbox = len(boxes)
    value = job_rate(nbox, args.steps, world, ms)
    cells = sum(b.cells for b in boxes)
    balg = sum(alg_bytes(b, rb) for b in boxes)

    # end to end: pinned host input → device, solve, device → pinned host output
    # End to end: every step copies its inputs from pinned host memory, solves
    # through sbp_solve_batched and copies its results back.  All boxes sit in
    # one pinned host buffer and one device buffer per direction (each box at
    # a 256-byte aligned offset), so a step's copies are one transfer each way.
    # Two device buffer sets let step i+1's host-to-device copy and step i-1's
    # device-to-host copy run on their own streams while step i solves; the
    # events keep every buffer's uses in order.
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
    dev_flat = [(torch.empty(total, dtype=tdt, device=dev), torch.empty(total, dtype=tdt, device=dev))
                for _ in range(2)]
    sets = [(views(fi), views(fo)) for fi, fo in dev_flat]
    s_in = torch.cuda.Stream(device=dev)
    s_out = torch.cuda.Stream(device=dev)
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    used = [False, False]

    def e2e_step(i):
        k = i % 2
        r_set, f_set = sets[k]
        with torch.cuda.stream(s_in):
            if used[k]:
                s_in.wait_event(ev_done[k])  # the solve two steps back has read these inputs
            dev_flat[k][0].copy_(flat_in, non_blocking=True)
            ev_in[k].record(s_in)
        stream.wait_event(ev_in[k])
        if used[k]:
            stream.wait_event(ev_out[k])  # the copy-out two steps back has read these outputs
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

    for i in range(4):
        e2e_step(i)
    e2e_drain()
    barrier()
    e2e_steps = max(4, args.steps // 4)
    s2, e2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s2.record(stream)
    s_in.wait_stream(stream)
    for i in range(e2e_steps):
        e2e_step(i)
    e2e_drain()
    e2.record(stream)
    barrier()
    e2e_value = job_rate(nbox, e2e_steps, world, max_over_ranks(s2.elapsed_time(e2), device=dev))

    # dominant kernel: the z pass of the largest box, timed alone with CUDA
    # events on the launching stream, on the same data
    big = max(range(nbox), key=lambda i: boxes[i].cells)
    bp = plans[big]
    spec = bp.new_spectrum()
    bp.run_stage(sbp.Stage.X_FORWARD, rhos[big], spec, stream=stream)
    bp.run_stage(sbp.Stage.Y_FORWARD, spec, spec, stream=stream)
    bp.run_stage(sbp.Stage.GREEN_FILL, None, spec, t=times[big], stream=stream)
    zreps = 20
    for _ in range(3):
        bp.run_stage(sbp.Stage.Z_CONVOLVE, spec, spec, stream=stream)
    zs, ze = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    zs.record(stream)
    for _ in range(zreps):
        bp.run_stage(sbp.Stage.Z_CONVOLVE, spec, spec, stream=stream)
    ze.record(stream)
    torch.cuda.synchronize()
    z_ms = zs.elapsed_time(ze) / zreps
    peaks, peak_src = measured_peaks()
    zbytes = z_pass_bytes(boxes[big], rb)
    z_gbs = zbytes / (z_ms / 1e3) / 1e9
    zb = boxes[big]
    zname = f"k_z_padded<{'float' if dt == 1 else 'double'}, {16 if dt == 1 else 8}, {zb.nz}>"
    roofline = {"bound": "hbm", "kernel": f"{zname} (z pass), {zb.nx}x{zb.ny}x{zb.nz}",
                "achieved": z_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": z_gbs / peaks["hbm_gbs"],
                "traffic": recorded_traffic(zname), "alg_bytes_per_launch": zbytes,
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                "step_alg_gbs": balg / (ms_per_step / 1e3) / 1e9,
                # the z pass is bound by instruction issue, not HBM: the same
                # launch against the SMs' issue rate (4 schedulers per SM, one
                # warp instruction each per clock at the measured max clock),
                # with the warp instructions counted by ncu for this launch
                "issue_view": issue_view(recorded_traffic(zname, "warp_instructions"), z_ms, dev, peaks),
                "step_frac": balg / (ms_per_step / 1e3) / 1e9 / peaks["hbm_gbs"]}

    # FP64 and FP32 single-box reference numbers (the "vs FP64" of the metric)
    side = {}
    if args.workload == "batch96":
        from paper_2510_10070_gb300 import workloads as W

        rho256 = W.lognormal_disc(W.BOX_256, seed=2, sigma=0.5)
        # the "next" rows on the same box: the paper's α = 1.1 with 4·nz padding
        # (Sect. 2.3), the physical frame (Sect. 2.1 mapping fused into the y
        # passes) and SASHA (Sect. 2.2); plus the force of Sect. 2.4's ghost rule
        O = sbp.Option
        cases = (("box256_fp64", 0, ()), ("box256_fp32", 1, ()),
                 ("box256_fp64_alpha1.1_pad4", 0, ((O.TRUNCATION, 1.1),)),
                 ("box256_fp32_alpha1.1_pad4", 1, ((O.TRUNCATION, 1.1),)),
                 ("box256_fp32_physical_frame", 1, ((O.FRAME, 1),)),
                 ("box256_fp32_sasha", 1, ((O.METHOD, 2),)),
                 ("box256_fp32_force", 1, ("force",)))
        for name, d, opts in cases:
            b = W.BOX_256
            p = sbp.Plan(b.nx, b.ny, b.nz, b.Lx, b.Ly, b.Lz, q=b.q, dtype=d)
            force = "force" in opts
            for o in opts:
                if o != "force":
                    p.set_option(o[0], o[1])
            r = torch.from_numpy(rho256).to(device=dev, dtype=torch.float64 if d == 0 else torch.float32)
            f = torch.empty_like(r)
            g = torch.empty((3,) + tuple(r.shape), dtype=r.dtype, device=dev) if force else None

            def once():
                if force:
                    p.force(r, t=1.3, out=g, stream=stream)
                else:
                    p.solve(r, f, t=1.3, stream=stream)
            for _ in range(3):
                once()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 5 if d == 0 else 20
            a0.record(stream)
            for _ in range(reps):
                once()
            a1.record(stream)
            torch.cuda.synchronize()
            t_ms = a0.elapsed_time(a1) / reps
            if force:
                side[name] = {"ms_per_call": t_ms, "gb_per_s": 4 * r.numel() * r.element_size() / (t_ms / 1e3) / 1e9}
            else:
                side[name] = {"ms_per_solve": t_ms, "solves_per_s": 1e3 / t_ms,
                              "gcells_per_s": b.cells / (t_ms / 1e3) / 1e9}
        side["batch_fp32_vs_box256_fp64_cells_speedup"] = (cells / (ms_per_step / 1e3) / 1e9) / \
            side["box256_fp64"]["gcells_per_s"]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, g, text, cores, tot = oracle_rate(boxes, rhos_np, times)
        cpu = {"value": r, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": text}

    per_box_kernels = 5
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if dt == 0 else "f32", "data": "synthetic",
            "config": {"workload": args.workload, "boxes": nbox, "cells_per_step": cells,
                       "gcells_per_s": world * cells * args.steps / (ms / 1e3) / 1e9,
                       "alg_bytes_per_step": balg, "l2": "inputs larger than L2 (no flush needed)"
                       if sum(r.numel() * r.element_size() for r in rhos) > 129e6 else "inputs smaller than L2",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d},
            "gpu_launches": per_box_kernels * nbox * args.steps,
            "clocks": clk.summary(),
            "single_box": side,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
