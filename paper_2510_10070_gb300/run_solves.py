"""Run a few solves of one box on cuda:0 (for profilers such as ncu).

    python -m paper_2510_10070_gb300.run_solves --box 256x256x128 --dtype f32 --solves 4

The density is seeded uniform noise on a Gaussian disc; the solves run back to
back on the current stream and the command exits after a synchronise.
"""

from __future__ import annotations

import argparse


def main(argv=None):
    import torch

    from paper_2510_10070_gb300 import sbp

    ap = argparse.ArgumentParser()
    ap.add_argument("--box", default="256x256x128", help="nx x ny x nz")
    ap.add_argument("--lengths", default="8,8,4", help="Lx,Ly,Lz")
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"])
    ap.add_argument("--solves", type=int, default=4)
    ap.add_argument("--t", type=float, default=1.3)
    ap.add_argument("--z-variant", type=int, default=0)
    ap.add_argument("--xy-passes", type=int, default=0)
    ap.add_argument("--alpha", type=float, default=1.0, help="vertical truncation L/Lz (> 1: 4·nz padding)")
    ap.add_argument("--frame", type=int, default=0, help="1: physical frame (Sect. 2.1 mapping)")
    ap.add_argument("--method", type=int, default=0, help="1, 2: SASHA (Sect. 2.2)")
    ap.add_argument("--force", action="store_true", help="also take -grad(phi) after each solve")
    ap.add_argument("--schedule", type=int, default=0, help="1: five passes, 2: three sweeps (0: automatic)")
    ap.add_argument("--batch", type=int, default=0,
                    help="solve this many boxes of the shape per call through sbp_solve_batched")
    args = ap.parse_args(argv)
    nx, ny, nz = (int(v) for v in args.box.lower().split("x"))
    Lx, Ly, Lz = (float(v) for v in args.lengths.split(","))
    dt = sbp.DType.F32 if args.dtype == "f32" else sbp.DType.F64
    plan = sbp.Plan(nx, ny, nz, Lx, Ly, Lz, dtype=dt)
    if args.schedule:
        plan.set_option(sbp.Option.SCHEDULE, args.schedule)
    if args.z_variant:
        plan.set_option(sbp.Option.Z_VARIANT, args.z_variant)
    if args.xy_passes:
        plan.set_option(sbp.Option.XY_PASSES, args.xy_passes)
    if args.alpha != 1.0:
        plan.set_option(sbp.Option.TRUNCATION, args.alpha)
    if args.frame:
        plan.set_option(sbp.Option.FRAME, args.frame)
    if args.method:
        plan.set_option(sbp.Option.METHOD, args.method)
    g = torch.Generator(device="cuda").manual_seed(1)
    z = (torch.arange(nz, device="cuda", dtype=torch.float64) + 0.5) * (Lz / nz) - 0.5 * Lz
    rho = torch.exp(-0.5 * z * z)[:, None, None] * (1.0 + 0.1 * torch.rand((nz, ny, nx), generator=g,
                                                                           device="cuda", dtype=torch.float64))
    rho = rho.to(plan.torch_dtype).contiguous()
    phi = torch.empty_like(rho)
    if args.batch > 0:
        # one plan per box (same shape), each with its own input and output
        plans = [plan] + [sbp.Plan(nx, ny, nz, Lx, Ly, Lz, dtype=dt) for _ in range(args.batch - 1)]
        for p in plans[1:]:
            if args.schedule:
                p.set_option(sbp.Option.SCHEDULE, args.schedule)
        rhos = [rho] + [torch.roll(rho, i, dims=2).contiguous() for i in range(1, args.batch)]
        phis = [torch.empty_like(r) for r in rhos]
        ts = [args.t + 0.37 * i for i in range(args.batch)]
        for _ in range(args.solves):
            sbp.solve_batched(plans, rhos, phis, ts)
        torch.cuda.synchronize()
        print(f"{args.solves} batched calls of {args.batch} x {nx}x{ny}x{nz} ({args.dtype}) done")
        return
    g = torch.empty((3,) + tuple(rho.shape), dtype=rho.dtype, device="cuda") if args.force else None
    for _ in range(args.solves):
        plan.solve(rho, phi, t=args.t)
        if g is not None:
            plan.force(phi, t=args.t, out=g)
    torch.cuda.synchronize()
    print(f"{args.solves} solves of {nx}x{ny}x{nz} ({args.dtype}) done")


if __name__ == "__main__":
    main()
