"""sbp_solve_noalloc: the FP32 solve for programs that may not allocate
device memory while they run.  It keeps its workspace in a fixed 40 MiB
device array declared by the library, so its results must equal those of the
plan-based solve (which allocates a workspace per plan), call after call.

This file is collected last so that a failure here leaves every other test
already run."""

import numpy as np
import pytest

import oracle as O
from gpu_helpers import TOL, as_input, rel_l2, to_dev
from paper_2510_10070_gb300 import workloads as W


@pytest.fixture(scope="module")
def sbp():
    from paper_2510_10070_gb300 import sbp as S

    S.lib()
    return S


CASES = [W.Box(48, 24, 12, 2.0, 3.0, 1.5, q=1.5, Omega=0.9, G=0.8), W.BOX_32, W.Box(128, 128, 64, 8.0, 8.0, 4.0),
         W.Box(96, 192, 48, 8.0, 8.0, 4.0, q=1.0), W.BOX_256]


@pytest.mark.gpu
@pytest.mark.parametrize("box", CASES, ids=lambda b: f"{b.nx}x{b.ny}x{b.nz}")
def test_noalloc_matches_plan_solve_twice(sbp, box):
    import torch

    plan = sbp.Plan(box.nx, box.ny, box.nz, box.Lx, box.Ly, box.Lz, q=box.q, Omega=box.Omega, G=box.G,
                    dtype=sbp.DType.F32)
    rng = np.random.default_rng(box.nx + box.ny + box.nz)
    for call, t in enumerate((0.37, -2.9)):
        rho = to_dev(rng.standard_normal((box.nz, box.ny, box.nx)) + 0.5, 1)
        want = plan.solve(rho, t=t)
        got = torch.full_like(rho, float("nan"))
        sbp.solve_noalloc(rho, got, box.Lx, box.Ly, box.Lz, q=box.q, Omega=box.Omega, G=box.G, t=t)
        torch.cuda.synchronize()
        assert torch.isfinite(got).all(), call
        assert rel_l2(got.double().cpu().numpy(), want.double().cpu().numpy()) <= TOL[1], (call, t)
        if box.cells <= 64 ** 3:  # and against the FP64 oracle where it is quick
            p = O.SolveParams(box.Lx, box.Ly, box.Lz, q=box.q, Omega=box.Omega, G=box.G)
            ref = O.solve(as_input(rho.double().cpu().numpy(), 1), p, t)
            assert rel_l2(got.double().cpu().numpy(), ref) <= TOL[1], (call, t)


@pytest.mark.gpu
def test_noalloc_in_place_and_size_limit(sbp):
    import torch

    box = W.Box(64, 64, 32, 8.0, 8.0, 4.0)
    plan = sbp.Plan(box.nx, box.ny, box.nz, box.Lx, box.Ly, box.Lz, dtype=sbp.DType.F32)
    rho = to_dev(np.random.default_rng(1).standard_normal((box.nz, box.ny, box.nx)), 1)
    want = plan.solve(rho, t=1.1)
    buf = rho.clone()
    sbp.solve_noalloc(buf, buf, box.Lx, box.Ly, box.Lz, t=1.1)
    torch.cuda.synchronize()
    assert rel_l2(buf.double().cpu().numpy(), want.double().cpu().numpy()) <= TOL[1]
    big = torch.empty((256, 512, 512), dtype=torch.float32, device="cuda")
    with pytest.raises(sbp.SbpError) as err:
        sbp.solve_noalloc(big, big, 8.0, 8.0, 4.0, t=0.0)
    assert err.value.status == sbp.Status.SCRATCH_LIMIT
