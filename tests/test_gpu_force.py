"""Ghost layers and forces on the GPU (Sect. 2.4, last paragraph) against the oracle.

sbp_fill_ghosts continues the last active cell's gradient into ng layers;
sbp_force takes -∇Φ by central differences (periodic y; x periodic or, in the
physical frame, shear-periodic; one-sided in the boundary planes).  Inputs are
compared as the device holds them; FP64 to rounding, FP32 at rel-L2 ≤ 2e-5.
"""

import numpy as np
import pytest

import oracle as O
from gpu_helpers import TOL, as_input, rel_l2, to_dev
from paper_2510_10070_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sbp():
    from paper_2510_10070_gb300 import sbp as S

    S.lib()
    return S


def _plan(sbp, box, dtype, frame=0):
    plan = sbp.Plan(box.nx, box.ny, box.nz, box.Lx, box.Ly, box.Lz, q=box.q, dtype=dtype)
    if frame:
        plan.set_option(sbp.Option.FRAME, 1)
    return plan


def _params(box):
    return O.SolveParams(box.Lx, box.Ly, box.Lz, q=box.q, Omega=box.Omega, G=box.G)


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("ng", [1, 2, 5])
def test_fill_ghosts(sbp, dtype, ng):
    box = W.Box(48, 24, 12, 2.0, 3.0, 1.5)
    rng = np.random.default_rng(ng)
    phi = rng.standard_normal((12, 24, 48))
    got = _plan(sbp, box, dtype).fill_ghosts(to_dev(phi, dtype), ng).double().cpu().numpy()
    want = O.fill_ghosts(as_input(phi, dtype), ng)
    assert got.shape == want.shape
    assert np.max(np.abs(got - want)) <= (1e-14 if dtype == 0 else 2e-6) * np.max(np.abs(want))


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("shape", [(32, 32, 16), (64, 96, 12), (96, 64, 24), (256, 32, 8)])
@pytest.mark.parametrize("frame", [0, 1])
def test_force_parity(sbp, dtype, shape, frame):
    nx, ny, nz = shape
    box = W.Box(nx, ny, nz, 2.0, 3.0, 1.5, q=1.5)
    rng = np.random.default_rng(nx + ny + nz + frame)
    phi = rng.standard_normal((nz, ny, nx))
    t = 0.83
    got = _plan(sbp, box, dtype, frame).force(to_dev(phi, dtype), t=t).double().cpu().numpy()
    want = O.force(as_input(phi, dtype), _params(box), t, physical=bool(frame))
    assert rel_l2(got, want) <= (1e-13 if dtype == 0 else TOL[1])


@pytest.mark.parametrize("dtype", [0, 1])
def test_solve_then_force_physical_frame(sbp, dtype):
    box = W.Box(64, 64, 32, 4.0, 4.0, 2.0, q=1.5)
    rho = W.noisy_gaussian(box, seed=9)
    t = 2.4
    plan = _plan(sbp, box, dtype, frame=1)
    phi = plan.solve(to_dev(rho, dtype), t=t)
    g = plan.force(phi, t=t).double().cpu().numpy()
    want = O.force(O.solve_physical(as_input(rho, dtype), _params(box), t), _params(box), t, physical=True)
    assert rel_l2(g, want) <= TOL[dtype] * (1 if dtype else 10)


def test_ghost_and_force_argument_errors(sbp):
    import torch

    box = W.Box(32, 32, 8, 1.0, 1.0, 1.0)
    plan = _plan(sbp, box, 0)
    phi = torch.zeros((8, 32, 32), dtype=torch.float64, device="cuda")
    for bad in (0, 17):
        with pytest.raises(sbp.SbpError) as e:
            plan.fill_ghosts(phi, bad)
        assert e.value.status == sbp.Status.INVALID_ARG
    big = torch.zeros((3 * 8 + 8, 32, 32), dtype=torch.float64, device="cuda")
    with pytest.raises(sbp.SbpError) as e:  # force overlapping phi
        plan.force(big[:8], out=big[4:4 + 24].view(3, 8, 32, 32))
    assert e.value.status == sbp.Status.INVALID_ARG
