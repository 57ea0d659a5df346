"""Failure detection without a GPU fault: the TMA kernels wait for their
copies with a bounded clock budget; when the copy is withheld (a test switch
that arms nothing), the wait runs out, the kernel records the timeout in the
plan's status word and returns, the host reads SBP_ERR_DEVICE_TIMEOUT, and
the context stays usable."""

import numpy as np
import pytest

import oracle as O
from gpu_helpers import STAGE_TOL, np_to_spec, rel_l2, spec_input, spec_to_np
from paper_2510_10070_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sbp():
    from paper_2510_10070_gb300 import sbp as S

    S.lib()
    return S


def test_withheld_copy_times_out_and_plan_recovers(sbp):
    nx, ny, nz = 64, 128, 8
    plan = sbp.Plan(nx, ny, nz, 2.0, 3.0, 1.5, dtype=sbp.DType.F32)
    rng = np.random.default_rng(31)
    X = rng.standard_normal((nz, ny, nx // 2 + 1)) + 1j * rng.standard_normal((nz, ny, nx // 2 + 1))
    spec = np_to_spec(X, plan.spectrum_pitch, 1)
    plan.set_option(sbp.Option.SPIN_BUDGET, 2e6)  # about a millisecond
    plan.set_option(sbp.Option.DEBUG_WITHHOLD_COPY, 1)
    plan.run_stage(sbp.Stage.Y_FORWARD, spec, spec)
    with pytest.raises(sbp.SbpError) as err:
        plan.sync_status()
    assert err.value.status == sbp.Status.DEVICE_TIMEOUT
    plan.sync_status()  # the status word was cleared
    # the same plan and context work again
    plan.set_option(sbp.Option.DEBUG_WITHHOLD_COPY, 0)
    spec = np_to_spec(X, plan.spectrum_pitch, 1)
    plan.run_stage(sbp.Stage.Y_FORWARD, spec, spec)
    plan.sync_status()
    want = O.dft_y(spec_input(X, 1), -1.0)
    assert rel_l2(spec_to_np(spec, nx // 2 + 1), want) <= STAGE_TOL[1]


def test_y_pass_tma_and_plain_loads_agree(sbp):
    import torch

    nx, ny, nz = 96, 256, 4
    plan = sbp.Plan(nx, ny, nz, 2.0, 3.0, 1.5, dtype=sbp.DType.F32)
    rng = np.random.default_rng(32)
    X = rng.standard_normal((nz, ny, nx // 2 + 1)) + 1j * rng.standard_normal((nz, ny, nx // 2 + 1))
    a = np_to_spec(X, plan.spectrum_pitch, 1)
    b = a.clone()
    plan.run_stage(sbp.Stage.Y_FORWARD, a, a)        # TMA (default)
    plan.set_option(sbp.Option.Y_TMA, 1)
    plan.run_stage(sbp.Stage.Y_FORWARD, b, b)        # plain loads
    torch.cuda.synchronize()
    h = nx // 2 + 1
    assert torch.equal(a[..., :h, :], b[..., :h, :])


def test_sweep_tma_wait_times_out_and_plan_recovers(sbp):
    # The three-sweep schedule loads pass C's box of the half spectrum by TMA
    # (128x128x64 and 256x256x128): with the copy withheld its bounded wait
    # runs out, the status word reports it and the next solve is correct.
    import torch

    box = W.Box(128, 128, 64, 8.0, 8.0, 4.0)
    plan = sbp.Plan(box.nx, box.ny, box.nz, box.Lx, box.Ly, box.Lz, dtype=sbp.DType.F32)
    plan.set_option(sbp.Option.SCHEDULE, 2)
    rho = torch.tensor(np.random.default_rng(33).standard_normal((64, 128, 128)) + 1.0, dtype=torch.float32,
                       device="cuda")
    plan.set_option(sbp.Option.SPIN_BUDGET, 2e6)
    plan.set_option(sbp.Option.DEBUG_WITHHOLD_COPY, 1)
    plan.solve(rho, t=0.4)
    with pytest.raises(sbp.SbpError) as err:
        plan.sync_status()
    assert err.value.status == sbp.Status.DEVICE_TIMEOUT
    plan.sync_status()
    plan.set_option(sbp.Option.DEBUG_WITHHOLD_COPY, 0)
    got = plan.solve(rho, t=0.4).double().cpu().numpy()
    plan.sync_status()
    want = O.solve(rho.double().cpu().numpy(), O.SolveParams(box.Lx, box.Ly, box.Lz), 0.4)
    assert rel_l2(got, want) <= 2e-5
