"""SASHA on the GPU (SBP_OPT_METHOD = 1 or 2) against the oracle (Sect. 2.2).

Φ = Φ0 + Φ_P: a one-block FP64 kernel after the z pass forms ρ̄, z0, Φ0 and
the k = 0 column from the plane sums; the z pass applies -1/|k|² (the VGF
pipeline with e^{-kL} = 0).  Bars: rel-L2 ≤ 1e-12 (FP64), ≤ 2e-5 (FP32).
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


def _plan(sbp, box, dtype, method, frame=0):
    plan = sbp.Plan(box.nx, box.ny, box.nz, box.Lx, box.Ly, box.Lz, q=box.q, Omega=box.Omega, G=box.G,
                    dtype=dtype)
    if frame:
        plan.set_option(sbp.Option.FRAME, 1)
    plan.set_option(sbp.Option.METHOD, method)
    return plan


def _params(box):
    return O.SolveParams(box.Lx, box.Ly, box.Lz, q=box.q, Omega=box.Omega, G=box.G)


SHAPES = [(32, 32, 16), (48, 24, 12), (64, 64, 32), (96, 64, 24), (24, 16, 128), (12, 8, 256), (256, 32, 8)]


@pytest.mark.parametrize("method", [1, 2])
@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("shape", SHAPES)
def test_sasha_parity(sbp, shape, dtype, method):
    nx, ny, nz = shape
    box = W.Box(nx, ny, nz, 2.0, 3.0, 1.5, q=1.5, G=0.9)
    rng = np.random.default_rng(nx + ny + nz)
    z = (np.arange(nz) + 0.5) / nz - 0.3  # off-centre mass: z0 ≠ 0
    rho = np.exp(-8.0 * z * z)[:, None, None] * (1.0 + 0.2 * rng.standard_normal((nz, ny, nx)))
    t = 1.37
    got = _plan(sbp, box, dtype, method).solve(to_dev(rho, dtype), t=t).double().cpu().numpy()
    want = O.solve_sasha(as_input(rho, dtype), _params(box), t, 1.0 if method == 1 else 0.5)
    assert rel_l2(got, want) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [0, 1])
def test_sasha_physical_frame(sbp, dtype):
    box = W.Box(64, 32, 16, 2.0, 3.0, 1.5, q=1.5)
    rng = np.random.default_rng(3)
    rho = rng.standard_normal((16, 32, 64)) + 1.0
    t = 0.9
    got = _plan(sbp, box, dtype, 2, frame=1).solve(to_dev(rho, dtype), t=t).double().cpu().numpy()
    p = _params(box)
    u = O.remap_phase(64, p.Lx, p.Ly, O.shear_offset(p.q, p.Omega, p.Lx, p.Ly, t))
    want = O.remap_y(O.solve_sasha(O.remap_y(as_input(rho, dtype), u, -1.0), p, t, 0.5), u, +1.0)
    assert rel_l2(got, want) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [0, 1])
def test_sasha_batched_and_method_switch(sbp, dtype):
    import torch

    boxes = [W.Box(64, 64, 16, 2.0, 2.0, 1.0), W.Box(48, 24, 12, 2.0, 3.0, 1.5, q=1.0)]
    rng = np.random.default_rng(4)
    plans = [_plan(sbp, b, dtype, 0) for b in boxes]
    rhos = [to_dev(rng.standard_normal((b.nz, b.ny, b.nx)) + 0.5, dtype) for b in boxes]
    outs = [torch.empty_like(r) for r in rhos]
    ts = [0.2, 3.1]
    vgf = [plans[i].solve(rhos[i], t=ts[i]) for i in range(2)]
    sbp.solve_batched(plans, rhos, outs, ts)
    for pl in plans:
        pl.set_option(sbp.Option.METHOD, 1)
    sbp.solve_batched(plans, rhos, outs, ts)
    torch.cuda.synchronize()
    for i in range(2):
        assert torch.equal(outs[i], plans[i].solve(rhos[i], t=ts[i]))
        want = O.solve_sasha(as_input(rhos[i].double().cpu().numpy(), dtype), _params(boxes[i]), ts[i])
        assert rel_l2(outs[i].double().cpu().numpy(), want) <= TOL[dtype]
    plans[0].set_option(sbp.Option.METHOD, 0)
    assert torch.equal(plans[0].solve(rhos[0], t=ts[0]), vgf[0])


def test_sasha_option_errors(sbp):
    box = W.Box(32, 32, 32, 2.0, 2.0, 1.0)  # nz = 32: the fourfold-padding kernel exists
    plan = _plan(sbp, box, 0, 0)
    with pytest.raises(sbp.SbpError) as e:
        plan.set_option(sbp.Option.METHOD, 3)
    assert e.value.status == sbp.Status.INVALID_ARG
    plan.set_option(sbp.Option.TRUNCATION, 1.1)
    with pytest.raises(sbp.SbpError) as e:
        plan.set_option(sbp.Option.METHOD, 1)
    assert e.value.status == sbp.Status.UNSUPPORTED_SIZE
    plan.set_option(sbp.Option.TRUNCATION, 1.0)
    plan.set_option(sbp.Option.METHOD, 2)
    with pytest.raises(sbp.SbpError) as e:
        plan.set_option(sbp.Option.TRUNCATION, 1.1)
    assert e.value.status == sbp.Status.UNSUPPORTED_SIZE
    with pytest.raises(sbp.SbpError) as e:
        plan.run_stage(sbp.Stage.GREEN_FILL, None, plan.new_spectrum())
    assert e.value.status == sbp.Status.INVALID_ARG
