"""Physical-frame solves on the GPU (SBP_OPT_FRAME = 1) against the oracle.

The plan maps ρ to the periodic frame (Sect. 2.1, Fourier interpolation of
each x-column by s·x), solves and maps Φ back, with the mapping fused into the
y transforms.  The oracle composes the same three steps with direct sums.
Bars: rel-L2 ≤ 1e-12 (FP64), ≤ 2e-5 (FP32).
"""

import numpy as np
import pytest

import analytic as A
import oracle as O
from gpu_helpers import TOL, as_input, rel_l2, to_dev
from paper_2510_10070_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sbp():
    from paper_2510_10070_gb300 import sbp as S

    S.lib()
    return S


def _plan(sbp, box, dtype, frame=1, alpha=None):
    plan = sbp.Plan(box.nx, box.ny, box.nz, box.Lx, box.Ly, box.Lz, q=box.q, Omega=box.Omega, G=box.G,
                    dtype=dtype)
    plan.set_option(sbp.Option.FRAME, frame)
    if alpha is not None:
        plan.set_option(sbp.Option.TRUNCATION, alpha)
    return plan


def _params(box, alpha=1.0):
    return O.SolveParams(box.Lx, box.Ly, box.Lz, q=box.q, Omega=box.Omega, G=box.G,
                         pad=2 if alpha == 1.0 else 4, alpha=alpha)


SHAPES = [(32, 32, 16), (64, 32, 12), (32, 96, 8), (96, 64, 24), (128, 32, 32), (32, 192, 6), (192, 64, 6),
          (256, 32, 4), (32, 256, 48)]


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("shape", SHAPES)
def test_physical_frame_parity(sbp, shape, dtype):
    nx, ny, nz = shape
    box = W.Box(nx, ny, nz, 2.0, 3.0, 1.5, q=1.5)
    rng = np.random.default_rng(nx + 3 * ny + nz)
    rho = rng.standard_normal((nz, ny, nx)) + 0.5
    t = 0.77
    got = _plan(sbp, box, dtype).solve(to_dev(rho, dtype), t=t).double().cpu().numpy()
    want = O.solve_physical(as_input(rho, dtype), _params(box), t)
    assert rel_l2(got, want) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("t", [0.0, 0.31, -2.6, 11.9])
def test_physical_frame_times(sbp, dtype, t):
    box = W.Box(64, 64, 32, 4.0, 4.0, 2.0, q=1.5)
    rho = W.noisy_gaussian(W.Box(64, 64, 32, 4.0, 4.0, 2.0), seed=5)
    got = _plan(sbp, box, dtype).solve(to_dev(rho, dtype), t=t).double().cpu().numpy()
    want = O.solve_physical(as_input(rho, dtype), _params(box), t)
    assert rel_l2(got, want) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [0, 1])
def test_physical_frame_with_paper_truncation(sbp, dtype):
    box = W.Box(64, 32, 32, 2.0, 3.0, 1.5, q=1.5)
    rng = np.random.default_rng(8)
    rho = rng.standard_normal((32, 32, 64))
    got = _plan(sbp, box, dtype, alpha=1.1).solve(to_dev(rho, dtype), t=1.9).double().cpu().numpy()
    want = O.solve_physical(as_input(rho, dtype), _params(box, 1.1), 1.9)
    assert rel_l2(got, want) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [0, 1])
def test_shear_periodic_mode_closed_form(sbp, dtype):
    # a physical-frame wave cos(k_x x + K_y y) with k_x = K_x + s K_y: the
    # error against the closed form is the z discretisation only
    Lx = Ly = Lz = 4.0
    H = 1.0
    n, nz = 32, 64
    t = 0.7
    box = W.Box(n, n, nz, Lx, Ly, Lz, q=1.5)
    s = O.shear_offset(1.5, 1.0, Lx, Ly, t) / Lx
    Ky = 2.0 * np.pi * 2 / Ly
    kx = 2.0 * np.pi * 1 / Lx + s * Ky
    x = A.cell_centres(n, Lx)
    y = A.cell_centres(n, Ly)
    z = A.cell_centres(nz, Lz)
    horiz = np.cos(kx * x[None, :] + Ky * y[:, None])
    rho = horiz[None] * np.exp(-0.5 * (z / H) ** 2)[:, None, None]
    got = _plan(sbp, box, dtype).solve(to_dev(rho, dtype), t=t).double().cpu().numpy()
    ex = 4.0 * np.pi * horiz[None] * A.mode_profile_paper(z, np.hypot(kx, Ky), H, Lz)[:, None, None]
    want_err = rel_l2(O.solve_physical(rho, _params(box), t), ex)
    assert abs(rel_l2(got, ex) - want_err) < 0.02 * want_err


@pytest.mark.parametrize("dtype", [0, 1])
def test_frame_toggle_batched_and_errors(sbp, dtype):
    import torch

    boxes = [W.Box(64, 64, 16, 2.0, 2.0, 1.0), W.Box(32, 96, 12, 2.0, 3.0, 1.5, q=1.0)]
    rng = np.random.default_rng(21)
    plans = [_plan(sbp, b, dtype, frame=0) for b in boxes]
    rhos = [to_dev(rng.standard_normal((b.nz, b.ny, b.nx)), dtype) for b in boxes]
    outs = [torch.empty_like(r) for r in rhos]
    ts = [0.4, 2.2]
    periodic = [plans[i].solve(rhos[i], t=ts[i]) for i in range(2)]
    sbp.solve_batched(plans, rhos, outs, ts)
    plans[1].set_option(sbp.Option.FRAME, 1)
    sbp.solve_batched(plans, rhos, outs, ts)  # the cached graph must follow the new frame
    torch.cuda.synchronize()
    assert torch.equal(outs[0], periodic[0])
    assert torch.equal(outs[1], plans[1].solve(rhos[1], t=ts[1]))
    want = O.solve_physical(as_input(rhos[1].double().cpu().numpy(), dtype), _params(boxes[1]), ts[1])
    assert rel_l2(outs[1].double().cpu().numpy(), want) <= TOL[dtype]
    # the stage API is the periodic-frame passes
    with pytest.raises(sbp.SbpError) as e:
        plans[1].run_stage(sbp.Stage.X_FORWARD, rhos[1], plans[1].new_spectrum())
    assert e.value.status == sbp.Status.INVALID_ARG
    plans[1].set_option(sbp.Option.FRAME, 0)
    assert torch.equal(plans[1].solve(rhos[1], t=ts[1]), periodic[1])
    # sizes without physical-frame kernels keep the plan as it was
    odd = _plan(sbp, W.Box(48, 32, 8, 2.0, 2.0, 1.0), dtype, frame=0)
    with pytest.raises(sbp.SbpError) as e:
        odd.set_option(sbp.Option.FRAME, 1)
    assert e.value.status == sbp.Status.UNSUPPORTED_SIZE
    with pytest.raises(sbp.SbpError) as e:
        odd.set_option(sbp.Option.FRAME, 2)
    assert e.value.status == sbp.Status.INVALID_ARG
