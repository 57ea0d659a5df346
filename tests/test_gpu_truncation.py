"""The paper's own vertical truncation on the GPU: L = α·Lz with 4·nz padding.

Sect. 2.3 takes α = 1.1 and pads the vertical transform fourfold; the plan
option SBP_OPT_TRUNCATION selects it.  Parity bars are the end-to-end ones
(rel-L2 ≤ 1e-12 FP64, ≤ 2e-5 FP32) against the oracle run with the same
(pad, α).
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


def _plan(sbp, box, dtype, alpha=None):
    plan = sbp.Plan(box.nx, box.ny, box.nz, box.Lx, box.Ly, box.Lz, q=box.q, Omega=box.Omega, G=box.G,
                    dtype=dtype)
    if alpha is not None:
        plan.set_option(sbp.Option.TRUNCATION, alpha)
    return plan


def _params(box, alpha):
    pad = 2 if alpha == 1.0 else 4
    return O.SolveParams(box.Lx, box.Ly, box.Lz, q=box.q, Omega=box.Omega, G=box.G, pad=pad, alpha=alpha)


CASES = [  # (nx, ny, nz), dtypes
    ((32, 32, 32), (0, 1)),
    ((48, 24, 64), (0, 1)),
    ((24, 16, 128), (0, 1)),
    ((12, 8, 256), (0, 1)),
    ((8, 6, 512), (1,)),
]


@pytest.mark.parametrize("alpha", [1.1, 2.0, 3.0])
@pytest.mark.parametrize("shape,dtype", [(s, d) for s, ds in CASES for d in ds])
def test_truncation_parity(sbp, shape, dtype, alpha):
    nx, ny, nz = shape
    box = W.Box(nx, ny, nz, 2.0, 3.0, 1.5, q=1.5)
    rng = np.random.default_rng(nz + nx)
    rho = rng.standard_normal((nz, ny, nx)) + 0.3
    plan = _plan(sbp, box, dtype, alpha)
    got = plan.solve(to_dev(rho, dtype), t=0.83).double().cpu().numpy()
    want = O.solve(as_input(rho, dtype), _params(box, alpha), 0.83)
    assert rel_l2(got, want) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [0, 1])
def test_paper_3d_mode_alpha_11(sbp, dtype):
    # Sect. 3.2 mixed-BC mode at 64³ with the paper's α = 1.1 and fourfold
    # padding: equal to the oracle, and as accurate as α = 1 with 2·nz.
    L, H, n = 6.0, 1.0, 64
    box = W.Box(n, n, n, L, L, L)
    x = A.cell_centres(n, L)
    k = 2.0 * np.pi / L
    horiz = np.cos(k * x)[None, :] * np.cos(k * x)[:, None]
    z = A.cell_centres(n, L)
    rho = horiz[None] * np.exp(-0.5 * (z / H) ** 2)[:, None, None]
    got = _plan(sbp, box, dtype, 1.1).solve(to_dev(rho, dtype), t=0.0).double().cpu().numpy()
    want = O.solve(as_input(rho, dtype), _params(box, 1.1), 0.0)
    assert rel_l2(got, want) <= TOL[dtype]
    ex = 4.0 * np.pi * horiz[None] * A.mode_profile_paper(z, np.sqrt(2.0) * k, H, L)[:, None, None]
    assert 8e-6 < rel_l2(got, ex) < 1.1e-5


@pytest.mark.parametrize("dtype", [0, 1])
def test_truncation_option_errors_keep_the_plan(sbp, dtype):
    box = W.Box(24, 16, 48, 2.0, 3.0, 1.5)  # nz = 48: no fourfold-padding kernel
    rng = np.random.default_rng(3)
    rho = to_dev(rng.standard_normal((48, 16, 24)), dtype)
    plan = _plan(sbp, box, dtype)
    before = plan.solve(rho, t=0.4)
    for bad in (0.5, 0.999, 3.01, float("inf")):
        with pytest.raises(sbp.SbpError) as e:
            plan.set_option(sbp.Option.TRUNCATION, bad)
        assert e.value.status == sbp.Status.INVALID_ARG
    with pytest.raises(sbp.SbpError) as e:
        plan.set_option(sbp.Option.TRUNCATION, 1.1)
    assert e.value.status == sbp.Status.UNSUPPORTED_SIZE
    import torch

    assert torch.equal(plan.solve(rho, t=0.4), before)


@pytest.mark.parametrize("dtype", [0, 1])
def test_truncation_toggles_back_and_pins_z_variant(sbp, dtype):
    import torch

    box = W.Box(32, 16, 64, 2.0, 3.0, 1.5)
    rng = np.random.default_rng(5)
    rho = to_dev(rng.standard_normal((64, 16, 32)), dtype)
    plan = _plan(sbp, box, dtype)
    ref = plan.solve(rho, t=1.7)
    plan.set_option(sbp.Option.TRUNCATION, 1.1)
    with pytest.raises(sbp.SbpError) as e:
        plan.set_option(sbp.Option.Z_VARIANT, 3)
    assert e.value.status == sbp.Status.UNSUPPORTED_SIZE
    paper = plan.solve(rho, t=1.7)
    assert not torch.equal(paper, ref)
    plan.set_option(sbp.Option.TRUNCATION, 1.0)
    assert torch.equal(plan.solve(rho, t=1.7), ref)


@pytest.mark.parametrize("dtype", [0, 1])
def test_batched_graph_follows_option_change(sbp, dtype):
    # a captured batch graph holds the plan's kernels: changing the
    # truncation must not replay the old one
    import torch

    boxes = [W.Box(32, 32, 32, 2.0, 2.0, 1.0), W.Box(48, 24, 64, 2.0, 3.0, 1.5, q=1.0)]
    rng = np.random.default_rng(11)
    plans = [_plan(sbp, b, dtype) for b in boxes]
    rhos = [to_dev(rng.standard_normal((b.nz, b.ny, b.nx)), dtype) for b in boxes]
    outs = [torch.empty_like(r) for r in rhos]
    ts = [0.2, -1.3]
    sbp.solve_batched(plans, rhos, outs, ts)
    plans[1].set_option(sbp.Option.TRUNCATION, 1.1)
    sbp.solve_batched(plans, rhos, outs, ts)
    torch.cuda.synchronize()
    for i in range(2):
        assert torch.equal(outs[i], plans[i].solve(rhos[i], t=ts[i]))
    want = O.solve(as_input(rhos[1].double().cpu().numpy(), dtype), _params(boxes[1], 1.1), ts[1])
    assert rel_l2(outs[1].double().cpu().numpy(), want) <= TOL[dtype]
