"""Guard bands around every buffer a call touches.

This pool offers no device memory checker, so out-of-bounds writes and
stray reads are caught the plain way: each input and output sits inside a
larger allocation whose margins hold a canary bit pattern (a NaN with a
payload).  After the call the margins must be bit for bit unchanged, an
out-of-place call must leave its input unchanged, and the output must be
finite (a read from a margin would bring a NaN in).  Covered: the three
sweeps and the five passes of every shape the sweeps are built for, shapes
with radix-3 factors and odd nz, both dtypes, the physical frame, α = 1.1
padding, SASHA, the batched executor (grouped sweeps, per-box kernels, an
in-place box), the allocation-free entry point, the force and the ghost fill.
"""

import numpy as np
import pytest

from gpu_helpers import np_real_dtype

pytestmark = pytest.mark.gpu

MARGIN = 4096  # elements on each side (16 or 32 KB)
CANARY = {4: 0x7FC0A5A5, 8: 0x7FF8A5A5A5A5A5A5}  # quiet NaNs with a payload


@pytest.fixture(scope="module")
def sbp():
    from paper_2510_10070_gb300 import sbp as S

    S.lib()
    return S


def _int_dtype(torch, size):
    return torch.int32 if size == 4 else torch.int64


class Guarded:
    """A tensor of `shape` and float dtype inside a canary-filled allocation."""

    def __init__(self, torch, shape, dtype, fill=None):
        size = torch.empty((), dtype=dtype).element_size()
        n = int(np.prod(shape))
        self.raw = torch.full((n + 2 * MARGIN,), CANARY[size], dtype=_int_dtype(torch, size), device="cuda")
        self.size = size
        self.n = n
        self.t = self.raw.view(dtype)[MARGIN:MARGIN + n].view(shape)
        if fill is not None:
            self.t.copy_(fill)

    def margins_intact(self):
        c = CANARY[self.size]
        return bool((self.raw[:MARGIN] == c).all()) and bool((self.raw[MARGIN + self.n:] == c).all())


def _density(nx, ny, nz, dtype, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((nz, ny, nx)) + 1.5).astype(np_real_dtype(dtype))


def _plan(sbp, nx, ny, nz, dtype, opts=()):
    p = sbp.Plan(nx, ny, nz, 8.0, 6.0, 4.0, q=1.5, Omega=1.0, dtype=dtype)
    for o, v in opts:
        p.set_option(o, v)
    return p


def _check_single(sbp, plan, dtype, t=1.7, seed=0):
    import torch

    nx, ny, nz = plan.nx, plan.ny, plan.nz
    rho_np = _density(nx, ny, nz, dtype, seed)
    td = torch.float64 if dtype == 0 else torch.float32
    rho = Guarded(torch, (nz, ny, nx), td, torch.from_numpy(rho_np).cuda())
    phi = Guarded(torch, (nz, ny, nx), td)
    plan.solve(rho.t, phi.t, t=t)
    torch.cuda.synchronize()
    assert rho.margins_intact() and phi.margins_intact()
    assert torch.equal(rho.t.cpu(), torch.from_numpy(rho_np))
    assert bool(torch.isfinite(phi.t).all())
    return phi.t


SWEEP_SHAPES = [(32, 32, 32), (64, 64, 32), (64, 64, 64), (128, 128, 64), (128, 128, 128), (192, 192, 96),
                (256, 256, 64), (256, 256, 128)]


@pytest.mark.parametrize("shape", SWEEP_SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("schedule", [2, 1], ids=["sweeps", "five"])
def test_fp32_solve_stays_in_its_buffers(sbp, shape, schedule):
    plan = _plan(sbp, *shape, 1, ((sbp.Option.SCHEDULE, schedule),))
    _check_single(sbp, plan, 1)


@pytest.mark.parametrize("shape", [(6, 4, 3), (12, 24, 6), (48, 24, 12), (96, 64, 48)],
                         ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("dtype", [1, 0], ids=["f32", "f64"])
def test_radix3_and_small_shapes_stay_in_their_buffers(sbp, shape, dtype):
    _check_single(sbp, _plan(sbp, *shape, dtype), dtype)


@pytest.mark.parametrize("dtype", [1, 0], ids=["f32", "f64"])
@pytest.mark.parametrize("variant", ["physical_frame", "alpha_1.1", "sasha"])
def test_variants_stay_in_their_buffers(sbp, dtype, variant):
    O_ = sbp.Option
    opts = {"physical_frame": ((O_.FRAME, 1),), "alpha_1.1": ((O_.TRUNCATION, 1.1),),
            "sasha": ((O_.METHOD, 2),)}[variant]
    _check_single(sbp, _plan(sbp, 64, 64, 32, dtype, opts), dtype)


def test_batched_solve_stays_in_its_buffers(sbp):
    import torch

    shapes = [(64, 64, 64), (128, 128, 64), (64, 64, 64), (32, 32, 32), (48, 48, 24), (256, 256, 64)]
    plans = [_plan(sbp, *s, 1) for s in shapes]
    rho_np = [_density(*s, 1, seed=i) for i, s in enumerate(shapes)]
    rhos = [Guarded(torch, r.shape, torch.float32, torch.from_numpy(r).cuda()) for r in rho_np]
    phis = [Guarded(torch, r.shape, torch.float32) for r in rho_np]
    outs = [p.t for p in phis]
    outs[2] = rhos[2].t  # one box in place
    ts = [0.3 * i for i in range(len(shapes))]
    for _ in range(2):  # the first call tunes (temporary outputs), the second replays the graph
        for i, r in enumerate(rho_np):
            rhos[i].t.copy_(torch.from_numpy(r))
        sbp.solve_batched(plans, [g.t for g in rhos], outs, ts)
        torch.cuda.synchronize()
        for i in range(len(shapes)):
            assert rhos[i].margins_intact() and phis[i].margins_intact(), i
            assert bool(torch.isfinite(outs[i]).all()), i
            if i != 2:
                assert torch.equal(rhos[i].t.cpu(), torch.from_numpy(rho_np[i])), i


def test_noalloc_solve_stays_in_its_buffers(sbp):
    import torch

    r = _density(64, 64, 64, 1, seed=3)
    rho = Guarded(torch, r.shape, torch.float32, torch.from_numpy(r).cuda())
    phi = Guarded(torch, r.shape, torch.float32)
    sbp.solve_noalloc(rho.t, phi.t, 8.0, 6.0, 4.0, t=0.9)
    torch.cuda.synchronize()
    assert rho.margins_intact() and phi.margins_intact()
    assert torch.equal(rho.t.cpu(), torch.from_numpy(r))
    assert bool(torch.isfinite(phi.t).all())


@pytest.mark.parametrize("dtype", [1, 0], ids=["f32", "f64"])
def test_force_and_ghosts_stay_in_their_buffers(sbp, dtype):
    import torch

    plan = _plan(sbp, 64, 64, 32, dtype)
    td = torch.float64 if dtype == 0 else torch.float32
    phi_np = _density(64, 64, 32, dtype, seed=5)
    phi = Guarded(torch, phi_np.shape, td, torch.from_numpy(phi_np).cuda())
    g = Guarded(torch, (3,) + phi_np.shape, td)
    plan.force(phi.t, t=1.1, out=g.t)
    ng = 2
    gh = Guarded(torch, (32 + 2 * ng, 64, 64), td)
    plan.fill_ghosts(phi.t, ng, out=gh.t)
    torch.cuda.synchronize()
    assert phi.margins_intact() and g.margins_intact() and gh.margins_intact()
    assert torch.equal(phi.t.cpu(), torch.from_numpy(phi_np))
    assert bool(torch.isfinite(g.t).all()) and bool(torch.isfinite(gh.t).all())
