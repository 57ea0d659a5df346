"""The three-sweep schedule (SBP_OPT_SCHEDULE) against the FP64 oracle and
against the five-pass schedule of the same plan.

The y transform's two radix stages are fused into the passes around the z
pass; the result must meet the FP32 bars of the method (rel-L2, rel-L2
without the plane means, max-norm) on every shape the sweeps are built for,
ragged last column groups included (nx/2 + 1 columns), sheared and not.
"""

import numpy as np
import pytest

import oracle as O
from gpu_helpers import TOL, as_input, parity, rel_l2, same_as_a_single_solve, to_dev
from paper_2510_10070_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SWEEP_SHAPES = [(32, 32, 32), (64, 64, 32), (64, 64, 64), (128, 128, 64), (128, 128, 128), (192, 192, 96),
                (256, 256, 64), (256, 256, 128)]


@pytest.fixture(scope="module")
def sbp():
    from paper_2510_10070_gb300 import sbp as S

    S.lib()
    return S


def _plan(sbp, box, dtype=1, schedule=None):
    p = sbp.Plan(box.nx, box.ny, box.nz, box.Lx, box.Ly, box.Lz, q=box.q, Omega=box.Omega, G=box.G, dtype=dtype)
    if schedule is not None:
        p.set_option(sbp.Option.SCHEDULE, schedule)
    return p


def _params(box):
    return O.SolveParams(box.Lx, box.Ly, box.Lz, q=box.q, Omega=box.Omega, G=box.G)


@pytest.mark.parametrize("shape", SWEEP_SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_sweep_matches_oracle_and_five_passes(sbp, shape):
    nx, ny, nz = shape
    box = W.Box(nx, ny, nz, 8.0, 8.0, 4.0, q=1.5, Omega=1.0, G=0.9)
    three = _plan(sbp, box, schedule=2)
    five = _plan(sbp, box, schedule=1)
    auto = _plan(sbp, box)
    rho = W.lognormal_disc(box, seed=nx + nz, sigma=0.7, dtype=np.float32)
    dev = to_dev(rho, 1)
    small = nx * ny * nz <= 128 * 128 * 64
    for t in (0.0, 1.3, -4.4):
        got = three.solve(dev, t=t).double().cpu().numpy()
        # automatic picks the sweeps for these shapes: the same bits
        assert np.array_equal(auto.solve(dev, t=t).double().cpu().numpy(), got)
        ref5 = five.solve(dev, t=t).double().cpu().numpy()
        assert rel_l2(got, ref5) <= 2e-6, t
        if small:
            want = O.solve(as_input(rho, 1), _params(box), t)
            parity(got, want, TOL[1])


@pytest.mark.parametrize("shape", [(64, 64, 64), (256, 256, 128)], ids=lambda s: "x".join(map(str, s)))
def test_sweep_sampled_against_oracle(sbp, shape):
    # the largest sweep shape at cells the oracle computes one by one
    nx, ny, nz = shape
    box = W.Box(nx, ny, nz, 8.0, 8.0, 4.0)
    rho = W.lognormal_disc(box, seed=7, sigma=0.7, dtype=np.float32)
    plan = _plan(sbp, box, schedule=2)
    got = plan.solve(to_dev(rho, 1), t=2.3).double().cpu().numpy()
    rng = np.random.default_rng(3)
    pts = [(0, 0, 0), (nz - 1, ny - 1, nx - 1), (nz // 2, ny // 2, nx // 2)]
    pts += [(int(rng.integers(nz)), int(rng.integers(ny)), int(rng.integers(nx))) for _ in range(9)]
    want = O.solve_at(as_input(rho, 1), _params(box), 2.3, pts)
    assert rel_l2(np.array([got[p] for p in pts]), want) <= TOL[1]


def test_sweep_in_place_and_batched(sbp):
    import torch

    boxes = [W.Box(64, 64, 64, 8.0, 8.0, 4.0), W.Box(128, 128, 64, 8.0, 8.0, 4.0, q=1.0),
             W.Box(192, 192, 96, 8.0, 8.0, 4.0), W.Box(32, 32, 32, 4.0, 4.0, 4.0)]
    plans = [_plan(sbp, b) for b in boxes]
    rng = np.random.default_rng(41)
    rhos = [to_dev(rng.standard_normal((b.nz, b.ny, b.nx)) + 1.0, 1) for b in boxes]
    ts = [0.3, 6.1, -2.2, 9.9]
    singles = [p.solve(r, t=t) for p, r, t in zip(plans, rhos, ts)]
    outs = [torch.empty_like(r) for r in rhos]
    sbp.solve_batched(plans, rhos, outs, ts)
    buf = rhos[2].clone()
    plans[2].solve(buf, phi=buf, t=ts[2])
    torch.cuda.synchronize()
    for i in range(len(boxes)):
        assert same_as_a_single_solve(sbp, plans[i], rhos[i], ts[i], outs[i]), i
    assert torch.equal(buf, singles[2])


@pytest.mark.parametrize("schedule", ["2", "1"])
def test_grouped_sweeps_many_boxes(sbp, monkeypatch, schedule):
    # Several boxes per shape, grouped into one launch per sweep (or forced to
    # per-box five-pass kernels): each box equals its own single solve on the
    # same schedule, and the grouped graph launches three kernels per shape.
    import torch

    monkeypatch.setenv("SBP_BATCH_SCHEDULE", schedule)
    shapes = [(64, 64, 64)] * 5 + [(128, 128, 64)] * 3 + [(32, 32, 32)] * 2
    boxes = [W.Box(nx, ny, nz, 8.0, 8.0, 4.0, q=1.5 if i % 2 else 1.0) for i, (nx, ny, nz) in enumerate(shapes)]
    plans = [_plan(sbp, b) for b in boxes]
    rng = np.random.default_rng(55)
    rho_np = [rng.standard_normal((b.nz, b.ny, b.nx)) + 0.7 for b in boxes]
    rhos = [to_dev(r, 1) for r in rho_np]
    outs = [torch.empty_like(r) for r in rhos]
    ts = list(rng.uniform(-5.0, 5.0, len(boxes)))
    for _ in range(2):
        sbp.solve_batched(plans, rhos, outs, ts)
    torch.cuda.synchronize()
    launches, grouped = sbp.batch_info(plans, rhos, outs)
    if schedule == "2":
        assert (launches, grouped) == (9, len(boxes))
    else:
        assert grouped == 0 and launches > 9
    for i, p in enumerate(plans):
        assert same_as_a_single_solve(sbp, p, rhos[i], ts[i], outs[i]), i
    want = O.solve(as_input(rho_np[6], 1), _params(boxes[6]), ts[6])
    parity(outs[6].double().cpu().numpy(), want, TOL[1])
    if schedule == "2":
        # the three sweeps of one group run alone through sbp_batch_run_stage
        # give that group's batched result again, bit for bit
        before = [o.clone() for o in outs]
        for o in outs[:5]:
            o.zero_()
        for stage in (sbp.Stage.SWEEP_FORWARD, sbp.Stage.SWEEP_MIDDLE, sbp.Stage.SWEEP_INVERSE):
            sbp.batch_run_stage(plans, rhos, outs, (64, 64, 64), stage)
        torch.cuda.synchronize()
        for i in range(len(plans)):
            assert torch.equal(outs[i], before[i]), i
        with pytest.raises(sbp.SbpError):
            sbp.batch_run_stage(plans, rhos, outs, (16, 16, 16), sbp.Stage.SWEEP_MIDDLE)


def test_schedule_option_rules(sbp):
    box = W.Box(48, 24, 12, 2.0, 3.0, 1.5)
    p = _plan(sbp, box)
    with pytest.raises(sbp.SbpError) as err:
        p.set_option(sbp.Option.SCHEDULE, 2)  # no sweep kernels for this shape
    assert err.value.status == sbp.Status.UNSUPPORTED_SIZE
    with pytest.raises(sbp.SbpError):
        p.set_option(sbp.Option.SCHEDULE, 3)
    q = _plan(sbp, W.Box(64, 64, 64, 8.0, 8.0, 4.0), dtype=0)
    with pytest.raises(sbp.SbpError):
        q.set_option(sbp.Option.SCHEDULE, 2)  # FP64 plans run five passes
    # the sweeps give way to the physical frame and come back after it
    r = _plan(sbp, W.Box(64, 64, 64, 8.0, 8.0, 4.0), schedule=2)
    rho = to_dev(np.random.default_rng(2).standard_normal((64, 64, 64)), 1)
    a = r.solve(rho, t=0.7).double().cpu().numpy()
    r.set_option(sbp.Option.FRAME, 1)
    r.set_option(sbp.Option.FRAME, 0)
    b = r.solve(rho, t=0.7).double().cpu().numpy()
    assert rel_l2(a, b) <= 2e-6


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("shape", [(32, 16, 16), (64, 64, 64)], ids=lambda s: "x".join(map(str, s)))
def test_nyquist_planes_sheared(sbp, shape, dtype):
    # A density that lives on the Nyquist planes a = -nx/2 and b = -ny/2, where
    # a sheared box has k(a, b) != k(-a, -b) and the solve takes the real
    # part (the partner-averaged Green's function): the end-to-end check of
    # that reading, on both schedules for FP32.
    nx, ny, nz = shape
    box = W.Box(nx, ny, nz, 4.0, 6.0, 3.0, q=1.5)
    x = np.arange(nx)
    y = np.arange(ny)
    z = W.cell_centres(nz, box.Lz)
    rng = np.random.default_rng(nx + dtype)
    prof = np.exp(-0.5 * z ** 2)[:, None, None]
    rho = prof * ((-1.0) ** x[None, None, :] * (1.0 + 0.3 * np.cos(2 * np.pi * 3 * y / ny))[None, :, None]
                  + (-1.0) ** y[None, :, None] * np.cos(2 * np.pi * 5 * x / nx)[None, None, :]
                  + 0.2 * (-1.0) ** (x[None, None, :] + y[None, :, None]))
    rho = rho + 0.05 * rng.standard_normal(rho.shape)
    for t in (0.9, 3.7):
        want = O.solve(as_input(rho, dtype), _params(box), t)
        schedules = (None,) if dtype == 0 else (1, None)
        for sch in schedules:
            plan = _plan(sbp, box, dtype, schedule=sch)
            got = plan.solve(to_dev(rho, dtype), t=t).double().cpu().numpy()
            parity(got, want, TOL[dtype])


@pytest.mark.parametrize("shape", [(128, 128, 64), (256, 256, 64)], ids=["table", "green_in_middle"])
def test_sweep_stages_compose_to_the_solve(sbp, shape):
    # 128x128x64: the forward sweep fills the Green's table; 256x256x64: the
    # middle sweep evaluates the Green's parameters at t itself
    import torch

    nx, ny, nz = shape
    box = W.Box(nx, ny, nz, 8.0, 8.0, 4.0)
    plan = _plan(sbp, box, schedule=2)
    rho = to_dev(np.random.default_rng(8).standard_normal((nz, ny, nx)) + 1.0, 1)
    want = plan.solve(rho, t=3.1)
    out = torch.empty_like(rho)
    plan.run_stage(sbp.Stage.SWEEP_FORWARD, rho, None, t=3.1)
    plan.run_stage(sbp.Stage.SWEEP_MIDDLE, None, None, t=3.1)
    plan.run_stage(sbp.Stage.SWEEP_INVERSE, None, out, t=3.1)
    torch.cuda.synchronize()
    assert torch.equal(out, want)
    five = _plan(sbp, box, schedule=1)
    with pytest.raises(sbp.SbpError):
        five.run_stage(sbp.Stage.SWEEP_MIDDLE, None, None)


_TUNE_SCRIPT = """
import sys
sys.path.insert(0, {root!r})
import torch
from paper_2510_10070_gb300 import sbp
shapes = [(64, 64, 64)] * 3 + [(128, 128, 64)] * 2
plans = [sbp.Plan(nx, ny, nz, 8.0, 8.0, 4.0, dtype=1) for nx, ny, nz in shapes]
rhos = [torch.rand((nz, ny, nx), device="cuda") for nx, ny, nz in shapes]
outs = [torch.empty_like(r) for r in rhos]
sbp.solve_batched(plans, rhos, outs, [0.1 * i for i in range(len(plans))])
torch.cuda.synchronize()
print("launches", sbp.batch_info(plans, rhos, outs)[0])
"""


def test_tuning_choice_is_saved_and_reloaded(tmp_path):
    # The batched executor's first call times its candidates and appends the
    # choice to the SBP_TUNE_CACHE file; a later process with the same batch
    # shapes on the same GPU reads it and skips the timing (SBP_TUNE_LOG shows
    # which happened).
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "batch.py"
    script.write_text(_TUNE_SCRIPT.format(root=root))
    cache = tmp_path / "tune.txt"
    env = dict(os.environ, SBP_TUNE_CACHE=str(cache), SBP_TUNE_LOG="1")
    for k in ("SBP_BATCH_SCHEDULE", "SBP_BATCH_BRANCHES", "SBP_BATCH_CHUNK"):
        env.pop(k, None)
    first = subprocess.run([sys.executable, str(script)], env=env, capture_output=True, text=True, timeout=300)
    assert first.returncode == 0, first.stderr
    assert "[sbp tune] choice" in first.stderr
    lines = cache.read_text().strip().splitlines()
    assert len(lines) == 1 and "\t" in lines[0]
    second = subprocess.run([sys.executable, str(script)], env=env, capture_output=True, text=True, timeout=300)
    assert second.returncode == 0, second.stderr
    assert "[sbp tune]" not in second.stderr  # no timing: the saved choice was used
    assert first.stdout.split()[-1] == second.stdout.split()[-1]
    assert len(cache.read_text().strip().splitlines()) == 1
