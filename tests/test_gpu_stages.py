"""Stage-level parity of the CUDA passes against the oracle's direct sums.

Each stage runs alone through sbp_run_stage on seeded inputs that both sides
receive; the shapes cover every elements-per-thread variant (lengths 2^a and
3·2^a from 2 to 2048), ragged last tiles of the nx/2+1 columns and several
blocks per pass.
"""

import numpy as np
import pytest

import oracle as O
from gpu_helpers import STAGE_TOL, as_input, np_to_spec, rel_l2, spec_input, spec_to_np, to_dev

pytestmark = pytest.mark.gpu

SHAPES = [
    (4, 4, 2), (6, 6, 3), (8, 12, 6), (12, 8, 4), (16, 16, 8), (24, 48, 12), (48, 24, 24), (64, 32, 16),
    (96, 64, 48), (256, 16, 32), (32, 256, 8), (16, 8, 256), (384, 6, 4), (6, 384, 6), (1024, 4, 2),
    (2048, 4, 2), (4, 2048, 2), (4, 4, 1536), (8, 4, 2048), (192, 96, 96), (768, 8, 12),
]
DTYPES = [0, 1]
L = (2.0, 3.0, 1.5)


@pytest.fixture(scope="module")
def sbp():
    from paper_2510_10070_gb300 import sbp as S

    S.lib()
    return S


def _plan(sbp, shape, dtype, q=1.5, Omega=1.0, G=0.7):
    nx, ny, nz = shape
    return sbp.Plan(nx, ny, nz, *L, q=q, Omega=Omega, G=G, dtype=dtype)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("shape", SHAPES)
def test_x_forward(sbp, shape, dtype):
    nx, ny, nz = shape
    plan = _plan(sbp, shape, dtype)
    rho = np.random.default_rng(1).standard_normal((nz, ny, nx))
    spec = plan.new_spectrum()
    plan.run_stage(sbp.Stage.X_FORWARD, to_dev(rho, dtype), spec)
    got = spec_to_np(spec, nx // 2 + 1)
    want = O.dft_x(as_input(rho, dtype))
    assert rel_l2(got, want) <= STAGE_TOL[dtype]


@pytest.mark.parametrize("inverse", [False, True])
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("shape", SHAPES)
def test_y_pass(sbp, shape, dtype, inverse):
    nx, ny, nz = shape
    h = nx // 2 + 1
    plan = _plan(sbp, shape, dtype)
    rng = np.random.default_rng(2)
    X = rng.standard_normal((nz, ny, h)) + 1j * rng.standard_normal((nz, ny, h))
    spec = np_to_spec(X, plan.spectrum_pitch, dtype)
    stage = sbp.Stage.Y_INVERSE if inverse else sbp.Stage.Y_FORWARD
    plan.run_stage(stage, spec, spec)
    want = O.dft_y(spec_input(X, dtype), +1.0 if inverse else -1.0)
    assert rel_l2(spec_to_np(spec, h), want) <= STAGE_TOL[dtype]


@pytest.mark.parametrize("t", [0.0, 0.7, -3.3])
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("shape", SHAPES)
def test_z_convolve(sbp, shape, dtype, t):
    nx, ny, nz = shape
    h = nx // 2 + 1
    G = 0.7
    plan = _plan(sbp, shape, dtype, G=G)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((nz, ny, h)) + 1j * rng.standard_normal((nz, ny, h))
    spec = np_to_spec(X, plan.spectrum_pitch, dtype)
    plan.run_stage(sbp.Stage.GREEN_FILL, None, spec, t=t)
    plan.run_stage(sbp.Stage.Z_CONVOLVE, spec, spec, t=t)
    p = O.SolveParams(*L, q=1.5, Omega=1.0, G=G)
    c = O.vertical_kernel(O.green_eff(nx, ny, nz, p, t)[:, :h], nz)
    want = O.vertical_convolve(c, spec_input(X, dtype)) * (4.0 * np.pi * G / (nx * ny))
    if dtype == 1:
        want[:, 0, 0] = 0.0  # FP32: the (0,0) column belongs to the FP64 mean-mode path
    assert rel_l2(spec_to_np(spec, h), want) <= STAGE_TOL[dtype]


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("shape", [(8, 6, 64), (48, 24, 128), (16, 8, 256), (8, 4, 512), (6, 4, 96)])
def test_z_convolve_variants(sbp, shape, variant):
    # The alternative z-pass kernels give the default kernel's result (FP32).
    nx, ny, nz = shape
    h = nx // 2 + 1
    plan = _plan(sbp, shape, 1)
    try:
        plan.set_option(sbp.Option.Z_VARIANT, variant)
    except sbp.SbpError as err:
        assert err.status == sbp.Status.UNSUPPORTED_SIZE
        pytest.skip(f"variant {variant} not built for nz={nz}")
    rng = np.random.default_rng(13)
    X = rng.standard_normal((nz, ny, h)) + 1j * rng.standard_normal((nz, ny, h))
    spec = np_to_spec(X, plan.spectrum_pitch, 1)
    plan.run_stage(sbp.Stage.GREEN_FILL, None, spec, t=0.9)
    plan.run_stage(sbp.Stage.Z_CONVOLVE, spec, spec, t=0.9)
    p = O.SolveParams(*L, q=1.5, Omega=1.0, G=0.7)
    c = O.vertical_kernel(O.green_eff(nx, ny, nz, p, 0.9)[:, :h], nz)
    want = O.vertical_convolve(c, spec_input(X, 1)) * (4.0 * np.pi * 0.7 / (nx * ny))
    want[:, 0, 0] = 0.0
    assert rel_l2(spec_to_np(spec, h), want) <= STAGE_TOL[1]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("shape", SHAPES)
def test_x_inverse(sbp, shape, dtype):
    nx, ny, nz = shape
    h = nx // 2 + 1
    plan = _plan(sbp, shape, dtype)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((nz, ny, h)) + 1j * rng.standard_normal((nz, ny, h))
    spec = np_to_spec(X, plan.spectrum_pitch, dtype)
    import torch

    out = torch.empty((nz, ny, nx), dtype=plan.torch_dtype, device="cuda")
    plan.run_stage(sbp.Stage.X_INVERSE, spec, out)
    want = O.inverse_dft_x_half(spec_input(X, dtype), nx)
    assert rel_l2(out.double().cpu().numpy(), want) <= STAGE_TOL[dtype]


def _within_f32_ulp(got, want):
    """Every entry is the FP64 value rounded to float, give or take one float ulp."""
    w32 = want.astype(np.float32)
    return bool(np.all(np.abs(got - w32.astype(np.float64)) <= np.spacing(np.abs(w32)).astype(np.float64)))


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("t", [0.0, 0.7, 5.0, -1.1])
@pytest.mark.parametrize("shape", [(8, 6, 4), (96, 64, 8), (256, 256, 2), (192, 128, 2)])
def test_green_table(sbp, shape, t, dtype):
    # The table a solve reads: |k|² and 1 - e^{-kL} of every stored mode and
    # of its Hermitian partner, tabulated in FP64 (an FP32 plan stores them
    # rounded once to float) against the oracle's sheared wave-vectors.
    nx, ny, nz = shape
    h = nx // 2 + 1
    plan = _plan(sbp, shape, dtype)
    import torch

    out = torch.zeros((ny, h, 4), dtype=torch.float64, device="cuda")
    plan.run_stage(sbp.Stage.GREEN_TABLE, None, out, t=t)
    got = out.cpu().numpy()
    s = O.shear_offset(1.5, 1.0, L[0], L[1], t) / L[0]
    k1, k2, is0 = O.mode_wavenumbers(nx, ny, L[0], L[1], s)
    k1, k2, is0 = k1[:, :h], k2[:, :h], is0[:, :h]
    Lz = L[2]
    om1 = np.where(is0, 0.0, -np.expm1(-k1 * Lz))
    om2 = np.where(is0, got[..., 3], -np.expm1(-k2 * Lz))
    if dtype == 0:
        assert np.allclose(got[..., 0], k1 ** 2, rtol=1e-14, atol=1e-14)
        assert np.allclose(got[..., 2], k2 ** 2, rtol=1e-14, atol=1e-14)
        assert np.allclose(got[..., 1], om1, rtol=1e-14, atol=1e-15)
        assert np.allclose(got[..., 3], om2, rtol=1e-14, atol=1e-15)
    else:
        assert _within_f32_ulp(got[..., 0], k1 ** 2)
        assert _within_f32_ulp(got[..., 2], k2 ** 2)
        assert _within_f32_ulp(got[..., 1], om1)
        assert _within_f32_ulp(got[..., 3], om2)
    # the partner differs only on the Nyquist planes, and only when sheared
    differ = np.abs(got[..., 0] - got[..., 2]) > 0
    if s == 0.0:
        assert not differ.any()
    else:
        rows = np.zeros((ny, h), bool)
        rows[ny // 2, :] = True
        rows[:, nx // 2] = True
        assert not differ[~rows].any()
