"""Helpers shared by the GPU parity tests (data movement only)."""

import numpy as np

TOL = {0: 1e-12, 1: 2e-5}        # end-to-end rel-L2 bars: FP64, FP32
STAGE_TOL = {0: 1e-12, 1: 2e-6}  # single stages (one or two FFTs)


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def plane_mean_removed(a):
    """Φ minus its mean over every z-plane: the k ≠ 0 part of the solution."""
    a = np.asarray(a, dtype=np.float64)
    return a - a.mean(axis=(-2, -1), keepdims=True)


def max_rel(a, b):
    """max |a - b| relative to max |b|."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def parity(got, want, tol):
    """The three end-to-end bars: rel-L2 of Φ, rel-L2 of Φ without its plane
    means (the k = 0 mode dominates ‖Φ‖ for stratified densities and would hide
    errors in the rest), and the max-norm error relative to ‖Φ‖∞.  Returns
    the three errors; asserts each against its bar.

    rel-L2 and max-norm: ≤ tol.  Without the plane means: ≤ max(tol, floor)
    with floor = 4 log2(N) ε ‖Φ‖ / ‖Φ without plane means‖, ε the unit
    roundoff of the arithmetic (2^-52 for the FP64 bar, 2^-23 for FP32): the
    transforms carry the plane means too, and their rounding (about
    log2(N) ε ‖Φ‖) lands in every mode, so a field whose fluctuations are tiny
    next to its mean cannot have them more accurate than that."""
    want = np.asarray(want, dtype=np.float64)
    got = np.asarray(got, dtype=np.float64)
    e1 = rel_l2(got, want)
    wk = plane_mean_removed(want)
    e2 = rel_l2(plane_mean_removed(got), wk)
    e3 = max_rel(got, want)
    eps = 2.0 ** -52 if tol < 1e-9 else 2.0 ** -23
    ratio = float(np.linalg.norm(want.ravel()) / max(np.linalg.norm(wk.ravel()), 1e-300))
    tol_k = max(tol, 4.0 * np.log2(want.size) * eps * ratio)
    assert e1 <= tol and e2 <= tol_k and e3 <= tol, (e1, e2, e3, tol, tol_k)
    return e1, e2, e3


def torch_dtype(dtype):
    import torch

    return torch.float64 if int(dtype) == 0 else torch.float32


def np_real_dtype(dtype):
    return np.float64 if int(dtype) == 0 else np.float32


def to_dev(x, dtype):
    import torch

    return torch.tensor(np.ascontiguousarray(x), dtype=torch_dtype(dtype), device="cuda")


def as_input(x, dtype):
    """The input exactly as the device sees it, widened back to float64."""
    return np.asarray(x, dtype=np_real_dtype(dtype)).astype(np.float64)


def spec_to_np(spec, h):
    s = spec.double().cpu().numpy()
    return (s[..., 0] + 1j * s[..., 1])[..., :h]


def np_to_spec(X, pitch, dtype):
    import torch

    nz, ny, h = X.shape
    out = np.zeros((nz, ny, pitch, 2))
    out[..., :h, 0] = X.real
    out[..., :h, 1] = X.imag
    return torch.tensor(out, dtype=torch_dtype(dtype), device="cuda")


def spec_input(X, dtype):
    """A complex spectrum rounded as the device stores it."""
    if int(dtype) == 0:
        return np.asarray(X, dtype=np.complex128)
    return (X.real.astype(np.float32).astype(np.float64) + 1j * X.imag.astype(np.float32).astype(np.float64))


def same_as_a_single_solve(sbp, plan, rho, t, out):
    """True when a batched box's output equals, bit for bit, a single solve of
    the same plan on one of the two schedules (the batched executor picks the
    grouped three sweeps or the five passes per group of boxes by timing)."""
    import torch

    one = plan.solve(rho, t=t)
    if torch.equal(out, one):
        return True
    other = sbp.Plan(plan.nx, plan.ny, plan.nz, plan.Lx, plan.Ly, plan.Lz, q=plan.q, Omega=plan.Omega, G=plan.G,
                     dtype=plan.dtype)
    other.set_option(sbp.Option.SCHEDULE, 1 if plan.schedule_is_sweep() else 0)
    return bool(torch.equal(out, other.solve(rho, t=t)))
