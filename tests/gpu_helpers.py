"""Helpers shared by the GPU parity tests (data movement only)."""

import numpy as np

TOL = {0: 1e-12, 1: 2e-5}        # end-to-end rel-L2 bars: FP64, FP32
STAGE_TOL = {0: 1e-12, 1: 2e-6}  # single stages (one or two FFTs)


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


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
