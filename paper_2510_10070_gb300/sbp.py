"""Thin ctypes binding of libsbp.so (argument marshalling only).

Every step of a solve runs in the library's CUDA kernels; PyTorch supplies
device memory and the current stream.  If the library is missing this module
raises instead of computing anything on the CPU.
"""

from __future__ import annotations

import ctypes
import os
from enum import IntEnum

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsbp.so")


class DType(IntEnum):
    F64 = 0
    F32 = 1
    F32_SPLIT_F16 = 2
    F32_SPLIT_BF16 = 3


class Status(IntEnum):
    OK = 0
    INVALID_ARG = 1
    UNSUPPORTED_SIZE = 2
    OUT_OF_MEMORY = 3
    CUDA = 4
    DEVICE_TIMEOUT = 5
    NOT_SAME_DTYPE = 6
    UNSUPPORTED_DTYPE = 7
    SCRATCH_LIMIT = 8


class Stage(IntEnum):
    X_FORWARD = 0
    Y_FORWARD = 1
    Z_CONVOLVE = 2
    Y_INVERSE = 3
    X_INVERSE = 4
    GREEN_TABLE = 5
    GREEN_FILL = 6
    SWEEP_FORWARD = 7
    SWEEP_MIDDLE = 8
    SWEEP_INVERSE = 9


class Option(IntEnum):
    Z_VARIANT = 1
    XY_PASSES = 2
    Y_TMA = 3
    SPIN_BUDGET = 4
    DEBUG_WITHHOLD_COPY = 5
    TRUNCATION = 6
    FRAME = 7
    METHOD = 8
    XY_CHUNK = 9
    SCHEDULE = 10


class SbpError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = Status(status) if status in Status._value2member_map_ else status
        msg = lib().sbp_status_string(int(status)).decode() if _lib is not None else str(status)
        if _lib is not None and int(status) == int(Status.CUDA):
            msg += " (" + lib().sbp_last_cuda_error().decode() + ")"
        super().__init__(f"{where}: {msg} (status {int(status)})")


_c_double = ctypes.c_double
_c_int = ctypes.c_int
_vp = ctypes.c_void_p

# name: (restype, argtypes) — the exact set declared in include/sbp.h
SIGNATURES = {
    "sbp_plan_create": (_c_int, [ctypes.POINTER(_vp), _c_int, _c_int, _c_int, _c_double, _c_double, _c_double,
                                 _c_double, _c_double, _c_double, _c_int]),
    "sbp_solve": (_c_int, [_vp, _vp, _vp, _c_double, _vp]),
    "sbp_solve_batched": (_c_int, [_c_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                   ctypes.POINTER(_c_double), _vp]),
    "sbp_plan_destroy": (None, [_vp]),
    "sbp_status_string": (ctypes.c_char_p, [_c_int]),
    "sbp_last_cuda_error": (ctypes.c_char_p, []),
    "sbp_fill_ghosts": (_c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, _c_int, ctypes.c_void_p]),
    "sbp_force": (_c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, _c_double, ctypes.c_void_p]),
    "sbp_plan_set_option": (_c_int, [_vp, _c_int, _c_double]),
    "sbp_plan_info": (_c_int, [_vp, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int), ctypes.POINTER(_c_int),
                               ctypes.POINTER(_c_int), ctypes.POINTER(_c_int), ctypes.POINTER(ctypes.c_size_t)]),
    "sbp_run_stage": (_c_int, [_vp, _c_int, _vp, _vp, _c_double, _vp]),
    "sbp_plan_sync_status": (_c_int, [_vp, _vp]),
    "sbp_version": (ctypes.c_char_p, []),
    "sbp_solve_noalloc": (_c_int, [_c_int, _c_int, _c_int, _c_double, _c_double, _c_double, _c_double, _c_double,
                                   _c_double, _vp, _vp, _c_double, _vp]),
    "sbp_plan_query": (_c_int, [_vp, _c_int, ctypes.POINTER(_c_double)]),
    "sbp_batch_info": (_c_int, [_c_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                ctypes.POINTER(_c_int), ctypes.POINTER(_c_int)]),
    "sbp_batch_run_stage": (_c_int, [_c_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp), _c_int,
                                     _c_int, _c_int, _c_int, _vp]),
}

_lib = None


def lib():
    """Load libsbp.so (built in-tree by ``paper_2510_10070_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run `python -m paper_2510_10070_gb300.build` "
                               "(there is no CPU fallback)")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def _check(status: int, where: str):
    if status != 0:
        raise SbpError(status, where)


def _stream_handle(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """A solver plan for one box (Sect. 2.3 method, see include/sbp.h)."""

    def __init__(self, nx, ny, nz, Lx, Ly, Lz, q=1.5, Omega=1.0, G=1.0, dtype=DType.F64):
        self._h = ctypes.c_void_p()
        _check(lib().sbp_plan_create(ctypes.byref(self._h), nx, ny, nz, Lx, Ly, Lz, q, Omega, G, int(dtype)),
               "sbp_plan_create")
        self.nx, self.ny, self.nz = nx, ny, nz
        self.Lx, self.Ly, self.Lz, self.q, self.Omega, self.G = Lx, Ly, Lz, q, Omega, G
        self.dtype = DType(dtype)
        pitch = ctypes.c_int()
        ws = ctypes.c_size_t()
        _check(lib().sbp_plan_info(self._h, None, None, None, None, ctypes.byref(pitch), ctypes.byref(ws)),
               "sbp_plan_info")
        self.spectrum_pitch = pitch.value
        self.workspace_bytes = ws.value

    @property
    def handle(self):
        return self._h

    @property
    def torch_dtype(self):
        import torch

        return torch.float64 if self.dtype == DType.F64 else torch.float32

    def _check_tensor(self, x, name):
        import torch

        if not isinstance(x, torch.Tensor) or not x.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if x.dtype != self.torch_dtype or tuple(x.shape) != (self.nz, self.ny, self.nx) or not x.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {self.torch_dtype} tensor of shape "
                             f"{(self.nz, self.ny, self.nx)}")

    def solve(self, rho, phi=None, t: float = 0.0, stream=None):
        """Φ̃ for density ρ̃ at shear time t; returns ``phi`` (allocated if None)."""
        import torch

        self._check_tensor(rho, "rho")
        if phi is None:
            phi = torch.empty_like(rho)
        self._check_tensor(phi, "phi")
        _check(lib().sbp_solve(self._h, ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(phi.data_ptr()),
                               float(t), _stream_handle(stream)), "sbp_solve")
        return phi

    def query(self, what: int) -> float:
        """sbp_plan_query: 1 = the schedule solves run (1 five passes, 2 three
        sweeps), 2 = kernels per sbp_solve."""
        v = ctypes.c_double()
        _check(lib().sbp_plan_query(self._h, int(what), ctypes.byref(v)), "sbp_plan_query")
        return v.value

    def schedule_is_sweep(self) -> bool:
        return self.query(1) == 2.0

    def set_option(self, option, value):
        _check(lib().sbp_plan_set_option(self._h, int(option), float(value)), "sbp_plan_set_option")

    def sync_status(self, stream=None):
        """Synchronise and raise SbpError if a device-side bounded wait gave up."""
        _check(lib().sbp_plan_sync_status(self._h, _stream_handle(stream)), "sbp_plan_sync_status")

    def new_spectrum(self):
        import torch

        return torch.zeros((self.nz, self.ny, self.spectrum_pitch, 2), dtype=self.torch_dtype, device="cuda")

    def fill_ghosts(self, phi, ng: int, out=None, stream=None):
        """phi with ng vertical ghost layers on each side (gradient of the last active cell kept)."""
        import torch

        self._check_tensor(phi, "phi")
        if out is None:
            out = torch.empty((self.nz + 2 * ng, self.ny, self.nx), dtype=self.torch_dtype, device=phi.device)
        _check(lib().sbp_fill_ghosts(self._h, ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                     int(ng), _stream_handle(stream)), "sbp_fill_ghosts")
        return out

    def force(self, phi, t: float = 0.0, out=None, stream=None):
        """g = -∇Φ, shape [3, nz, ny, nx], in the plan's frame at shear time t."""
        import torch

        self._check_tensor(phi, "phi")
        if out is None:
            out = torch.empty((3, self.nz, self.ny, self.nx), dtype=self.torch_dtype, device=phi.device)
        _check(lib().sbp_force(self._h, ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                               float(t), _stream_handle(stream)), "sbp_force")
        return out

    def run_stage(self, stage, inp, out, t: float = 0.0, stream=None):
        ip = ctypes.c_void_p(inp.data_ptr()) if inp is not None else None
        op = ctypes.c_void_p(out.data_ptr()) if out is not None else None
        _check(lib().sbp_run_stage(self._h, int(stage), ip, op, float(t), _stream_handle(stream)),
               f"sbp_run_stage({Stage(stage).name})")
        return out

    def close(self):
        if self._h is not None and self._h.value:
            lib().sbp_plan_destroy(self._h)
        self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batched(plans, rhos, phis, ts, stream=None):
    """Solve box i with plans[i] at time ts[i] (one call, one stream)."""
    n = len(plans)
    if not (len(rhos) == len(phis) == len(ts) == n):
        raise ValueError("plans, rhos, phis and ts must have the same length")
    for p, r, f in zip(plans, rhos, phis):
        p._check_tensor(r, "rho")
        p._check_tensor(f, "phi")
    hp = (ctypes.c_void_p * n)(*[p.handle.value for p in plans])
    rp = (ctypes.c_void_p * n)(*[r.data_ptr() for r in rhos])
    fp = (ctypes.c_void_p * n)(*[f.data_ptr() for f in phis])
    tp = (ctypes.c_double * n)(*[float(t) for t in ts])
    _check(lib().sbp_solve_batched(n, hp, rp, fp, tp, _stream_handle(stream)), "sbp_solve_batched")
    return phis


def batch_info(plans, rhos, phis):
    """(kernels per call, boxes in grouped sweeps) of the cached
    sbp_solve_batched graph for exactly these plans and buffers."""
    n = len(plans)
    hp = (ctypes.c_void_p * n)(*[p.handle.value for p in plans])
    rp = (ctypes.c_void_p * n)(*[r.data_ptr() for r in rhos])
    fp = (ctypes.c_void_p * n)(*[f.data_ptr() for f in phis])
    launches, grouped = ctypes.c_int(), ctypes.c_int()
    _check(lib().sbp_batch_info(n, hp, rp, fp, ctypes.byref(launches), ctypes.byref(grouped)), "sbp_batch_info")
    return launches.value, grouped.value


def batch_run_stage(plans, rhos, phis, shape, stage, stream=None):
    """One sweep (Stage.SWEEP_*) of the grouped boxes of `shape` (nx, ny, nz)
    of the cached sbp_solve_batched graph for exactly these plans and buffers."""
    n = len(plans)
    hp = (ctypes.c_void_p * n)(*[p.handle.value for p in plans])
    rp = (ctypes.c_void_p * n)(*[r.data_ptr() for r in rhos])
    fp = (ctypes.c_void_p * n)(*[f.data_ptr() for f in phis])
    nx, ny, nz = shape
    _check(lib().sbp_batch_run_stage(n, hp, rp, fp, int(nx), int(ny), int(nz), int(stage), _stream_handle(stream)),
           f"sbp_batch_run_stage({Stage(stage).name})")


def solve_noalloc(rho, phi, Lx, Ly, Lz, q=1.5, Omega=1.0, G=1.0, t=0.0, stream=None):
    """FP32 solve without any device allocation (fixed 40 MiB library workspace).

    For programs that may not allocate device memory while they run; see
    sbp_solve_noalloc in include/sbp.h.  ``rho`` and ``phi`` are contiguous
    float32 CUDA tensors [nz, ny, nx]; the caller allocates them.
    """
    import torch

    for x, name in ((rho, "rho"), (phi, "phi")):
        if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype != torch.float32 or not x.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    if rho.dim() != 3 or tuple(phi.shape) != tuple(rho.shape):
        raise ValueError("rho and phi must have the same shape [nz, ny, nx]")
    nz, ny, nx = rho.shape
    _check(lib().sbp_solve_noalloc(nx, ny, nz, Lx, Ly, Lz, q, Omega, G, ctypes.c_void_p(rho.data_ptr()),
                                   ctypes.c_void_p(phi.data_ptr()), float(t), _stream_handle(stream)),
           "sbp_solve_noalloc")
    return phi


def version() -> str:
    return lib().sbp_version().decode()
