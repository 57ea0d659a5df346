"""Seeded synthetic inputs and the named workloads (shared by tests and bench).

This module holds no arithmetic of the solver: only box geometries, shear
times and density generators.  Both the CUDA path and the CPU oracle take
their inputs from here.

Density families (stand-ins for NIRVANA-III stratified-disc fields, which are
not available):

* ``noisy_gaussian``  ρ = exp(-z²/2H²)(1 + 0.1 u), u ~ U[-1, 1] i.i.d.
* ``lognormal_disc``  ρ = exp(-z²/2H²) exp(σ g); g is white noise filtered per
  z-plane to a horizontal amplitude ∝ 1/|K_h| (power ∝ K_h⁻², K_h = 0
  removed) and normalised to unit variance.
* ``clumpy_disc``     ρ = exp(-z²/2H²) + Σ_c A_c exp(-|r - r_c|²/2 w_c²) with
  minimum-image distances in x and y.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def cell_centres(n: int, L: float):
    """Cell-centred coordinates in [-L/2, L/2]."""
    return -0.5 * L + (np.arange(n) + 0.5) * (L / n)


@dataclass(frozen=True)
class Box:
    nx: int
    ny: int
    nz: int
    Lx: float
    Ly: float
    Lz: float
    q: float = 1.5
    Omega: float = 1.0
    G: float = 1.0

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz


def noisy_gaussian(box: Box, seed: int = 0, H: float = 1.0, dtype=np.float64):
    rng = np.random.default_rng(seed)
    u = rng.uniform(-1.0, 1.0, (box.nz, box.ny, box.nx))
    z = cell_centres(box.nz, box.Lz)
    rho = np.exp(-0.5 * (z / H) ** 2)[:, None, None] * (1.0 + 0.1 * u)
    return rho.astype(dtype)


def lognormal_disc(box: Box, seed: int, sigma: float = 0.5, H: float = 1.0, dtype=np.float64):
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((box.nz, box.ny, box.nx))
    kx = np.fft.rfftfreq(box.nx, d=box.Lx / box.nx) * 2.0 * np.pi
    ky = np.fft.fftfreq(box.ny, d=box.Ly / box.ny) * 2.0 * np.pi
    kh = np.sqrt(kx[None, :] ** 2 + ky[:, None] ** 2)
    amp = np.zeros_like(kh)
    amp[kh > 0] = 1.0 / kh[kh > 0]
    for j in range(box.nz):  # plane by plane keeps the memory bounded
        g[j] = np.fft.irfft2(np.fft.rfft2(g[j]) * amp, s=(box.ny, box.nx))
    g /= g.std()
    z = cell_centres(box.nz, box.Lz)
    strat = np.exp(-0.5 * (z / H) ** 2)
    out = np.empty((box.nz, box.ny, box.nx), dtype=dtype)
    for j in range(box.nz):
        out[j] = (strat[j] * np.exp(sigma * g[j])).astype(dtype)
    return out


def clumpy_disc(box: Box, seed: int, nclump: int = 2000, H: float = 1.0, dtype=np.float32,
                device=None):
    """Gaussian disc plus ``nclump`` random clumps (width 0.02-0.1 H, amplitude 1-10).

    Evaluated with torch (on ``device`` if given) because the large box has
    5e8 cells; each clump only touches cells within 5 widths of its centre.
    """
    import torch

    rng = np.random.default_rng(seed)
    xc = rng.uniform(-0.5 * box.Lx, 0.5 * box.Lx, nclump)
    yc = rng.uniform(-0.5 * box.Ly, 0.5 * box.Ly, nclump)
    zc = np.clip(rng.standard_normal(nclump) * H, -0.5 * box.Lz, 0.5 * box.Lz)
    wc = rng.uniform(0.02, 0.1, nclump) * H
    Ac = rng.uniform(1.0, 10.0, nclump)
    dev = torch.device(device) if device is not None else torch.device("cpu")
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    x = torch.tensor(cell_centres(box.nx, box.Lx), dtype=tdt, device=dev)
    y = torch.tensor(cell_centres(box.ny, box.Ly), dtype=tdt, device=dev)
    z = torch.tensor(cell_centres(box.nz, box.Lz), dtype=tdt, device=dev)
    rho = torch.exp(-0.5 * (z / H) ** 2)[:, None, None].expand(box.nz, box.ny, box.nx).contiguous()
    dx, dy, dz = box.Lx / box.nx, box.Ly / box.ny, box.Lz / box.nz
    for c in range(nclump):
        r = 5.0 * wc[c]
        iz0 = max(0, int(np.floor((zc[c] - r + 0.5 * box.Lz) / dz)))
        iz1 = min(box.nz, int(np.ceil((zc[c] + r + 0.5 * box.Lz) / dz)) + 1)
        ix = np.arange(int(np.floor((xc[c] - r + 0.5 * box.Lx) / dx)),
                       int(np.ceil((xc[c] + r + 0.5 * box.Lx) / dx)) + 1) % box.nx
        iy = np.arange(int(np.floor((yc[c] - r + 0.5 * box.Ly) / dy)),
                       int(np.ceil((yc[c] + r + 0.5 * box.Ly) / dy)) + 1) % box.ny
        ix = np.unique(ix)
        iy = np.unique(iy)
        ddx = x[torch.as_tensor(ix, device=dev)] - xc[c]
        ddx = ddx - box.Lx * torch.round(ddx / box.Lx)
        ddy = y[torch.as_tensor(iy, device=dev)] - yc[c]
        ddy = ddy - box.Ly * torch.round(ddy / box.Ly)
        ddz = z[iz0:iz1] - zc[c]
        r2 = ddz[:, None, None] ** 2 + ddy[None, :, None] ** 2 + ddx[None, None, :] ** 2
        blob = Ac[c] * torch.exp(-0.5 * r2 / wc[c] ** 2)
        sub = rho[iz0:iz1][:, torch.as_tensor(iy, device=dev)][:, :, torch.as_tensor(ix, device=dev)]
        rho[iz0:iz1, torch.as_tensor(iy, device=dev)[:, None], torch.as_tensor(ix, device=dev)[None, :]] = sub + blob
    return rho


def random_half_spectrum(nz: int, ny: int, nx: int, seed: int, pitch: int | None = None):
    """Seeded complex array [nz, ny, pitch] (pitch ≥ nx/2+1) for single-stage tests."""
    rng = np.random.default_rng(seed)
    pitch = pitch or (nx // 2 + 1)
    return (rng.standard_normal((nz, ny, pitch)) + 1j * rng.standard_normal((nz, ny, pitch)))


# ---------------------------------------------------------------------------
# Named workloads (the sizes and parameters of the benchmarked cases)
# ---------------------------------------------------------------------------

BOX_32 = Box(32, 32, 32, 4.0, 4.0, 4.0)                 # 32³, L = 4, t = 0.7
T_32 = 0.7
BOX_256 = Box(256, 256, 128, 8.0, 8.0, 4.0)             # 256×256×128, t ∈ {0, 1.3, 5.0}
T_256 = (0.0, 1.3, 5.0)
BOX_512 = Box(512, 512, 256, 8.0, 8.0, 4.0)             # 512×512×256, t = 2.1
T_512 = 2.1
BOX_1024 = Box(1024, 1024, 512, 8.0, 8.0, 4.0)          # 1024×1024×512, t = 3.3
T_1024 = 3.3


@dataclass
class BatchCase:
    boxes: list = field(default_factory=list)
    seeds: list = field(default_factory=list)
    times: np.ndarray | None = None


def batch_96() -> BatchCase:
    """96 boxes: 32× 64³, 32× 128²×64, 16× 192²×96, 16× 256²×128.

    Box i: seed 100 + i, t_i ~ U[0, 10] from seed 4, q = 1.5 (even i) or 1.0
    (odd i), L = (8, 8, 4), σ = 0.7.
    """
    shapes = [(64, 64, 64)] * 32 + [(128, 128, 64)] * 32 + [(192, 192, 96)] * 16 + [(256, 256, 128)] * 16
    times = np.random.default_rng(4).uniform(0.0, 10.0, len(shapes))
    boxes = []
    for i, (nx, ny, nz) in enumerate(shapes):
        boxes.append(Box(nx, ny, nz, 8.0, 8.0, 4.0, q=1.5 if i % 2 == 0 else 1.0))
    return BatchCase(boxes=boxes, seeds=[100 + i for i in range(len(shapes))], times=times)


def downsample(rho, fx: int, fy: int, fz: int):
    """Every fx-th x, fy-th y and fz-th z sample (a coarse copy of the same field)."""
    return np.ascontiguousarray(rho[::fz, ::fy, ::fx])
