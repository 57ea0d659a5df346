"""Pins of the oracle's physical-frame mapping (Sect. 2.1, spectral variant).

The mapping shifts every x-column in y by s·x (Fourier interpolation); these
tests fix it against things it must reproduce exactly: integer-cell shifts are
rolls, a shear-periodic plane wave becomes a lattice mode, the two directions
invert each other and preserve the norm (without Nyquist content), and the
composed physical-frame solve of a shear-periodic mode has the closed-form
profile at |k(t)|.
"""

import numpy as np
import pytest

import analytic as A
import oracle as O


def _no_nyquist(f):
    """f with its y-Nyquist row removed (library FFT used only to build the input)."""
    F = np.fft.fft(f, axis=-2)
    F[..., f.shape[-2] // 2, :] = 0.0
    return np.fft.ifft(F, axis=-2).real


def test_integer_cell_shift_is_a_roll():
    # nx = 4, ny = 16, Δy0 = Ly/2: the shift of column i is
    # s x_i / dy = (Δy0/Ly) ny (x_i/Lx) = 8 (2i - 3)/8 = 2i - 3 cells.
    nx, ny = 4, 16
    Lx, Ly = 2.0, 3.0
    rng = np.random.default_rng(0)
    f = rng.standard_normal((3, ny, nx))
    u = O.remap_phase(nx, Lx, Ly, 0.5 * Ly)
    shifts = u * ny
    assert np.allclose(shifts, [-3, -1, 1, 3], atol=1e-14)
    g = O.remap_y(f, u, -1.0)  # ρ̃(x, y) = ρ(x, y - s x): column i moves by +shift_i
    want = np.stack([np.roll(f[..., i], int(round(shifts[i])), axis=-1) for i in range(nx)], axis=-1)
    assert np.max(np.abs(g - want)) < 1e-12
    back = O.remap_y(g, u, +1.0)
    assert np.max(np.abs(back - f)) < 1e-12


def test_shear_periodic_wave_becomes_lattice_mode():
    # cos(k_x x + K_y y + φ) with k_x = K_x + s K_y obeys f(x+Lx, y) = f(x, y+Δy0)
    # and maps to cos(K_x x + K_y y + φ) exactly (band-limited in y).
    nx, ny = 6, 10
    Lx, Ly = 2.0, 3.0
    dy0 = 1.234
    s = dy0 / Lx
    a, b, phi0 = 2, 3, 0.4
    Kx, Ky = 2 * np.pi * a / Lx, 2 * np.pi * b / Ly
    x = A.cell_centres(nx, Lx)
    y = A.cell_centres(ny, Ly)
    phys = np.cos((Kx + s * Ky) * x[None, :] + Ky * y[:, None] + phi0)
    lattice = np.cos(Kx * x[None, :] + Ky * y[:, None] + phi0)
    u = O.remap_phase(nx, Lx, Ly, dy0)
    assert np.max(np.abs(O.remap_y(phys, u, -1.0) - lattice)) < 1e-13
    assert np.max(np.abs(O.remap_y(lattice, u, +1.0) - phys)) < 1e-13


def test_round_trip_and_norm_without_nyquist():
    rng = np.random.default_rng(1)
    f = _no_nyquist(rng.standard_normal((2, 12, 8)))
    u = O.remap_phase(8, 2.0, 3.0, 2.71)
    g = O.remap_y(f, u, -1.0)
    assert np.max(np.abs(O.remap_y(g, u, +1.0) - f)) < 1e-12
    assert abs(np.linalg.norm(g) - np.linalg.norm(f)) < 1e-12 * np.linalg.norm(f)
    # zero shift is the identity, with or without Nyquist content
    h = rng.standard_normal((2, 12, 8))
    assert np.max(np.abs(O.remap_y(h, np.zeros(8), -1.0) - h)) < 1e-12


def test_nyquist_row_scaled_by_cosine():
    # a pure Nyquist row (-1)^y keeps its shape and is scaled by cos(π ny u_x)
    nx, ny = 4, 8
    u = O.remap_phase(nx, 1.0, 1.0, 0.3)
    f = np.tile(((-1.0) ** np.arange(ny))[:, None], (1, nx))
    g = O.remap_y(f, u, -1.0)
    assert np.max(np.abs(g - f * np.cos(np.pi * ny * u)[None, :])) < 1e-13


@pytest.mark.parametrize("t", [0.0, 0.7, 2.3])
def test_physical_frame_solve_of_shear_periodic_mode(t):
    # ρ = cos(k_x x + K_y y) e^{-z²/2H²} with k_x = K_x + s K_y in the physical
    # frame: Φ = 4πG cos(k_x x + K_y y) F(|k(t)|, z), error = z discretisation only
    Lx = Ly = Lz = 4.0
    H = 1.0
    p = O.SolveParams(Lx, Ly, Lz, q=1.5, Omega=1.0)
    s = O.shear_offset(1.5, 1.0, Lx, Ly, t) / Lx
    a, b = 1, 2
    Ky = 2.0 * np.pi * b / Ly
    kx = 2.0 * np.pi * a / Lx + s * Ky
    n = 8
    x = A.cell_centres(n, Lx)
    y = A.cell_centres(n, Ly)
    horiz = np.cos(kx * x[None, :] + Ky * y[:, None])
    errs = []
    ns = [32, 64, 128]
    for nz in ns:
        z = A.cell_centres(nz, Lz)
        rho = horiz[None] * np.exp(-0.5 * (z / H) ** 2)[:, None, None]
        phi = O.solve_physical(rho, p, t)
        ex = 4.0 * np.pi * horiz[None] * A.mode_profile_paper(z, np.hypot(kx, Ky), H, Lz)[:, None, None]
        errs.append(A.rel_l2(phi, ex))
    assert errs[0] < 5e-4
    order = np.polyfit(np.log(ns), np.log(errs), 1)[0]
    assert -2.15 < order < -1.85  # second order in dz


def test_physical_solve_equals_periodic_solve_at_zero_shear():
    rng = np.random.default_rng(2)
    rho = rng.standard_normal((6, 8, 6))
    p = O.SolveParams(2.0, 3.0, 1.5, q=1.5, Omega=1.0)
    period = p.Ly / (p.q * p.Omega * p.Lx)
    for t in (0.0, period):
        assert np.max(np.abs(O.solve_physical(rho, p, t) - O.solve(rho, p, t))) < 1e-12
