"""Pins of the oracle's ghost-cell fill and force (Sect. 2.4, last paragraph).

Ghost layers continue the last active cell's gradient; the force is -∇Φ by
second-order central differences (periodic y; periodic or shear-periodic x).
Checked against exact results: linear fields continue exactly, central
differences of lattice modes and quadratics have closed forms, and across the
x boundary of the physical frame a shear-periodic wave has the same closed
form as in the interior.
"""

import numpy as np
import pytest

import analytic as A
import oracle as O


def test_ghosts_continue_linear_fields_exactly():
    nz, ny, nx, ng = 6, 4, 5, 3
    Lz = 1.5
    z = A.cell_centres(nz, Lz)
    dz = Lz / nz
    zg = np.concatenate([z[0] - dz * np.arange(ng, 0, -1), z, z[-1] + dz * np.arange(1, ng + 1)])
    rng = np.random.default_rng(0)
    a, b = rng.standard_normal((ny, nx)), rng.standard_normal((ny, nx))
    phi = a[None] + b[None] * z[:, None, None]
    out = O.fill_ghosts(phi, ng)
    assert np.max(np.abs(out - (a[None] + b[None] * zg[:, None, None]))) < 1e-13
    # every ghost step repeats the gradient of the last active cell
    f = rng.standard_normal((nz, ny, nx))
    g = O.fill_ghosts(f, ng)
    for k in range(ng):
        assert np.allclose(g[ng + nz + k] - g[ng + nz + k - 1], f[-1] - f[-2], atol=1e-14)
        assert np.allclose(g[ng - 1 - k] - g[ng - k], f[0] - f[1], atol=1e-14)


def test_force_of_lattice_mode_and_quadratic():
    nz, ny, nx = 8, 12, 10
    p = O.SolveParams(2.0, 3.0, 1.5)
    x, y, z = A.cell_centres(nx, p.Lx), A.cell_centres(ny, p.Ly), A.cell_centres(nz, p.Lz)
    dx, dy, dz = p.Lx / nx, p.Ly / ny, p.Lz / nz
    Kx, Ky = 2 * np.pi * 3 / p.Lx, 2 * np.pi * 2 / p.Ly
    arg = Kx * x[None, :] + Ky * y[:, None]
    phi = np.cos(arg)[None] * np.ones((nz, 1, 1)) + (z ** 2)[:, None, None]
    g = O.force(phi, p, 0.9, physical=False)
    # central differences: d/dx cos → -sin · sin(K dx)/dx, so g_x = +sin · sin(K dx)/dx
    assert np.max(np.abs(g[0] - np.sin(arg)[None] * np.sin(Kx * dx) / dx)) < 1e-12
    assert np.max(np.abs(g[1] - np.sin(arg)[None] * np.sin(Ky * dy) / dy)) < 1e-12
    # z²: exact -2z inside, one-sided -(z0 + z1) and -(z_{n-2} + z_{n-1}) at the ends
    gz = g[2][:, 0, 0]
    assert np.max(np.abs(gz[1:-1] + 2 * z[1:-1])) < 1e-12
    assert abs(gz[0] + (z[0] + z[1])) < 1e-12 and abs(gz[-1] + (z[-2] + z[-1])) < 1e-12


@pytest.mark.parametrize("t", [0.37, 1.9])
def test_force_across_the_shearing_boundary(t):
    nz, ny, nx = 3, 16, 8
    p = O.SolveParams(2.0, 3.0, 1.0, q=1.5, Omega=1.0)
    s = O.shear_offset(p.q, p.Omega, p.Lx, p.Ly, t) / p.Lx
    x, y = A.cell_centres(nx, p.Lx), A.cell_centres(ny, p.Ly)
    dx = p.Lx / nx
    Ky = 2 * np.pi * 3 / p.Ly
    kx = 2 * np.pi * 1 / p.Lx + s * Ky  # shear-periodic: Φ(x + Lx, y) = Φ(x, y + Δy0)
    arg = kx * x[None, :] + Ky * y[:, None]
    phi = np.cos(arg)[None] * np.ones((nz, 1, 1))
    g = O.force(phi, p, t, physical=True)
    assert np.max(np.abs(g[0] - np.sin(arg)[None] * np.sin(kx * dx) / dx)) < 1e-12
    # the periodic-frame stencil would be wrong at the two boundary columns
    gp = O.force(phi, p, t, physical=False)
    assert np.max(np.abs(gp[0][:, :, 1:-1] - g[0][:, :, 1:-1])) < 1e-14
    assert np.max(np.abs(gp[0][:, :, 0] - g[0][:, :, 0])) > 1e-2
