"""Pins of the FP64 oracle against things other than itself.

* Ĝ^L against quadrature of its defining Fourier integral (Eq. VGF shearing
  box, Appendix A), and the k_z → 0 limit printed in Appendix A.
* Whole solves against closed-form potentials: the uniform slab, the shifted
  1D Gaussian of Sect. 3.1 (with the constant the paper drops), the 3D mode of
  Sect. 3.2, and a sheared single mode (Sect. 2.1 wave-vector).
* Convergence: 2nd order in the standard relative L2 norm and "slightly
  better than third order" in the paper's norm (Sect. 3.3).
* The same discrete operator computed by a library FFT on the zero-padded
  grid (Sect. 2.3, Φ = 4πG F⁻¹(Ĝ·ρ̂)) on tiny grids, plus brute-force
  operator properties (symmetry, linearity, translations, reflection,
  shear periodicity).
"""

import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")

import analytic as A
import oracle as O


# --------------------------------------------------------------------------
# Green's function in Fourier space
# --------------------------------------------------------------------------

@pytest.mark.parametrize("L", [1.0, 4.0, 4.4, 6.6])
@pytest.mark.parametrize("k", [0.0, 0.31, 1.7, 5.0])
@pytest.mark.parametrize("kz", [0.0, 0.4, 2.5, 7.1, 30.0])
def test_green_hat_matches_quadrature(L, k, kz):
    got = float(O.green_hat(k, kz, L, k == 0.0))
    want = A.green_hat_quad(k, kz, L)
    assert abs(got - want) <= 1e-11 * max(1.0, abs(want)), (got, want)


def test_green_hat_k0_small_kz_limit_is_L2_over_2():
    # Appendix A: expanding the k = 0 formula to second order gives L²/2 at k_z = 0.
    for L in (1.0, 4.0, 6.6):
        for kz in (1e-3, 1e-4):
            got = float(O.green_hat(0.0, kz, L, True))
            assert abs(got - 0.5 * L * L) < 1e-5 * L * L
        assert float(O.green_hat(0.0, 0.0, L, True)) == 0.5 * L * L


def test_green_hat_alpha1_closed_form():
    # With L = Lz and k_z = π m / Lz the trig terms are sin = 0, cos = (-1)^m,
    # so Ĝ = -(1 - (-1)^m e^{-kL})/(k² + k_z²); pinned against quadrature.
    Lz = 4.0
    for k in (0.7, 2.0):
        for m in range(0, 9):
            kz = np.pi * m / Lz
            want = A.green_hat_quad(k, kz, Lz)
            got = -(1.0 - (-1.0) ** m * np.exp(-k * Lz)) / (k * k + kz * kz)
            assert abs(got - want) < 1e-11
            assert abs(float(O.green_hat(k, kz, Lz, False)) - want) < 1e-11


def test_shear_offset_wraps_into_box():
    Lx, Ly = 8.0, 8.0
    assert O.shear_offset(1.5, 1.0, Lx, Ly, 0.0) == 0.0
    period = Ly / (1.5 * 1.0 * Lx)
    for t in (0.3, 1.3, 5.0, -2.2, -1e-18):
        d = O.shear_offset(1.5, 1.0, Lx, Ly, t)
        assert 0.0 <= d < Ly
        d2 = O.shear_offset(1.5, 1.0, Lx, Ly, t + period)
        assert abs(d - d2) < 1e-12 or abs(abs(d - d2) - Ly) < 1e-12


def test_signed_index_and_partner():
    n = 8
    s = O.signed_index(np.arange(n), n)
    assert list(s) == [0, 1, 2, 3, -4, -3, -2, -1]
    k1, k2, z = O.mode_wavenumbers(8, 6, 2.0, 3.0, 0.37)
    assert z.sum() == 1 and z[0, 0]
    # off the Nyquist planes the partner has the same |k|
    assert np.allclose(k1[:3, :4], k2[:3, :4], rtol=0, atol=0) or np.allclose(k1[1:3, 1:4], k2[1:3, 1:4])
    # unsheared: k(-K) = k(K) everywhere, including the Nyquist planes
    k1, k2, _ = O.mode_wavenumbers(8, 6, 2.0, 3.0, 0.0)
    assert np.array_equal(k1, k2)


# --------------------------------------------------------------------------
# Closed-form potentials
# --------------------------------------------------------------------------

def _fit_order(ns, errs):
    return -np.polyfit(np.log(ns), np.log(errs), 1)[0]


def test_uniform_slab_second_order():
    Lz = 4.0
    p = O.SolveParams(4.0, 4.0, Lz)
    ns = [16, 32, 64]
    errs = []
    for nz in ns:
        z = A.cell_centres(nz, Lz)
        phi = O.solve(np.ones((nz, 4, 4)), p, 0.0)
        assert np.ptp(phi, axis=(1, 2)).max() < 1e-12 * np.abs(phi).max()  # x,y independent
        errs.append(A.rel_l2(phi[:, 0, 0], A.slab_potential(z, Lz)))
    assert errs[0] < 2e-3
    assert 1.9 < _fit_order(ns, errs) < 2.1


def test_paper_1d_constant_reading():
    # The printed 1D potential equals the exact integral up to the constant
    # Sect. 3.1 sets to zero; both sides are independent of the oracle.
    for z0 in (0.0, 2.0):
        z = np.linspace(-3.0, 3.0, 13)
        exact = A.gauss1d_potential_exact(z, z0, 6.0)
        paper = A.gauss1d_potential_paper(z, z0, 6.0)
        C = A.gauss1d_dropped_constant(z0, 6.0)
        assert np.allclose(paper - 4.0 * np.pi * C, exact, rtol=0, atol=1e-12)
    assert abs(A.gauss1d_dropped_constant(0.0, 6.0) - np.exp(-4.5)) < 1e-15


@pytest.mark.parametrize("z0", [0.0, 2.0])
def test_paper_1d_gaussian(z0):
    # Sect. 3.1: L = 6, shifted and centred Gaussians.  A horizontally uniform
    # density only excites the (0,0) mode, so 4×4 horizontal cells suffice.
    L = 6.0
    p = O.SolveParams(L, L, L)
    ns = [16, 32, 64, 128]
    rel, pnorm, emax = [], [], []
    for nz in ns:
        z = A.cell_centres(nz, L)
        rho = np.broadcast_to(np.exp(-0.5 * (z - z0) ** 2)[:, None, None], (nz, 4, 4)).copy()
        phi = O.solve(rho, p, 0.0)[:, 0, 0]
        ex = A.gauss1d_potential_exact(z, z0, L)
        eps = np.abs((phi - ex) / ex)
        rel.append(A.rel_l2(phi, ex))
        # paper norm over an nz³ grid of identical columns: (1/N)√(N/nz Σ_z ε²)
        pnorm.append(np.sqrt(nz * nz * np.sum(eps ** 2)) / nz ** 3)
        emax.append(eps.max())
    assert 1.95 < _fit_order(ns, rel) < 2.05
    assert 3.0 < _fit_order(ns, pnorm) < 4.0          # "slightly better than third order"
    assert 1e-7 < pnorm[0] < 1e-4                       # 16³: between ~1e-7 and ~1e-5
    if z0 != 0.0:
        assert 1e-6 < emax[-1] < 1e-4                   # 128³ shifted: 1e-6 .. 1e-4


@pytest.mark.parametrize("H", [1.0, 3.0])
def test_paper_3d_mode(H):
    # Sect. 3.2: ρ = cos(k x) cos(k y) exp(-z²/2H²), L = 6, k_x = k_y = 2π/L.
    L = 6.0
    p = O.SolveParams(L, L, L)
    kx = 2.0 * np.pi / L
    n = 8
    x = A.cell_centres(n, L)
    horiz = np.cos(kx * x)[None, :] * np.cos(kx * x)[:, None]
    ns = [16, 32, 64]
    rel, pnorm = [], []
    for nz in ns:
        z = A.cell_centres(nz, L)
        rho = horiz[None] * np.exp(-0.5 * (z / H) ** 2)[:, None, None]
        phi = O.solve(rho, p, 0.0)
        ex = 4.0 * np.pi * horiz[None] * A.mode_profile_paper(z, np.sqrt(2.0) * kx, H, L)[:, None, None]
        rel.append(A.rel_l2(phi, ex))
        col = np.abs((phi[:, 1, 1] - ex[:, 1, 1]) / ex[:, 1, 1])
        pnorm.append(np.sqrt(nz * nz * np.sum(col ** 2)) / nz ** 3)
    assert 1.85 < _fit_order(ns, rel) < 2.15
    assert 3.0 < _fit_order(ns, pnorm) < 4.0
    assert rel[-1] < (2e-5 if H == 1.0 else 2e-4)


def test_mode_profile_paper_matches_quadrature():
    for (k, H, Lz) in [(np.sqrt(2.0) * 2 * np.pi / 6, 1.0, 6.0), (2.277655, 1.0, 4.0), (0.5, 0.7, 2.0)]:
        for z in np.linspace(-0.5 * Lz, 0.5 * Lz, 7):
            a = A.mode_profile_paper(z, k, H, Lz)
            b = A.mode_profile_quad(z, k, H, Lz)
            assert abs(a - b) < 1e-10 * abs(b)


def test_sheared_single_mode():
    # A plane wave cos(K'·r) in the physical frame, remapped y → y - s x,
    # becomes the lattice mode cos(2πa x/Lx + 2πb y/Ly) with K'x = 2πa/Lx + s K'y.
    # Its potential is the ordinary 3D-mode profile at |K'| = k(t) of Sect. 2.1.
    Lx = Ly = Lz = 4.0
    H = 1.0
    p = O.SolveParams(Lx, Ly, Lz, q=1.5, Omega=1.0)
    t = 0.7
    s = O.shear_offset(1.5, 1.0, Lx, Ly, t) / Lx
    a, b = 1, 2
    Ky = 2.0 * np.pi * b / Ly
    kphys = np.hypot(2.0 * np.pi * a / Lx + s * Ky, Ky)
    n = 8
    x = A.cell_centres(n, Lx)
    y = A.cell_centres(n, Ly)
    horiz = np.cos(2.0 * np.pi * a * x[None, :] / Lx + 2.0 * np.pi * b * y[:, None] / Ly)
    errs = []
    ns = [32, 64, 128]
    for nz in ns:
        z = A.cell_centres(nz, Lz)
        rho = horiz[None] * np.exp(-0.5 * (z / H) ** 2)[:, None, None]
        phi = O.solve(rho, p, t)
        ex = 4.0 * np.pi * horiz[None] * A.mode_profile_paper(z, kphys, H, Lz)[:, None, None]
        errs.append(A.rel_l2(phi, ex))
    assert errs[0] < 5e-4
    assert 1.85 < _fit_order(ns, errs) < 2.15
    # the unsheared wave number gives a clearly different (wrong) answer
    z = A.cell_centres(32, Lz)
    rho = horiz[None] * np.exp(-0.5 * z ** 2)[:, None, None]
    wrong = 4.0 * np.pi * horiz[None] * A.mode_profile_paper(z, np.hypot(2 * np.pi * a / Lx, Ky), H, Lz)[:, None, None]
    assert A.rel_l2(O.solve(rho, p, t), wrong) > 1e-2


# --------------------------------------------------------------------------
# Library-FFT definition and brute-force properties on tiny grids
# --------------------------------------------------------------------------

def _fft_definition(rho, p, t, symmetrize):
    """Φ = 4πG Re F⁻¹[Ĝ · F(ρ zero-padded to pad·nz)] with numpy's FFT."""
    nz, ny, nx = rho.shape
    M = p.pad * nz
    pad = np.zeros((M, ny, nx))
    pad[:nz] = rho
    F = np.fft.fftn(pad)
    s = O.shear_offset(p.q, p.Omega, p.Lx, p.Ly, t) / p.Lx
    k1, k2, is0 = O.mode_wavenumbers(nx, ny, p.Lx, p.Ly, s)
    m = O.signed_index(np.arange(M), M)
    kz = 2.0 * np.pi * m / (M * (p.Lz / nz))
    L = p.alpha * p.Lz
    g = O.green_hat(k1[None], kz[:, None, None], L, is0[None])
    if symmetrize:
        g = 0.5 * (g + O.green_hat(k2[None], kz[:, None, None], L, is0[None]))
    out = np.fft.ifftn(g * F)[:nz] * 4.0 * np.pi * p.G
    return out


@pytest.mark.parametrize("shape,t", [((8, 6, 8), 0.7), ((8, 8, 8), 0.0), ((6, 4, 12), 2.3), ((3, 4, 6), 0.41)])
def test_matches_padded_library_fft(shape, t):
    rng = np.random.default_rng(11)
    rho = rng.standard_normal(shape)
    p = O.SolveParams(2.0, 3.0, 1.5, q=1.5, Omega=0.9, G=0.8)
    got = O.solve(rho, p, t)
    full = _fft_definition(rho, p, t, symmetrize=False)
    # R3: the oracle's output is the real part of the full complex solve
    assert A.rel_l2(got, full.real) < 1e-13
    sym = _fft_definition(rho, p, t, symmetrize=True)
    assert np.abs(sym.imag).max() < 1e-13 * np.abs(sym.real).max()
    assert A.rel_l2(got, sym.real) < 1e-13


def test_alpha_11_with_fourfold_padding_matches_library_fft():
    rng = np.random.default_rng(12)
    rho = rng.standard_normal((8, 6, 8))
    p = O.SolveParams(2.0, 3.0, 1.5, pad=4, alpha=1.1)
    got = O.solve(rho, p, 0.9)
    full = _fft_definition(rho, p, 0.9, symmetrize=False)
    assert A.rel_l2(got, full.real) < 1e-13


def test_operator_is_symmetric_and_linear():
    nz, ny, nx = 8, 6, 8
    p = O.SolveParams(2.0, 3.0, 1.5)
    N = nz * ny * nx
    Aop = np.empty((N, N))
    for i in range(N):
        e = np.zeros(N)
        e[i] = 1.0
        Aop[:, i] = O.solve(e.reshape(nz, ny, nx), p, 0.7).ravel()
    assert np.abs(Aop - Aop.T).max() < 1e-13 * np.abs(Aop).max()
    rng = np.random.default_rng(3)
    r1, r2 = rng.standard_normal((2, nz, ny, nx))
    lhs = O.solve(2.0 * r1 - 0.5 * r2, p, 0.7)
    rhs = 2.0 * O.solve(r1, p, 0.7) - 0.5 * O.solve(r2, p, 0.7)
    assert A.rel_l2(lhs, rhs) < 1e-13
    assert A.rel_l2(Aop @ r1.ravel(), O.solve(r1, p, 0.7).ravel()) < 1e-13


def test_translation_reflection_and_shear_period():
    rng = np.random.default_rng(4)
    rho = rng.standard_normal((8, 6, 8))
    p = O.SolveParams(2.0, 3.0, 1.5, q=1.5, Omega=1.0)
    t = 0.7
    base = O.solve(rho, p, t)
    # integer-cell translations in x and y commute with the solve
    assert A.rel_l2(O.solve(np.roll(rho, 3, axis=2), p, t), np.roll(base, 3, axis=2)) < 1e-13
    assert A.rel_l2(O.solve(np.roll(rho, -2, axis=1), p, t), np.roll(base, -2, axis=1)) < 1e-13
    # z-reflection (Ĝ depends on k_z²)
    assert A.rel_l2(O.solve(rho[::-1], p, t), base[::-1]) < 1e-13
    # shear periodicity: Δy0 is taken mod L_y
    period = p.Ly / (p.q * p.Omega * p.Lx)
    assert A.rel_l2(O.solve(rho, p, t + period), base) < 1e-12
    # t = 0 is the unsheared solve, and sheared differs from it
    p0 = O.SolveParams(2.0, 3.0, 1.5, q=0.0)
    assert A.rel_l2(O.solve(rho, p, 0.0), O.solve(rho, p0, 5.0)) < 1e-15
    assert A.rel_l2(base, O.solve(rho, p, 0.0)) > 1e-3


def test_ky0_modes_do_not_depend_on_shear_time():
    rng = np.random.default_rng(5)
    f = rng.standard_normal((8, 1, 8))
    rho = np.broadcast_to(f, (8, 6, 8)).copy()
    p = O.SolveParams(2.0, 3.0, 1.5)
    assert A.rel_l2(O.solve(rho, p, 0.3), O.solve(rho, p, 2.9)) < 1e-13


def test_stage_functions_compose():
    rng = np.random.default_rng(6)
    rho = rng.standard_normal((6, 8, 12))
    X = O.dft_x(rho)
    assert np.allclose(X, np.fft.rfft(rho, axis=2), atol=1e-12)
    R = O.horizontal_dft(rho)
    assert np.allclose(R, np.fft.fft2(rho), atol=1e-11)
    assert np.allclose(O.dft_y(X), R[:, :, :7], atol=1e-11)
    assert np.allclose(O.inverse_horizontal_dft(R), rho, atol=1e-13)
    S = O.plane_sums(rho)
    assert np.allclose(S, R[:, 0, 0].real, atol=1e-12)
    # half-spectrum inverse = unnormalised library irfft (which also drops
    # the imaginary parts of the a = 0 and a = nx/2 terms)
    Xn = X + 1j * rng.standard_normal(X.shape)
    assert np.allclose(O.inverse_dft_x_half(Xn, 12), np.fft.irfft(Xn, n=12, axis=2) * 12, atol=1e-12)
    assert np.allclose(O.inverse_dft_x_half(X, 12), rho * 12, atol=1e-12)


def test_solve_at_matches_solve():
    rng = np.random.default_rng(7)
    rho = rng.standard_normal((8, 6, 8))
    p = O.SolveParams(2.0, 3.0, 1.5)
    full = O.solve(rho, p, 1.1)
    pts = [(0, 0, 0), (7, 5, 7), (3, 2, 6), (3, 4, 1)]
    got = O.solve_at(rho, p, 1.1, pts)
    want = np.array([full[i, y, x] for (i, y, x) in pts])
    assert np.allclose(got, want, rtol=1e-13, atol=1e-13)


def test_k0_potential_is_mean_mode():
    # With zero-mean planes removed, the k = 0 contribution alone equals the
    # solve of the plane-averaged density.
    rng = np.random.default_rng(8)
    rho = rng.standard_normal((8, 6, 8))
    p = O.SolveParams(2.0, 3.0, 1.5)
    mean = np.broadcast_to(rho.mean(axis=(1, 2), keepdims=True), rho.shape).copy()
    v = O.k0_potential(O.plane_sums(rho), 8, 6, 8, p)
    assert np.allclose(O.solve(mean, p, 0.4)[:, 0, 0], v, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("H", [1.0, 3.0])
def test_paper_alpha_11_fourfold_padding_3d_mode(H):
    # Sect. 2.3/2.4 parameters (α = 1.1, domain quadrupled in z): same
    # closed-form error and 2nd-order convergence as α = 1 with 2× padding.
    L = 6.0
    kx = 2.0 * np.pi / L
    n = 8
    x = A.cell_centres(n, L)
    horiz = np.cos(kx * x)[None, :] * np.cos(kx * x)[:, None]
    errs = []
    ns = [16, 32, 64]
    for nz in ns:
        z = A.cell_centres(nz, L)
        rho = horiz[None] * np.exp(-0.5 * (z / H) ** 2)[:, None, None]
        ex = 4.0 * np.pi * horiz[None] * A.mode_profile_paper(z, np.sqrt(2.0) * kx, H, L)[:, None, None]
        e4 = A.rel_l2(O.solve(rho, O.SolveParams(L, L, L, pad=4, alpha=1.1), 0.0), ex)
        e2 = A.rel_l2(O.solve(rho, O.SolveParams(L, L, L), 0.0), ex)
        assert abs(e4 - e2) < 0.05 * e2
        errs.append(e4)
    assert 1.85 < _fit_order(ns, errs) < 2.15


def test_alpha_11_needs_fourfold_padding():
    # R1: with 2× padding the α = 1.1 kernel aliases the k = 0 column's image
    # at ±2Lz; the centred 1D Gaussian then stalls near 5e-3 instead of converging.
    L = 6.0
    z = A.cell_centres(64, L)
    rho = np.broadcast_to(np.exp(-0.5 * z ** 2)[:, None, None], (64, 4, 4)).copy()
    ex = A.gauss1d_potential_exact(z, 0.0, L)
    bad = A.rel_l2(O.solve(rho, O.SolveParams(L, L, L, pad=2, alpha=1.1), 0.0)[:, 0, 0], ex)
    good = A.rel_l2(O.solve(rho, O.SolveParams(L, L, L, pad=4, alpha=1.1), 0.0)[:, 0, 0], ex)
    assert bad > 1e-3 and good < 2e-5
