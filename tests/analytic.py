"""Closed-form potentials used to pin the oracle (test helpers, not the method).

Each function here is an independent statement of a potential that the paper
prints or that follows from its Green's function by direct integration; none
of them calls the oracle.
"""

from __future__ import annotations

import numpy as np
from scipy import integrate, special

SQRT_HALF_PI = np.sqrt(np.pi / 2.0)


def cell_centres(n: int, L: float):
    """Cell-centred coordinates of a window [-L/2, L/2] (Sect. 3.1 grid)."""
    return -0.5 * L + (np.arange(n) + 0.5) * (L / n)


def slab_potential(z, Lz: float, rho0: float = 1.0, G: float = 1.0):
    """Uniform slab of density rho0 filling |z| ≤ Lz/2 (Eq. one-dim-green integrated).

    Φ(z) = 4πG ρ0 ∫ ½|z - z'| dz' = 4πG ρ0 (z² + Lz²/4) / 2 inside the slab.
    """
    z = np.asarray(z, dtype=np.float64)
    return 4.0 * np.pi * G * rho0 * 0.5 * (z * z + 0.25 * Lz * Lz)


def _phi_g(x):
    """∫_0^x exp(-u²/2) du."""
    return SQRT_HALF_PI * special.erf(x / np.sqrt(2.0))


def gauss1d_potential_exact(z, z0: float, Lz: float, G: float = 1.0):
    """Φ(z) = 4πG ∫_{-Lz/2}^{Lz/2} ½|z - z'| exp(-(z'-z0)²/2) dz', in closed form.

    Derived by splitting the integral at z' = z (w = z - z0, c± = ±Lz/2 - z0):
    Φ/4πG = w Φg(w) + e^{-w²/2} - ½ w [Φg(c-) + Φg(c+)] - ½ [e^{-c-²/2} + e^{-c+²/2}].
    """
    z = np.asarray(z, dtype=np.float64)
    w = z - z0
    cm = -0.5 * Lz - z0
    cp = 0.5 * Lz - z0
    val = (w * _phi_g(w) + np.exp(-0.5 * w * w)
           - 0.5 * w * (_phi_g(cm) + _phi_g(cp))
           - 0.5 * (np.exp(-0.5 * cm * cm) + np.exp(-0.5 * cp * cp)))
    return 4.0 * np.pi * G * val


def gauss1d_potential_paper(z, z0: float, Lz: float, G: float = 1.0):
    """The potential as printed in Sect. 3.1 (integration constant taken as zero)."""
    z = np.asarray(z, dtype=np.float64)
    a = -0.5 * SQRT_HALF_PI * (special.erf((-0.5 * Lz - z0) / np.sqrt(2.0))
                               + special.erf((0.5 * Lz - z0) / np.sqrt(2.0)))
    w = z - z0
    val = SQRT_HALF_PI * w * special.erf(w / np.sqrt(2.0)) + np.exp(-0.5 * w * w) + a * z
    return 4.0 * np.pi * G * val


def gauss1d_dropped_constant(z0: float, Lz: float):
    """C such that exact = paper's printed form - 4πG·C (the constant Sect. 3.1 sets to zero).

    C = ½(e^{-c+²/2} + e^{-c-²/2}) + ½ z0 (M+ - M-), M+ = √(π/2) erfc(c+/√2),
    M- = √(π/2) erfc(-c-/√2).
    """
    cp = 0.5 * Lz - z0
    cm = -0.5 * Lz - z0
    Mp = SQRT_HALF_PI * special.erfc(cp / np.sqrt(2.0))
    Mm = SQRT_HALF_PI * special.erfc(-cm / np.sqrt(2.0))
    return 0.5 * (np.exp(-0.5 * cp * cp) + np.exp(-0.5 * cm * cm)) + 0.5 * z0 * (Mp - Mm)


def mode_profile_paper(z, k: float, H: float, Lz: float):
    """Vertical profile F(z) of the 3D test of Sect. 3.2 (as printed).

    For ρ = cos(k_x x) cos(k_y y) exp(-z²/2H²) the paper gives
    Φ = 4πG cos(k_x x) cos(k_y y) [2a cosh(kz) + F+ + F-].
    Returns the bracket.
    """
    z = np.asarray(z, dtype=np.float64)
    pre = SQRT_HALF_PI * H / (2.0 * k)
    fp = pre * np.exp(0.5 * k * H * (k * H + 2.0 * z / H)) * special.erf((k * H + z / H) / np.sqrt(2.0))
    fm = pre * np.exp(0.5 * k * H * (k * H - 2.0 * z / H)) * special.erf((k * H - z / H) / np.sqrt(2.0))
    a = -pre * np.exp(0.5 * (k * H) ** 2) * special.erf((k * H + Lz / (2.0 * H)) / np.sqrt(2.0))
    return 2.0 * a * np.cosh(k * z) + fp + fm


def mode_profile_quad(z: float, k: float, H: float, Lz: float):
    """Same bracket by quadrature of the k ≠ 0 Green's function over the box."""
    def f(zp):
        return -np.exp(-k * abs(z - zp)) * np.exp(-zp * zp / (2.0 * H * H)) / (2.0 * k)
    v1 = integrate.quad(f, -0.5 * Lz, z, epsabs=1e-15, epsrel=1e-13, limit=200)[0]
    v2 = integrate.quad(f, z, 0.5 * Lz, epsabs=1e-15, epsrel=1e-13, limit=200)[0]
    return v1 + v2


def green_hat_quad(k: float, kz: float, L: float):
    """∫_{-L}^{L} G_k(z) e^{i k_z z} dz by quadrature (Eq. VGF shearing box).

    G_k is Eq. (Green's function original): ½|z| for k = 0, -e^{-k|z|}/(2k)
    otherwise.  G_k is even, so only the cosine part survives.
    """
    if k == 0.0:
        def f(z):
            return 0.5 * abs(z) * np.cos(kz * z)
    else:
        def f(z):
            return -np.exp(-k * abs(z)) * np.cos(kz * z) / (2.0 * k)
    v = integrate.quad(f, 0.0, L, epsabs=1e-15, epsrel=1e-13, limit=400)[0]
    return 2.0 * v


def paper_norm(eps):
    """‖ε‖₂ = (1/N) √(Σ ε²) over all N cells (Sect. 3.3)."""
    eps = np.asarray(eps, dtype=np.float64)
    return np.sqrt(np.sum(eps * eps)) / eps.size


def rel_l2(a, b):
    """‖a - b‖₂ / ‖b‖₂."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))
