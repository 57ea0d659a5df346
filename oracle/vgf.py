"""VGF-HybridBC discrete operator, written out as direct sums in FP64.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares nothing
with the CUDA library.

What it computes (arXiv 2510.10070, Sect. 2.1 and 2.3):

* Sect. 2.1 (unnumbered equation for k(t)): in the periodic frame the
  horizontal wave-vector is k_x = K_x + (Δy0/L_x) K_y, k_y = K_y with
  Δy0 = mod(q Ω L_x t, L_y).  The paper writes q = 3/2.
* Eq. (Helmholtz equation) + Eq. (Green's function original): after an xy
  Fourier transform each column solves a screened Poisson problem with the 1D
  Green's function G_k(z).
* Eq. (Green's function with rect) + Eq. (VGF shearing box) + Eq. (Green's
  function regularized in Fourier), derived in Appendix A: the truncated
  kernel G^L = rect(z/2L) G_k has the closed-form transform Ĝ^L(k, k_z).
* Sect. 2.3, last equation: Φ = 4πG F⁻¹(Ĝ^L · ρ̂), with the density
  zero-padded in z (Sect. 2.4, zero-padding paragraph).

Written as direct sums (no FFT anywhere):

    R(a, b, j)  = Σ_{y,x} ρ̃[j, y, x] exp(-2πi (a x / N_x + b y / N_y))
    c_n(a, b)   = (1/M) Σ_{m=-M/2}^{M/2-1} Ĝ_eff(a, b, m) cos(2π m n / M),
                  |n| ≤ N_z - 1, k_z,m = 2π m / (M dz)
    Φ̂(a, b, i)  = Σ_{j<N_z} c_{i-j}(a, b) R(a, b, j)
    Φ̃[i, y, x]  = 4πG / (N_x N_y) · Re Σ_{a,b} Φ̂(a, b, i) exp(+2πi (...))

Readings of the paper that this module takes (where the paper is silent or garbled):

* padding M = 2 N_z with L = L_z (α = 1); the paper's α = 1.1 needs M = 4 N_z
  and is available through ``SolveParams(pad=4, alpha=1.1)``;
* no dz factor: the transform's dz and the series' 1/(M dz) give 1/M;
* Ĝ_eff = ½[Ĝ(k(a,b)) + Ĝ(k(partner))] with partner = (-a, -b) wrapped into
  the signed range; this equals taking the real part of the full complex
  solve and differs from Ĝ only on the Nyquist planes when sheared;
* k = 0 exactly iff the signed mode is (0, 0) (integer test);
* cell-centred grid, z_k = -L_z/2 + (k + ½) dz.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "SolveParams",
    "shear_offset",
    "signed_index",
    "green_hat",
    "mode_wavenumbers",
    "green_eff",
    "vertical_kernel",
    "dft_x",
    "dft_y",
    "inverse_dft_x_half",
    "horizontal_dft",
    "inverse_horizontal_dft",
    "vertical_convolve",
    "solve",
    "solve_columns",
    "solve_at",
    "plane_sums",
    "k0_potential",
    "remap_phase",
    "remap_y",
    "solve_physical",
    "fill_ghosts",
    "force",
    "green_periodic",
    "sasha_mean_terms",
    "solve_sasha",
]


@dataclass(frozen=True)
class SolveParams:
    """Box and physics parameters of one solve.

    Lx, Ly, Lz : box lengths; the vertical window is [-Lz/2, Lz/2] (Sect. 3.1).
    q, Omega   : shear rate q·Ω (Sect. 2.1 uses q = 3/2).
    G          : gravitational constant in ∇²Φ = 4πGρ (Eq. Poisson).
    pad        : vertical zero-padding factor, M = pad · Nz.
    alpha      : enclosure factor, L = alpha · Lz (Eq. Green's function with rect).
    """

    Lx: float
    Ly: float
    Lz: float
    q: float = 1.5
    Omega: float = 1.0
    G: float = 1.0
    pad: int = 2
    alpha: float = 1.0


def shear_offset(q: float, Omega: float, Lx: float, Ly: float, t: float) -> float:
    """Δy0(t) = mod(q Ω L_x t, L_y), taken into [0, L_y) (Sect. 2.1)."""
    dy0 = math.fmod(q * Omega * Lx * t, Ly)
    if dy0 < 0.0:
        dy0 += Ly
    if dy0 >= Ly:
        dy0 -= Ly
    return dy0


def signed_index(i, n: int):
    """Map an FFT index i ∈ [0, n) to the signed range [-n/2, n/2)."""
    i = np.asarray(i)
    return np.where(i < n // 2, i, i - n)


def green_hat(k, kz, L: float, k_is_zero):
    """Ĝ^L(k, k_z) of Eq. (Green's function regularized in Fourier).

    Three cases, exactly as printed (Appendix A derives them):
      k = 0, k_z = 0 : L²/2
      k = 0, k_z ≠ 0 : [k_z L sin(k_z L) + cos(k_z L) - 1] / k_z²
      otherwise      : -[e^{-kL} ((k_z/k) sin(k_z L) - cos(k_z L)) + 1] / (k² + k_z²)
    ``k_is_zero`` selects the k = 0 branches (an exact integer test upstream).
    """
    k = np.asarray(k, dtype=np.float64)
    kz = np.asarray(kz, dtype=np.float64)
    k, kz, zero_k = np.broadcast_arrays(k, kz, np.asarray(k_is_zero, dtype=bool))
    out = np.empty(k.shape, dtype=np.float64)

    both_zero = zero_k & (kz == 0.0)
    out[both_zero] = 0.5 * L * L

    only_k_zero = zero_k & (kz != 0.0)
    q = kz[only_k_zero]
    out[only_k_zero] = (q * L * np.sin(q * L) + np.cos(q * L) - 1.0) / (q * q)

    screened = ~zero_k
    kk = k[screened]
    q = kz[screened]
    e = np.exp(-kk * L)
    out[screened] = -(e * ((q / kk) * np.sin(q * L) - np.cos(q * L)) + 1.0) / (kk * kk + q * q)
    return out


def mode_wavenumbers(nx: int, ny: int, Lx: float, Ly: float, s: float):
    """Sheared |k| for every horizontal mode and for its Hermitian partner.

    Returns (k1, k2, is_zero), each of shape [ny, nx] indexed by the unsigned
    FFT indices (b, a).  K = (2π a_s/L_x, 2π b_s/L_y) with signed (a_s, b_s);
    k_x = K_x + s K_y with s = Δy0/L_x (Sect. 2.1).  The partner is
    (wrap(-a_s), wrap(-b_s)), which differs from (-a_s, -b_s) only on the
    Nyquist planes a_s = -N_x/2 or b_s = -N_y/2.
    """
    a = signed_index(np.arange(nx), nx).astype(np.float64)
    b = signed_index(np.arange(ny), ny).astype(np.float64)
    a2 = signed_index((-signed_index(np.arange(nx), nx)) % nx, nx).astype(np.float64)
    b2 = signed_index((-signed_index(np.arange(ny), ny)) % ny, ny).astype(np.float64)

    def kabs(av, bv):
        Kx = 2.0 * np.pi * av / Lx
        Ky = 2.0 * np.pi * bv / Ly
        kx = Kx[None, :] + s * Ky[:, None]
        return np.sqrt(kx * kx + (Ky * Ky)[:, None])

    k1 = kabs(a, b)
    k2 = kabs(a2, b2)
    is_zero = (a[None, :] == 0.0) & (b[:, None] == 0.0)
    return k1, k2, is_zero


def _kz_signed(nz: int, Lz: float, pad: int):
    """Signed vertical indices m ∈ [-M/2, M/2) and k_z,m = 2π m / (M dz)."""
    M = pad * nz
    dz = Lz / nz
    m = np.arange(-(M // 2), M // 2)
    return m, 2.0 * np.pi * m / (M * dz)


def green_eff(nx: int, ny: int, nz: int, p: SolveParams, t: float):
    """Ĝ_eff(b, a, m) = ½[Ĝ(k1, k_z,m) + Ĝ(k2, k_z,m)] over signed m ∈ [-M/2, M/2).

    Shape [ny, nx, M]; the last axis runs over m = -M/2 .. M/2-1.
    """
    s = shear_offset(p.q, p.Omega, p.Lx, p.Ly, t) / p.Lx
    k1, k2, is_zero = mode_wavenumbers(nx, ny, p.Lx, p.Ly, s)
    _, kz = _kz_signed(nz, p.Lz, p.pad)
    L = p.alpha * p.Lz
    g1 = green_hat(k1[..., None], kz[None, None, :], L, is_zero[..., None])
    g2 = green_hat(k2[..., None], kz[None, None, :], L, is_zero[..., None])
    return 0.5 * (g1 + g2)


def vertical_kernel(geff, nz: int, pad: int = 2):
    """c_n = (1/M) Σ_m Ĝ_eff(m) cos(2π m n / M) for n = -(nz-1) .. nz-1.

    A naive inverse DFT of the real, even kernel samples (its sine part
    cancels pairwise).  Input shape [..., M]; output shape [2 nz - 1, ...]
    with row n + nz - 1 holding c_n.
    """
    M = pad * nz
    m = np.arange(-(M // 2), M // 2)
    n = np.arange(-(nz - 1), nz)
    phase = np.mod(np.outer(m, n), M)  # exact integer argument reduction
    cosmat = np.cos(2.0 * np.pi * phase / M)  # [M, 2nz-1]
    c = (geff @ cosmat) / M  # [..., 2nz-1]
    return np.moveaxis(c, -1, 0).copy()


def _dft_matrix(n: int, sign: float):
    idx = np.arange(n)
    phase = np.mod(np.outer(idx, idx), n)
    return np.exp(sign * 2j * np.pi * phase / n)


def dft_x(rho):
    """Naive DFT along x of real rows: X[j, y, a] for a ∈ [0, nx/2] (half spectrum)."""
    rho = np.asarray(rho, dtype=np.float64)
    nx = rho.shape[-1]
    F = _dft_matrix(nx, -1.0)[: nx // 2 + 1]  # [a, x]
    return rho @ F.T


def dft_y(X, sign: float = -1.0):
    """Naive DFT along y (axis -2) of complex data, exp(sign·2πi b y / ny)."""
    ny = X.shape[-2]
    F = _dft_matrix(ny, sign)  # [b, y]
    return np.einsum("by,...ya->...ba", F, X)


def inverse_dft_x_half(X, nx: int):
    """Real rows from a half spectrum X[..., a], a ≤ nx/2, by the Hermitian sum.

    φ[x] = Σ_{a=0}^{nx-1} X̃[a] exp(+2πi a x/nx) with X̃[a] = X[a] for a ≤ nx/2
    and X̃[a] = conj(X[nx-a]) above; the a = 0 and a = nx/2 terms use their
    real parts only (they are real for any Hermitian spectrum).  Unscaled.
    """
    h = nx // 2 + 1
    X = np.array(X[..., :h], dtype=np.complex128)
    X[..., 0] = X[..., 0].real
    X[..., nx // 2] = X[..., nx // 2].real
    full = np.concatenate([X, np.conj(X[..., 1:nx // 2][..., ::-1])], axis=-1)
    F = _dft_matrix(nx, +1.0)  # [x, a]
    return (full @ F.T).real


def horizontal_dft(rho):
    """R[j, b, a] = Σ_{y,x} ρ[j, y, x] exp(-2πi (a x/nx + b y/ny)) over all (a, b)."""
    rho = np.asarray(rho, dtype=np.float64)
    nx = rho.shape[-1]
    Fx = _dft_matrix(nx, -1.0)
    return dft_y(rho @ Fx.T)


def inverse_horizontal_dft(phat):
    """Re of (1/(nx ny)) Σ_{a,b} Φ̂[i, b, a] exp(+2πi (a x/nx + b y/ny))."""
    ny, nx = phat.shape[-2:]
    Fx = _dft_matrix(nx, +1.0)
    out = dft_y(phat, +1.0) @ Fx.T
    return out.real / (nx * ny)


def vertical_convolve(c, R):
    """Φ̂[i, ...] = Σ_{j<nz} c_{i-j}[...] R[j, ...] (linear Toeplitz sum).

    ``c`` has shape [2nz-1, ...] (row n + nz - 1 = c_n); ``R`` has [nz, ...].
    For each output row i the sum over j is one vectorised product-sum.
    """
    nz = R.shape[0]
    out = np.zeros(R.shape, dtype=np.result_type(c, R))
    j = np.arange(nz)
    for i in range(nz):
        out[i] = np.sum(c[i - j + nz - 1] * R, axis=0)
    return out


def solve_columns(R, p: SolveParams, t: float):
    """The vertical step only: Φ̂(a, b, i) = Σ_j c_{i-j}(a, b) R(a, b, j).

    ``R`` is the full horizontal spectrum [nz, ny, nx] (unsigned (b, a)).
    """
    nz, ny, nx = R.shape
    c = vertical_kernel(green_eff(nx, ny, nz, p, t), nz, p.pad)  # [2nz-1, ny, nx]
    return vertical_convolve(c, R)


def solve(rho, p: SolveParams, t: float):
    """Φ̃ on the physical grid for density ρ̃ [nz, ny, nx] in the periodic frame."""
    rho = np.asarray(rho, dtype=np.float64)
    R = horizontal_dft(rho)
    phat = solve_columns(R, p, t)
    return 4.0 * np.pi * p.G * inverse_horizontal_dft(phat)


def solve_at(rho, p: SolveParams, t: float, points):
    """Φ̃ at sampled cells ``points`` = iterable of (i, y, x), one by one.

    Uses the full horizontal spectrum and kernel, then for each sample the
    direct sums over j and over (a, b).
    """
    rho = np.asarray(rho, dtype=np.float64)
    nz, ny, nx = rho.shape
    R = horizontal_dft(rho)
    c = vertical_kernel(green_eff(nx, ny, nz, p, t), nz, p.pad)
    a = np.arange(nx)
    b = np.arange(ny)
    out = []
    cache = {}
    for (i, y, x) in points:
        if i not in cache:
            acc = np.zeros((ny, nx), dtype=np.complex128)
            for j in range(nz):
                acc += c[i - j + nz - 1] * R[j]
            cache[i] = acc
        ph = np.exp(2j * np.pi * (np.mod(b * y, ny)[:, None] / ny + np.mod(a * x, nx)[None, :] / nx))
        val = np.sum(cache[i] * ph).real / (nx * ny)
        out.append(4.0 * np.pi * p.G * val)
    return np.array(out)


def plane_sums(rho):
    """S[j] = Σ_{y,x} ρ[j, y, x]: the (0, 0) horizontal mode of each plane."""
    rho = np.asarray(rho, dtype=np.float64)
    return np.array([math.fsum(plane.ravel()) for plane in rho])


def k0_potential(S, nx: int, ny: int, nz: int, p: SolveParams):
    """Contribution of the k = 0 mode: 4πG/(nx ny) Σ_j c00_{i-j} S[j].

    c00 is the vertical kernel of the (0, 0) mode (no shear dependence).
    """
    _, kz = _kz_signed(nz, p.Lz, p.pad)
    g = green_hat(np.zeros_like(kz), kz, p.alpha * p.Lz, np.ones(kz.shape, dtype=bool))
    c = vertical_kernel(g, nz, p.pad)  # [2nz-1]
    out = np.zeros(nz)
    for i in range(nz):
        out[i] = sum(c[i - j + nz - 1] * S[j] for j in range(nz))
    return 4.0 * np.pi * p.G * out / (nx * ny)


# ---------------------------------------------------------------------------
# Mapping to the periodic frame (Sect. 2.1: "Mapping to fully periodic
# points", spectral variant, i.e. shear advection by Fourier interpolation).
#
# The k(t) of Sect. 2.1 (k_x = K_x + (Δy0/L_x) K_y) is the wave-vector of a
# field f that obeys f(x + L_x, y) = f(x, y + Δy0) seen through the frame
# f̃(x, y) = f(x, y - s x), s = Δy0/L_x: f̃ is periodic in x, and a periodic-
# frame mode exp(i(K_x x + K_y y)) is the physical mode with k_x = K_x + s K_y.
# Step 1 of the scheme maps ρ → ρ̃, step 2 solves for Φ̃ (``solve``), step 3
# maps Φ̃ back: Φ(x, y) = Φ̃(x, y + s x).  Each x-column is shifted in y by a
# Fourier interpolation; x is the cell centre -L_x/2 + (i + ½) dx (any other
# origin only translates ρ̃ and Φ̃ in y, which cancels between steps 1 and 3).
# The Nyquist coefficient (K_y = -π N_y/L_y) is multiplied by the real part of
# its phase factor (the same reading as Ĝ_eff on the Nyquist planes): the
# shifted column stays real.
# ---------------------------------------------------------------------------

def remap_phase(nx: int, Lx: float, Ly: float, dy0: float):
    """u_i = s x_i / L_y = (Δy0/L_y)(x_i/L_x) for every cell centre x_i (shape [nx])."""
    xi = (np.arange(nx) + 0.5) / nx - 0.5
    return (dy0 / Ly) * xi


def remap_y(f, u, sign: float):
    """Shift every x-column of f [..., ny, nx] by sign·u_x·L_y in y.

    sign = -1 maps the physical frame to the periodic one (ρ̃(x, y) = ρ(x, y - s x)),
    sign = +1 maps back.  Naive DFT along y, coefficient K_y(b) multiplied by
    exp(sign·2πi b_s u_x) (b_s signed, |b_s| < ny/2) and by cos(π ny u_x) on the
    Nyquist row, then the naive inverse DFT; the result is real.
    """
    f = np.asarray(f, dtype=np.float64)
    ny, nx = f.shape[-2], f.shape[-1]
    u = np.asarray(u, dtype=np.float64)
    F = np.einsum("by,...yx->...bx", _dft_matrix(ny, -1.0), f)
    bs = signed_index(np.arange(ny), ny).astype(np.float64)
    ph = np.exp(sign * 2j * np.pi * np.outer(bs, u))  # [ny, nx]
    if ny % 2 == 0:
        ph[ny // 2, :] = np.cos(np.pi * ny * u)
    F = F * ph
    g = np.einsum("yb,...bx->...yx", _dft_matrix(ny, +1.0), F) / ny
    return g.real.copy()


def solve_physical(rho, p: SolveParams, t: float):
    """Φ in the physical (shearing) frame for a physical-frame density ρ [nz, ny, nx].

    The three steps of Sect. 2.1 in order: map ρ to the periodic frame, solve
    there (``solve``), map Φ̃ back.
    """
    rho = np.asarray(rho, dtype=np.float64)
    nz, ny, nx = rho.shape
    u = remap_phase(nx, p.Lx, p.Ly, shear_offset(p.q, p.Omega, p.Lx, p.Ly, t))
    rho_t = remap_y(rho, u, -1.0)
    phi_t = solve(rho_t, p, t)
    return remap_y(phi_t, u, +1.0)


# ---------------------------------------------------------------------------
# Ghost cells and forces (Sect. 2.4, last paragraph): beyond the last active
# cell in z the potential keeps that cell's gradient, i.e. the ghost layers
# continue Φ linearly.  The force g = -∇Φ uses second-order central
# differences; in z the ghost rule makes them one-sided in the boundary cells.
# Horizontally Φ is periodic in y and, in x, periodic in the periodic frame or
# shear-periodic in the physical frame: Φ(x + L_x, y) = Φ(x, y + Δy0), the
# shifted neighbour column taken by the same Fourier interpolation as the
# mapping of Sect. 2.1.
# ---------------------------------------------------------------------------

def fill_ghosts(phi, ng: int):
    """[nz + 2 ng, ny, nx]: phi in the middle, ng linearly continued layers on each side."""
    phi = np.asarray(phi, dtype=np.float64)
    nz = phi.shape[0]
    out = np.empty((nz + 2 * ng,) + phi.shape[1:], dtype=np.float64)
    out[ng:ng + nz] = phi
    top = phi[nz - 1] - phi[nz - 2]  # gradient of the last active cell (per dz)
    bot = phi[1] - phi[0]
    for g in range(1, ng + 1):
        out[ng + nz - 1 + g] = phi[nz - 1] + g * top
        out[ng - g] = phi[0] - g * bot
    return out


def force(phi, p: SolveParams, t: float, physical: bool):
    """g = -∇Φ, shape [3, nz, ny, nx] (x, y, z components), at the cell centres."""
    phi = np.asarray(phi, dtype=np.float64)
    nz, ny, nx = phi.shape
    dx, dy, dz = p.Lx / nx, p.Ly / ny, p.Lz / nz
    right = np.roll(phi, -1, axis=2)  # Φ(x + dx)
    left = np.roll(phi, 1, axis=2)  # Φ(x - dx)
    if physical:
        dy0 = shear_offset(p.q, p.Omega, p.Lx, p.Ly, t)
        # neighbour of the last column: Φ(x_0 + L_x, y) = Φ(x_0, y + Δy0)
        right[:, :, nx - 1] = remap_y(phi[:, :, 0:1], np.array([dy0 / p.Ly]), +1.0)[:, :, 0]
        # neighbour of the first column: Φ(x_{nx-1} - L_x, y) = Φ(x_{nx-1}, y - Δy0)
        left[:, :, 0] = remap_y(phi[:, :, nx - 1:nx], np.array([dy0 / p.Ly]), -1.0)[:, :, 0]
    gx = -(right - left) / (2.0 * dx)
    gy = -(np.roll(phi, -1, axis=1) - np.roll(phi, 1, axis=1)) / (2.0 * dy)
    ext = fill_ghosts(phi, 1)
    gz = -(ext[2:] - ext[:-2]) / (2.0 * dz)
    return np.stack([gx, gy, gz])


# ---------------------------------------------------------------------------
# SASHA (Sect. 2.2): Φ = Φ0 + Φ_P.  Φ0(z) = 4πG ρ̄ z (z/2 - z0) solves
# ∇²Φ0 = 4πG ρ̄ (ρ̄ the volume mean, z0 = <z ρ>/<ρ> the centre of mass);
# Φ_P solves ∇²Φ_P = 4πG (ρ - ρ̄) spectrally, Eq. (Poisson spectral)
# Φ̂ = -4πG ρ̂/|k|² (0 at k = 0), with the density zero-padded in z to 2 nz
# (Sect. 2.4, zero-padding paragraph) and k = (k_x(t), k_y, k_z) of the padded
# grid.  Readings: the volume averages are cell sums over the box; z is the
# cell centre measured from the box centre (another origin changes Φ by a
# constant); z0 = 0 when the total mass is zero; on the sheared Nyquist planes
# the kernel is averaged with the Hermitian partner, as for VGF.
#
# The printed Φ0 and the reported accuracy disagree for off-centre mass: the
# periodic solve on 2 L_z gives Φ_P the edge slope 4πG ρ̄ z0 / 2 (half of what
# the vacuum condition Φ'(L_z/2) = -Φ'(-L_z/2) needs with the printed Φ0), so
# Φ keeps a uniform field: a residual -2πG ρ̄ z0 z.  ``centre`` selects the
# vertex of Φ0: 1 is the printed form (vertex at z0), 1/2 puts it at z0/2,
# which cancels the residual and gives the third-order 1D convergence that
# Sect. 3.3 reports for the shifted Gaussian.
# ---------------------------------------------------------------------------

def green_periodic(k, kz, k_is_zero):
    """-1/(k² + k_z²) of Eq. (Poisson spectral), 0 at k = 0, k_z = 0."""
    k = np.asarray(k, dtype=np.float64)
    kz = np.asarray(kz, dtype=np.float64)
    k, kz, zero_k = np.broadcast_arrays(k, kz, np.asarray(k_is_zero, dtype=bool))
    den = k * k + kz * kz
    out = np.zeros(k.shape, dtype=np.float64)
    nz_ = ~(zero_k & (kz == 0.0))
    out[nz_] = -1.0 / den[nz_]
    return out


def sasha_mean_terms(rho, Lz: float):
    """(ρ̄, z0) of Sect. 2.2 from cell sums; z = cell centres from the box centre."""
    rho = np.asarray(rho, dtype=np.float64)
    nz = rho.shape[0]
    S = plane_sums(rho)
    z = (np.arange(nz) + 0.5) * (Lz / nz) - 0.5 * Lz
    total = math.fsum(S)
    rbar = total / rho.size
    z0 = math.fsum(z * S) / total if total != 0.0 else 0.0
    return rbar, z0


def solve_sasha(rho, p: SolveParams, t: float, centre: float = 1.0):
    """Φ̃ by SASHA for a periodic-frame density ρ̃ [nz, ny, nx] (pad = 2 nz).

    Φ0 = 4πG ρ̄ z (z/2 - centre·z0).
    """
    rho = np.asarray(rho, dtype=np.float64)
    nz, ny, nx = rho.shape
    rbar, z0 = sasha_mean_terms(rho, p.Lz)
    R = horizontal_dft(rho - rbar)
    s = shear_offset(p.q, p.Omega, p.Lx, p.Ly, t) / p.Lx
    k1, k2, is_zero = mode_wavenumbers(nx, ny, p.Lx, p.Ly, s)
    _, kz = _kz_signed(nz, p.Lz, 2)
    g1 = green_periodic(k1[..., None], kz[None, None, :], is_zero[..., None])
    g2 = green_periodic(k2[..., None], kz[None, None, :], is_zero[..., None])
    c = vertical_kernel(0.5 * (g1 + g2), nz, 2)
    phi_p = 4.0 * np.pi * p.G * inverse_horizontal_dft(vertical_convolve(c, R))
    z = (np.arange(nz) + 0.5) * (p.Lz / nz) - 0.5 * p.Lz
    phi0 = 4.0 * np.pi * p.G * rbar * z * (0.5 * z - centre * z0)
    return phi_p + phi0[:, None, None]
