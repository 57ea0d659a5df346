"""FP64 CPU oracle for the VGF-HybridBC shearing-box Poisson solve (arXiv 2510.10070).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` use it.  It shares no code, table or constant generator with
the CUDA library; the two meet only through the seeded input generators in
``paper_2510_10070_gb300.workloads``, which hold none of the method's
arithmetic.

Every function in :mod:`oracle.vgf` is pinned by the ``-m "not gpu"`` tests
against closed forms, quadrature of the paper's Green's function, a library
FFT definition of the same operator and brute-force invariants; no function is
left parity-unpinned.
"""

from .vgf import (  # noqa: F401
    SolveParams,
    shear_offset,
    signed_index,
    green_hat,
    mode_wavenumbers,
    green_eff,
    vertical_kernel,
    dft_x,
    dft_y,
    inverse_dft_x_half,
    horizontal_dft,
    inverse_horizontal_dft,
    vertical_convolve,
    solve,
    solve_columns,
    solve_at,
    plane_sums,
    k0_potential,
    remap_phase,
    remap_y,
    solve_physical,
    fill_ghosts,
    force,
    green_periodic,
    sasha_mean_terms,
    solve_sasha,
)
