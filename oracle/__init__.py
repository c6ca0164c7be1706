"""Plain FP64 CPU oracle of the FSIB time step (Chen & Peskin, arXiv 2302.08694).

TEST INFRASTRUCTURE ONLY. This package is the slow, obviously correct statement
of what the GPU library computes. Only the test suite, the smoke check and the
CPU-baseline leg of the benchmark import it. The library's product path never
imports, links or runs anything here, and this package shares no code with it.

What the oracle computes (no NUFFT, no fine grid, no spreading kernel):

* spectral.py   - the truncated mode set (Eq. kNh), the direct type-1 and
                  type-2 sums (Eqs. force_spreading_quad and velo_intp_fini),
                  the Stokeslet (Eq. stokeslet), the Leray projection and V-hat
                  (Eq. fourier_spectral_sol, Algorithm 2), the dealiased
                  nonlinear term by the three-halves rule (Eq. nonlinear_kspace),
                  and the backward-Euler / Crank-Nicolson substeps (Eqs.
                  spatial_2, spatial_3).
* lagrangian.py - force laws (Eq. elstic_force_2d; the cot-weight spring
                  membrane of Sec. 6.2.3), their energies, and the enclosed
                  area / volume.
* stepper.py    - the time step of Algorithm 1 (Eqs. spatial_1 to spatial_4)
                  and the quasi-static Stokes stepper.

Readings of the paper that the oracle fixes (the paper is silent or ambiguous):

* Even N: every mode with some m_a = -N/2 (the unpaired Nyquist mode) is set
  to zero in f-hat, u-hat and s-hat, so that the mode set is symmetric and the
  interpolated velocity is real.
* Wavenumbers are physical: k = 2*pi*m/L.
* The spread includes both the quadrature weight and the 1/L^d factor of Eq.
  force_spreading_quad.
* Dealiasing uses N~ = 3N/2 (enough for even N, see spectral.nonlinear).
* Algorithm 1's U^{m+1} is interpolated at X^{m+1}, after the position update.
* Quasi-static Stokes uses the same midpoint rule in time as Eqs. spatial_1/4.
* The enclosed volume is (1/6) sum X_i . (X_j x X_k) over ccw triangles; the
  formula as printed in Sec. 6.2.3 is identically zero.

All functions are parity-pinned by tests/test_oracle_*.py (-m "not gpu"):
nothing here is "parity unpinned".
"""
