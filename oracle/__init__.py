"""Plain FP64 CPU oracle for the hybrid nodal-staggered PSATD PIC step.

TEST INFRASTRUCTURE ONLY.  This package is a slow, direct restatement of the
method of Zoni et al., "A Hybrid Nodal-Staggered Pseudo-Spectral
Electromagnetic Particle-In-Cell Method with Finite-Order Centering"
(arXiv 2106.12919), written to check the CUDA path.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import it.  The product path never does, and the oracle never
imports the product package: the two share no code.

Every function follows the paper's notation and cites the section / equation it
restates.  Loops are vectorised over particles or grid points only; there is no
blocking, fusion or reordering beyond what the cited definitions state.

Modules
-------
fornberg     Fornberg coefficients, modified wave numbers, centering symbol
             (Sec. 3, Sec. 4.1, App. C).
grid         Yee staggering, discrete Fourier conventions (App. A.1) and the
             finite-order centering stencils (Sec. 3, Eq. staggered_finite_sum).
psatd        Standard / Galilean / averaged-Galilean PSATD coefficients and
             k-space updates (Sec. 4.2-4.4).
particles    B-spline shapes, gather, Boris push, direct deposition, tile bins.
step         The hybrid PIC cycle of Sec. 2 (and its comparison and FDTD cycles).
fdtd         Yee finite-difference Maxwell solver of order 2m (the FDTD form of the
             hybrid scheme, Sec. 6).
diagnostics  Field energy (Sec. 2 (iii)), the L2 error norm (Sec. 5.2), the stencil
             extent (Eq. stencil_extent), the beam RMS (Eq. RMS_pwfa) and the numerical
             vacuum dispersion of an update (Sec. 2 (i), App. B).

Parity status: every function is pinned by tests/test_oracle_*.py against
closed forms, brute force or invariants.  The full multi-step cycle has no
closed form; it is pinned by the pins of each of its stages, by invariants
(charge, vacuum energy, the cold-plasma oscillation at omega_p) and by exact
symmetries of the method that the whole cycle must keep (mirror reflection,
exchange of two axes, translation by a cell: tests/test_oracle_symmetry.py).
"""
