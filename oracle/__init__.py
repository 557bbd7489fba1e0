"""Plain FP64 CPU oracle for the Contour-FFT (C-FFT) MBF reaction tables.

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
or execute it.  The GPU product path never calls into it, and it never calls
into the GPU product path: the two share no code, no constants and no helpers.
The only module both sides use is ``workloads`` (seeded synthetic inputs, no
arithmetic of the method).

Everything here is written from the paper's definitions, in the paper's order:

* ``contour``   -- the parabolic deformation of the radial spectral variable
                   (Eq. 8, Fig. 1) sampled with the rectangle rule.
* ``green``     -- the grounded-slab spectral dyadic Green's function (the paper
                   cites it but does not print it; the standard TE/TM form for a
                   horizontal electric current on a grounded slab is used).
* ``spectra``   -- Fourier transforms of the elementary basis functions
                   (rooftops, the analytic strip dipole) and of MBFs (Eq. 11).
* ``reaction``  -- the MBF spectral kernel (Eq. 10), its azimuthal harmonics,
                   and the reaction table Z_q(rho) of Eq. 9 evaluated by direct
                   quadrature: the Bessel form ("O2", matched contour nodes),
                   the alpha form with exact exponentials, and an adaptive
                   quadrature along the contour ("O1", converged).
* ``fill``      -- exact per-entry evaluation of the reduced matrix Z' (Eq. 3
                   restated per element pair through Eq. 9).
* ``solve``     -- the reduced system of Section II: excitation V' = Q^H V
                   (Eq. 4), a direct solution of Z' I' = V', the currents
                   I = Q I' and the port currents of delta-gap excitations.
* ``cartesian`` -- the paper's own 2-D form (Section III-B-2/3, Eq. 21-24,
                   Appendix I): the kernel at the complex extension
                   k (1 + i gamma) on a real (kx, ky) grid, one FFT2 per Taylor
                   monomial with Appendix I's signs, the zero-padded 2x
                   refinement, second-order interpolation.

All arithmetic is numpy/scipy float64 / complex128.  Nothing here is blocked,
fused or reordered beyond the definitions; speed is not a goal.

Parity pins (what this oracle is checked against, in ``tests/test_oracle_*``):
closed forms (Gaussian Hankel pair, 2-D Gaussian Fourier pair, rooftop/strip
transforms by brute-force spatial quadrature), textbook surface-wave
dispersion relations, contour independence by Cauchy, real-axis quadrature
with surface-wave pole extraction, reciprocity and rotation symmetries; the
Cartesian form against a closed form, the direct sum of its own definition
and convergence to the polar integral.
"""
