"""CPU FP64 oracle for one T-REXI time step of the linear SWE on the rotating sphere.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the ``librexi`` C-ABI
library and its Python binding) may import, call, link or execute anything in
this package.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

It is a plain, slow, obviously-correct restatement of what the paper computes
(Schreiber & Loft, "A parallel time-integrator for solving the linearized
shallow water equations on the rotating sphere"):

* ``sphere``       -- Gaussian grid, orthonormal associated Legendre functions,
                      scalar and vector spherical-harmonic transforms (Sec. 3).
* ``rexi_coeffs``  -- the T-REXI coefficients (alpha_n, beta_n) from the
                      Gaussian rational approximation and the Gaussian-basis
                      expansion of the exponential, plus the beta
                      renormalisation of Sec. 6.1 (Sec. 4.1, Sec. 6.1).
* ``swe``          -- the linear SWE operator of Eq. (1) in spherical-harmonic
                      space, per zonal order m.
* ``step``         -- one REXI step  U <- sum_k beta_k (alpha_k + tau L)^{-1} U
                      (Sec. 4.2, Algorithm 1) in spectral and grid layouts, and
                      its adjoint.
* ``phi_solver``   -- the paper's own geopotential-only solve per pole (Sec. 4.3
                      and 5): the multiplied-through Phi equation, its Galerkin
                      matrix, velocities recovered in physical space.
* ``integrate``    -- reference integrators for the Gaussian-bump study
                      (Sec. 6.2): RK4, the exact exp(tL), modal REXI steps.

Everything is numpy/scipy in float64 / complex128.  The shifted systems are
solved with LAPACK's banded LU (``scipy.linalg.solve_banded``) on the full
(Phi, zeta, delta) system -- deliberately a different algorithm from the GPU
path's delta-eliminated tridiagonal recurrences.

Parity status per function is stated in each module header.  Every function
here is pinned by a ``-m "not gpu"`` test against something other than itself
(scipy/numpy library reductions, closed forms, dense brute force, invariants),
see ``tests/test_oracle_*.py``.
"""

from . import sphere, rexi_coeffs, swe, step  # noqa: F401
