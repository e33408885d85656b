"""Plain FP64 CPU oracle for the FE spinor ChFSI hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its ``cpu_baseline`` leg and ``--impl reference`` arm) may import
anything from this package.  The product path (the CUDA library and its
Python binding) never imports it and shares no code with it.

What it computes (each function cites the passage it follows):

* ``fe``      -- GLL/Gauss tables, Lagrange basis, the structured hex mesh, the
                 assembled complex Hermitian H^k = H^loc + H^nloc (Eqs. FEHloc,
                 FEHnloc, CMat) as an explicit sparse matrix (form O1a) and as an
                 element-by-element quadrature apply (form O1b), and the lumped
                 GLL mass M_D (Sec. III.B.2).
* ``chfsi``   -- the scaled Chebyshev filter on M_D^-1 H (Eq. chebfilt), the
                 generalised Lanczos bounds, Cholesky-Gram-Schmidt, Rayleigh-Ritz
                 with an own cyclic Jacobi Hermitian eigensolver, the ChFSI cycle,
                 the residual-split form of the filter, dense brute force.
* ``grad``    -- reverse-mode gradients of L = sum_i w_i y_i^H H y_i through
                 the filter.
* ``density`` -- electron density rho and magnetisation density m at the Gauss
                 points from an occupied spinor block (Eqs. rho, mag), and
                 Fermi-Dirac occupations with the electron-count chemical potential.
* ``twogrid`` -- transfer of a block from FE order p_c to p_f >= p_c on the same
                 mesh by nodal interpolation (Eq. FEWfnsCMesh, two-grid strategy).
* ``scf``     -- the SCF pieces around the eigensolver: an exchange-only local spin
                 density stand-in for V_xc / B_xc (closed form), the density inner
                 product (Eq. innerPdt) and Anderson mixing.

Parity status: every function is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_pins.py``, ``tests/test_oracle_grad.py``,
``tests/test_oracle_density.py``, ``tests/test_oracle_twogrid.py`` and
``tests/test_oracle_scf.py`` except the residual-split reformulation's
relation to the authors' unpublished variant ("parity unpinned" for that
relation only; its exact equality with the direct filter is pinned).
"""
