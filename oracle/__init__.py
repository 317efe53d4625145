"""Plain FP64 CPU oracle for phase-averaged rotating shallow water on the sphere.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) may import, call or link this package; only the tests,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` use it.  It shares no code, table or constant generator
with the CUDA path.

It follows Yamazaki, Cotter & Wingate, "Time parallel integration and phase
averaging for the nonlinear shallow water equations on the sphere"
(arXiv 2103.07706):

* ``mesh``       icosahedral sphere mesh (Sec. 3, mesh paragraph)
* ``quadrature`` Gauss rules on the reference triangle and interval
* ``elements``   reference BDM2 / DG1 elements (Sec. 2.5)
* ``assembly``   cell geometry, element matrices, global sparse M1, C, D, M2
                 (Sec. 2.5, Eq. ueq_int and the following eta equation)
* ``operators``  the discrete linear operator L and nonlinear operator N
                 (Sec. 2.5), energy and mass diagnostics
* ``expo``       Chebyshev exponential with FFT coefficients and magnitude
                 truncation (Sec. 2.4, Eq. cheby)
* ``averaging``  bump weight and Riemann-sum phase average (Sec. 2.2,
                 Eq. vt_averaged, Eq. vt_discretised), in its literal
                 per-shift form
* ``timestep``   averaged Lawson RK4 (Sec. 2.3, Eqs. stage1_c to stage4)
* ``spectrum``   lambda_max of L by power iteration (Sec. 2.4)
* ``model``      one object bundling all of the above for one mesh

Every mass-matrix solve is a sparse direct factorisation (scipy splu), so the
oracle's linear algebra is exact up to rounding.
"""


