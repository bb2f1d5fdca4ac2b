"""FP64 CPU oracle for the pairwise line-of-sight multipole estimators.

TEST INFRASTRUCTURE ONLY.  Nothing in the product library imports, calls or
links this package; only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.

It is a plain, slow, literal restatement of Philcox & Slepian,
"Beyond Yamamoto" (arXiv:2102.08384), written from the paper in FP64 with
numpy / scipy / sympy primitives, and it shares no code with the CUDA path:

* ``special``    -- Legendre/Gegenbauer coefficients, Gaunt and 3-j symbols,
                    solid-harmonic coupling A (Appendix A, Appendix B eq.
                    solid-harm-application), complex spherical harmonics.
* ``coeffs``     -- the series coefficients phi (Appendix B, eq.
                    shift-coeff-def), f (Appendix E, eq. f-alpha-def) and
                    B (Appendix F, eq. B-def), in the complex basis.
* ``mesh``       -- CIC/TSC painting, mesh/lag/Fourier grids, FKP
                    normalisation and shell binning (Sec. 2).
* ``estimators`` -- the FFT series estimators (O3): Yamamoto, midpoint and
                    bisector P_ell(k) and xi_ell(r) (Secs. 2-6).
* ``pairs``      -- brute-force pair sums: exact pairwise-LOS estimators on
                    the mesh (O2), the truncated series evaluated pair by pair,
                    and the particle pair sum for xi_ell (O1).

Each function cites the section / equation it follows.  Parity status of every
function is stated in its module header.
"""
