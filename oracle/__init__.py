"""FP64 CPU oracle for the SIPG viscous and Poisson operators (test infrastructure).

This package is test infrastructure, not part of the product. Only the test
suite, the smoke check in ``__graft_entry__`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it. The CUDA library never
calls into it and it never calls into the CUDA library: the two share no code.

Everything here is plain, slow and written to be checked against the paper by
eye (arXiv 2506.14424, "Higher-order discontinuous Galerkin splitting schemes
for fluids with variable viscosity"):

* ``quadrature``   Gauss-Legendre and Gauss-Lobatto rules (Newton on Legendre
                   polynomials), Sec. 5 (discrete spaces Q_k on hexahedra).
* ``basis``        Lagrange polynomials on the Gauss-Lobatto nodes.
* ``mesh``         structured box of affine hexahedra, Sec. 5.
* ``viscosity``    Eq. (viscosity_general) law, shear rate of Sec. 2, the
                   analytic field and the sphere ("sinker") field.
* ``sipg``         the element form of Eq. (viscous_term_weak) with the SIPG
                   fluxes of Sec. 5.2 and the pressure form of
                   Eq. (pressure_step_weak), assembled as explicit blocks.
* ``solvers``      CG / Jacobi-PCG / dense Cholesky on the assembled matrix.
* ``multigrid``    transfers, inverse diagonal, Chebyshev-Jacobi smoother and
                   V-cycle of Sec. 5.4 (matrix-free preconditioners).
* ``cph``          continuous multigrid levels below the DG level: injection,
                   Galerkin operators, composed transfers (Sec. 5.4).
* ``manufactured`` body-force loads for manufactured solutions (Sec. 7.1).
* ``mass``         element mass matrices (v, u)_e and their inverses (Sec. 3.2,
                   Eqs. convective_step_weak / projection_step_weak).
* ``nonlinear``    Picard iteration of the viscosity with Aitken relaxation
                   (Sec. 5.4, Alg. 1).
* ``mapped``       the SIPG operators on trilinear (non-affine) hexahedra:
                   per-point Jacobians, normals and surface weights (Sec. 5).
* ``splitting``    one step of the projection scheme on a box: BDF, explicit
                   convective step, pressure Poisson step with the consistent
                   Neumann datum, projection, viscous step, CFL time step
                   (Sec. 3.2 / 5.1, Alg. 1).

Parity status: see the header of each module. The multigrid V-cycle as a whole
is "parity unpinned" against the paper (the paper prints no iteration counts
for this problem); its pieces are pinned individually.
"""
