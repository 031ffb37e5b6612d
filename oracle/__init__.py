"""Plain FP64 CPU oracle for the Laplacian-preconditioned Schur solve of the
SIMPLE-based direct-forcing immersed boundary method (arXiv 2501.15314).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute anything in this package: only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.
It shares no code with the CUDA library; both sides receive the same seeded
inputs from ``paper_2501_15314_gb300.workloads``, which holds no arithmetic of
the method.

Equations are cited by the label they carry in the paper's source, sections
by number (2.3 = "Interpolation and regularization operators", 3.1 = "One-way
coupled moving boundary", 4.1 = "The Laplacian as a preconditioner",
4.2 = "Efficient matrix-free implementation", 5 = the spectral theorem,
6.2 = "Preconditioner efficiency", Appendix A = grid-spacing study).

Modules:

* ``mac``        staggered MAC grid, G, G^T = -div, L = G^T G (Sec. 3.1 and
                 Fig. "cell"; Eq. (Saddle)), exact Neumann L^+ by the cosine
                 transform (the uniform-grid form of the fast diagonalisation
                 the paper uses as its Laplacian solver, Sec. 4.2).
* ``delta``      Roma's 3-point discrete delta (Eq. (delta)) and the
                 regularisation / interpolation operators R, R^T
                 (Eqs. (interpolation), (regularization)).
* ``schur``      the saddle system (Eq. (Saddle)), the primal Schur complement
                 (Eqs. (SchurPrimal)-(SchurPrimalF)), its scalar approximation
                 (Eqs. (tildeSp)-(ApproxSchurPrimalF)); dense and Krylov solves.
* ``helmholtz``  the BDF2 momentum predictor (Eq. (ustar)): exact sine-transform
                 solve of (3/(2 dt) - nu Lap) u* = rhs on the no-slip MAC grid.
* ``step``       one one-way time step: predictor, correction RHS, Schur solve,
                 force recovery, update (Eqs. (ustar)-(Saddle),
                 (ApproxSchurPrimalP), (ApproxSchurPrimalF), (u_n_plus_1)) and
                 the force/torque diagnostics (Eq. (IBM_force)).
* ``fsi``        two-way coupled rigid spheres (Sec. 3.2): position and
                 Rodrigues orientation prediction, Newton's laws in BDF2 form
                 (Eqs. (bdy_linear_vel_iter), (bdy_angular_vel_iter)) with the
                 enclosed-fluid momentum from volume fractions
                 (Eq. (volume_integrals)), the relaxed correction loop with
                 its L1 stopping rule (Eq. (convergence_criterion)).
* ``adjoint``    reverse-mode derivative of that step and of the body force /
                 torque sums with respect to U^Gamma and the marker positions
                 (through phi', the derivative of Eq. (delta)); the paper has
                 no adjoint, so this differentiates the step as written.
* ``step_convergence``  a measurement, run by hand: the observed grid orders
                 of one step between 32^3, 64^3 and 128^3.

Parity status: every function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` except the full-step convergence order, which the
paper does not fix (its delta is first order, Sec. 2.3 footnote): "parity
unpinned" for that property only (``step_convergence`` measures it).
``tests/test_oracle_mutations.py`` plants mistakes in these modules' source
(on the CPU) and checks that a pin fails for each.
"""
