"""CPU FP64 oracle for the coupled multigrid method for the generalized Stokes system.

This package is TEST INFRASTRUCTURE. It is a plain, slow, obviously-correct restatement of
Takacs, "A robust multigrid method for the time-dependent Stokes problem" (SINUM 53(6), 2015),
written with NumPy/SciPy in float64. Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the product path (the CUDA library and its
Python binding) never does, and the two share no code.

Modules:
    mesh      -- the 8-triangle coarse mesh of the unit square and uniform red refinement (Sec. 6)
    fem       -- Taylor-Hood P2-P1 element matrices by exact polynomial integration, global
                 assembly of A = K + beta*M_U and B (Sec. 2, eq. gen:bil:mv)
    transfer  -- canonical prolongation (embedding) and restriction (its transpose) (Sec. 3)
    multigrid -- Uzawa-type and normal-equation smoothers (Sec. 4), the practical diagonal
                 preconditioner (eq. numintroduc), V/W cycles with an exact coarsest solve (Sec. 3),
                 solve loop, direct reference solve
    adjoint   -- gradients of a loss through the discrete solve (symmetric system)
    experiments -- the numerical experiment of Sec. 6: cone-based exact solution, its L2
                 projection, the error norm of eq. defMcL and the mean convergence rate
    timestep  -- implicit Euler steps of the time-dependent Stokes problem (Sec. 1: beta = 1/dt)
    lshape    -- the L-shaped (non-convex) domain: masked meshes, unknowns and transfers (Sec. 1)

Parity status: every function here is pinned by tests under tests/ against closed forms,
invariants or brute force (see the test files); nothing is "parity unpinned".
"""
