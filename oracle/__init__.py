"""FP64 CPU oracle for one k-omega RANS finite-volume time step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
path (the CUDA library and its Python binding) never imports, links or calls
it, and this package never imports the product.

It restates the method of "NeuralFVM: Neural-physics-based Finite Volume
Method for Turbulent Flows Using the k-omega Model" in plain numpy float64,
following the paper's tensor notation: fields are arrays of shape
(nx, ny, nz); BC_x pads one ghost layer along x (Section 2.7, Eqs. bc_x-bc);
L_x and D_x turn n cell values into n+1 face values once padded (Eq. Dx_Lx);
upwind selection follows Eq. upwind_x / Algorithm 2; fluxes are summed with
the divergence theorem (Eq. divergence_theorem).  Nothing is fused or
reordered beyond what the paper's algorithms state.

Modules
  model       closure constants and formulas (Eqs. ko_turb_diff - o_des)
  geometry    grid levels, boundary patches, ghost cells, face states
  destruction semi-implicit destruction half step (Eqs. k_des_step,
              o_des_step; Algorithm 4)
  transport   explicit stage for u, v, w, T, k, omega (Algorithms 2, 3 and
              the "rest" terms of Section 2.5)
  poisson     pressure right-hand side (Eq. pc_residual), the operator A,
              Jacobi smoothing (Eq. jacobi_pc), RES / PROL (Eqs. restriction,
              prolongation), the V-cycle, direct solves, projection
  step        one Strang-split time step (Section 2.6) and the seeded
              initial state
  diagnostics the lambda_2 vortex criterion of the transient results
              (Section 3.2.3)
  adjoint     vector-Jacobian products for a differentiable step: the
              projection (b(u*), exact solve, u* - dt G p), the destruction
              step, the explicit stage and a whole time step

Parity status: every function is pinned by tests in tests/test_oracle_*.py
against closed forms, invariants, special cases or brute force, except the
composition of a full turbulent step ("parity unpinned" against the paper:
the paper prints no field values for any case; the step is pinned only
through its components, symmetry and mass balance).
"""
