/*
 * fvm.h -- C-ABI of the GB300 k-omega RANS finite-volume step library.
 *
 * The library advances cell-centred fields u, v, w, p, T, k, omega on a
 * uniform structured grid by the time step of "NeuralFVM: Neural-physics-
 * based Finite Volume Method for Turbulent Flows Using the k-omega Model":
 *
 *   1. dt/2 of the semi-implicit destruction of k and omega
 *      (Section 2.5, Eqs. k_des_step and o_des_step, Algorithm 4);
 *   2. one forward-Euler step (or a strong-stability-preserving Runge-Kutta
 *      step of order 2 or 3, desc.rk_stages) of convection (first-order
 *      upwind, Eq. upwind_x, Algorithm 2), diffusion (Eq.
 *      divergence_theorem) and production (Eqs. k_gen, o_gen) for u, v, w,
 *      T, k, omega (Eqs. ko_mom - ko_temp, Algorithm 3 and Section A.4);
 *   3. dt/2 of the destruction again (Strang splitting, Section 2.6);
 *   4. the pressure right-hand side b = -div(u*)/dt (Eq. pc_residual);
 *   5. multigrid V-cycles on A p = b, A = -Laplacian (Eq. neg_lap_discretize,
 *      Eq. jacobi_pc, Eqs. restriction / prolongation, Algorithm 1);
 *   6. the projection u = u* - dt grad p (Section 2.4).
 * fvm_lambda2 evaluates the lambda_2 vortex criterion of Section 3.2.3 on
 * the current velocity.
 * Boundary conditions use one ghost layer (Section 2.7, Eqs. bc_x - bc) and
 * masks for solid boxes; walls use omega = 6 nu / (beta_i d^2) in the
 * adjacent cells (Section 2.7); inlet k and omega follow Section 3.2.4.
 *
 * Conventions
 *   - Grid: nx * ny * nz cells, spacing Lx/nx, Ly/ny, Lz/nz; an axis with
 *     n = 1 is degenerate (2D) and both its faces must be FVM_EMPTY.
 *   - Field layout everywhere (device and host buffers): one array per
 *     field, x fastest: index (k * ny + j) * nx + i.
 *   - Field ids (bit i of a field mask): u 0, v 1, w 2, p 3, T 4, k 5,
 *     omega 6.
 *   - Boundary faces: 0..5 = x-, x+, y-, y+, z-, z+.  A vent covers the
 *     boundary cells [a0, a1) x [b0, b1) of one face, a and b being the
 *     face's tangential axes in increasing order (x faces: y, z; y faces:
 *     x, z; z faces: x, y).
 *   - The library owns all device memory of a case (cudaMalloc at create,
 *     cudaFree at destroy).  The caller owns every host buffer it passes.
 *   - Every call returns an fvm_status; on error nothing is written to the
 *     caller's outputs and fvm_last_error() describes the failure.  No call
 *     aborts, traps or hangs on bad input; CUDA errors map to FVM_ERR_CUDA.
 *   - Work is issued on the case's stream (desc.stream, or a stream the
 *     library creates).  Calls that return data to the host synchronise it.
 *   - A case is not thread safe; different cases may be used from
 *     different threads.
 */
#ifndef FVM_H
#define FVM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fvm_case fvm_case;          /* opaque, library-owned */

typedef enum {
    FVM_OK = 0,
    FVM_ERR_INVALID = -1,        /* bad descriptor or argument */
    FVM_ERR_OOM = -2,            /* device allocation failed */
    FVM_ERR_BUDGET = -3,         /* case bytes exceed the caller's budget */
    FVM_ERR_NOT_CONVERGED = -4,  /* V-cycle cap reached above the tolerance */
    FVM_ERR_DIVERGED = -5,       /* non-finite residual or time step */
    FVM_ERR_CUDA = -6            /* a CUDA runtime error */
} fvm_status;

enum { FVM_WALL = 0, FVM_INLET = 1, FVM_OUTLET = 2, FVM_EMPTY = 3 };
enum { FVM_ADIABATIC = 0, FVM_FIXED_T = 1, FVM_HEAT_FLUX = 2 };
enum { FVM_FP64 = 0, FVM_FP32 = 1, FVM_BF16_MIXED = 2 };
enum { FVM_U = 0, FVM_V = 1, FVM_W = 2, FVM_P = 3, FVM_T = 4, FVM_K = 5, FVM_OMEGA = 6 };

/* Boundary condition of a face or vent (Section 2.7). */
typedef struct {
    int32_t kind;            /* FVM_WALL / FVM_INLET / FVM_OUTLET / FVM_EMPTY */
    int32_t thermal;         /* walls: FVM_ADIABATIC / FVM_FIXED_T / FVM_HEAT_FLUX */
    double  T_value;         /* wall temperature, or heat flux into the fluid in W/m^2 */
    double  u_normal;        /* inlet: speed into the domain, m/s */
    double  intensity;       /* inlet: turbulence intensity I0 (k0 = 1.5 (I0 u0)^2) */
    double  length_scale;    /* inlet: l0 (omega0 = k0^0.5 / (C_mu l0)) */
    double  T_in;            /* inlet temperature */
    double  k_value;         /* inlet: k used instead of the I0 formula when > 0 */
    double  omega_value;     /* inlet: omega used instead of the l0 formula when > 0 */
} fvm_patch;

typedef struct {
    int32_t face, a0, a1, b0, b1, reserved;
    fvm_patch bc;
} fvm_vent;

/* Solid box [i0,i1) x [j0,j1) x [k0,k1) with a thermal wall condition. */
typedef struct {
    int32_t i0, i1, j0, j1, k0, k1, thermal, reserved;
    double  T_value;
} fvm_box;

typedef struct {
    int32_t nx, ny, nz;
    int32_t precision;               /* FVM_FP64 / FVM_FP32 / FVM_BF16_MIXED */
    double  Lx, Ly, Lz;              /* m */
    double  nu, Pr, Prt;             /* kinematic viscosity, Prandtl, turbulent Prandtl */
    double  sigma_k, sigma_w;        /* turbulent Prandtl numbers of k and omega */
    double  rho, cp;                 /* for heat-flux walls */
    double  gravity[3], beta_T, T_ref;
    int32_t buoyancy;                /* 1: Boussinesq force -g beta_T (T - T_ref) */
    int32_t dt_adapt;                /* 1: cap dt each step by the explicit stability limit */
    double  dt;                      /* > 0: fixed dt0; else dt0 = cfl min h / max inlet speed */
    double  cfl;
    fvm_patch faces[6];
    const fvm_vent* vents;  int32_t n_vents;  int32_t reserved0;
    const fvm_box*  boxes;  int32_t n_boxes;  int32_t reserved1;
    int32_t mg_levels;               /* 2..12; active axes = 2^(levels-1) * m, m >= 2 */
    int32_t pre_sweeps, post_sweeps; /* weighted-Jacobi sweeps, each >= 1 */
    int32_t max_vcycles;             /* cap per solve */
    int32_t fixed_vcycles;           /* > 0: exactly this many per solve, no test */
    int32_t inner_cycles;            /* V-cycles per FP64 outer residual (0: 1 for FP64, 2 otherwise);
                                        the stopping test runs after each group */
    int32_t sweep_planes;            /* z planes per block of the four-cell level kernels, 1..64
                                        (0: the built-in rule, about eight blocks per SM) */
    int32_t mg_variant;              /* 0: V(pre, post) cycles; 1: the paper's scheme (Algorithm 1:
                                        residual restricted straight down, one unweighted Jacobi per
                                        coarse level, nearest upsampling, a final Jacobi on p) */
    int32_t krylov;                  /* 1: flexible CG with one kept direction around the
                                        V-cycles (each outer iteration steps along the V-cycle
                                        correction made A-orthogonal to the previous direction,
                                        by the length that minimises the error's A-norm); 0: none.
                                        Not with mg_variant 1.  An addition beyond the paper. */
    int32_t coarse_sweeps;           /* pre- and post-sweeps on every level below the finest;
                                        0: the finest level's counts.  Not with mg_variant 1. */
    int32_t rk_stages;               /* explicit stage (Section 2.6 leaves the Runge-Kutta scheme
                                        open): 0 or 1 forward Euler; 2 or 3 the strong-stability-
                                        preserving schemes of Shu and Osher of that order, each stage
                                        a forward-Euler update (clamps and wall omega included)
                                        combined with the stage-0 state.  3 keeps a third copy of
                                        the six state fields. */
    int32_t smoother;                /* 0: every weighted-Jacobi sweep takes jacobi_weight (Eq.
                                        jacobi_pc); 1: sweep i of the n on one side of a level takes
                                        1 / x_i, x_i the roots (largest first before the coarse
                                        correction, smallest first after it) of the degree-n
                                        Chebyshev polynomial of [1/4, 2], which bounds the spectrum
                                        of D^-1 A: the n sweeps damp its upper part by
                                        1 / T_n(9/7).  At most 16 sweeps a side.  Not with
                                        mg_variant 1.  An addition beyond the paper. */
    double  mg_rel_tol;              /* ||b - A p|| / ||b|| target */
    double  jacobi_weight;           /* <= 0: 6/7 in 3D, 4/5 in 2D */
    uint64_t seed;                   /* SplitMix64 seed of the initial perturbation */
    double  init_perturb;            /* fields start at base * (1 + eps xi), xi in [-1, 1) */
    double  init_vel[3], init_T;
    double  init_k, init_omega;      /* <= 0: the first inlet's k0 / omega0 */
    void*   stream;                  /* cudaStream_t to use, or NULL */
} fvm_case_desc;

typedef struct {
    int32_t steps;                   /* steps run by this call */
    int32_t vcycles_total;           /* V-cycles over those steps */
    int32_t vcycles_last;            /* V-cycles of the last step */
    int32_t reserved;
    double  rel_residual;            /* ||b - A p|| / ||b|| after the last solve */
    double  dt_last;                 /* dt of the last step */
    double  sim_time;                /* simulated time since creation */
} fvm_step_stats;

typedef struct {
    int64_t cells;
    int32_t levels, precision;
    double  dt0, dt;                 /* base and current time step */
    double  sim_time;
    int64_t device_bytes;            /* device memory held by the case */
    int64_t steps;
    int64_t kernel_launches;         /* kernels launched on the case since creation */
} fvm_case_info;

/* Per-kernel-class statistics of the profiling hook. */
typedef struct {
    char    name[32];                /* kernel class, e.g. "explicit", "smooth_L0" */
    int64_t launches;
    double  ms;                      /* summed device time between the bracketing events */
    double  bytes;                   /* summed algorithmic bytes (each array read or written once) */
} fvm_kernel_stat;

/* Stages of one step, for fvm_run_stage (in step order). */
enum {
    FVM_STAGE_DT = 0,            /* dt = min(dt0, cfl / max rate) (or dt0) */
    FVM_STAGE_DESTRUCTION = 1,   /* dt/2 of Eqs. k_des_step, o_des_step */
    FVM_STAGE_EXPLICIT = 2,      /* forward Euler of the remaining terms */
    FVM_STAGE_RHS = 3,           /* b = -div(u*) / dt */
    FVM_STAGE_SOLVE = 4,         /* V-cycles on A p = b */
    FVM_STAGE_PROJECT = 5        /* u = u* - dt grad p */
};

/* Device bytes a case with this descriptor would allocate (0 if invalid).
   Used for admission against a memory budget. */
size_t fvm_case_bytes(const fvm_case_desc* desc);

/* Set up one case of the problem statement of Section 2.1 (the k-omega
   equations, Eqs. ko_mom - ko_temp with the standard constants printed
   there) on its grid, with the boundary conditions of Section 2.7 (one
   ghost layer, Eqs. bc_x - bc; solid boxes by masks; wall omega
   6 nu / (beta_i d^2)) and the inlet turbulence of Section 3.2.4
   (k0 = 1.5 (u0 I0)^2, omega0 from the length scale l0).
   Validates desc, allocates the case's device memory, builds boundary
   tables, the multigrid levels of Section 2.4 (full coarsening, Eq.
   restriction) and the coarsest-level inverse, and sets the seeded initial
   state (p = 0).
     desc : caller-owned, read during the call only (vents, boxes copied)
     out  : receives the library-owned case; set only on FVM_OK
   FVM_ERR_INVALID for a bad descriptor (fvm_last_error says which field),
   FVM_ERR_OOM if device memory runs out (nothing is leaked). */
fvm_status fvm_create_case(const fvm_case_desc* desc, fvm_case** out);

/* Free everything the case holds (after finishing its queued work). */
void fvm_destroy_case(fvm_case* c);

/* Advance nsteps time steps of the Strang-split scheme of Section 2.6: the
   destruction half step dt/2 (Section 2.5, Eqs. k_des_step / o_des_step,
   Algorithm 4), the explicit stage of convection, diffusion and production
   (Algorithms 2 and 3, Section A.4), the second half step, the pressure
   right-hand side (Eq. pc_residual), the multigrid solve of Section 2.4 and
   the projection u = u* - dt grad p.  Each step is one CUDA graph on the
   case's stream; the call synchronises that stream at the end.
     c     : the case (not thread safe)
     out   : caller-owned, may be NULL; statistics of the last step
   FVM_ERR_NOT_CONVERGED if a solve hit max_vcycles above mg_rel_tol (the
   step is still taken), FVM_ERR_DIVERGED on a non-finite residual or time
   step, FVM_ERR_INVALID for nsteps < 0. */
fvm_status fvm_step(fvm_case* c, int nsteps, fvm_step_stats* out);

/* Run one stage of the step (FVM_STAGE_*), for verification. */
fvm_status fvm_run_stage(fvm_case* c, int stage);

/* Run ncycles multigrid cycles on A p = b with the case's current b and p
   (Section 2.4: A the negative Laplacian of Eq. neg_lap_discretize,
   weighted Jacobi smoothing of Eq. jacobi_pc, Eqs. restriction and
   prolongation; Algorithm 1's own scheme with desc.mg_variant = 1), with no
   convergence test; p is updated in place on the device.
     rel_residual : caller-owned, may be NULL; ||b - A p|| / ||b|| over the
                    fluid cells after the cycles (FP64)
   Synchronises the case's stream.  FVM_ERR_INVALID for ncycles < 0. */
fvm_status fvm_vcycle(fvm_case* c, int ncycles, double* rel_residual);

/* Copy the fields of Section 2.1 selected by field_mask (u, v, w, p, T, k,
   omega: bit i for field id i) converted to double into host_out: the
   selected fields in id order, each nx*ny*nz values, x fastest.
     host_out : caller-owned host buffer of n doubles (pinned or pageable)
   An empty mask copies nothing.  Synchronises the case's stream.
   FVM_ERR_INVALID for mask bits above 6, a null buffer with a non-empty
   mask, or n below the number of values selected. */
fvm_status fvm_read_fields(fvm_case* c, unsigned field_mask, double* host_out, size_t n);

/* Overwrite the fields in field_mask from host_in (same layout as
   fvm_read_fields); values are rounded to the case's storage precision.
   Synchronises. */
fvm_status fvm_write_fields(fvm_case* c, unsigned field_mask, const double* host_in, size_t n);

/* fvm_read_fields / fvm_write_fields with FP32 host values (n floats, same
   layout, errors and synchronisation), half the bytes moved.  The state
   fields of an FP32 or BF16-corrections case are stored in FP32 and copy as
   they are, without conversion; p (held as a double-float pair) is rounded
   once to FP32 on reading and written as that FP32 value; an FP64 case's
   fields are rounded to FP32 on reading and widened exactly on writing. */
fvm_status fvm_read_fields_f32(fvm_case* c, unsigned field_mask, float* host_out, size_t n);
fvm_status fvm_write_fields_f32(fvm_case* c, unsigned field_mask, const float* host_in, size_t n);

/* Set the Poisson right-hand side b (nx*ny*nz doubles, host). */
fvm_status fvm_set_poisson_rhs(fvm_case* c, const double* host_b, size_t n);

/* Read b (nx*ny*nz doubles) into host memory.  Synchronises. */
fvm_status fvm_read_poisson_rhs(fvm_case* c, double* host_b, size_t n);

/* lambda_2 vortex criterion of the transient results (Section 3.2.3, after
   Jeong and Hussain 1995): for every cell, the middle eigenvalue of
   S^2 + Omega^2, where S and Omega are the symmetric and antisymmetric parts
   of the cell velocity gradient L_j D_j BC_j(u_i) of Algorithm 4 (boundary
   and obstacle neighbours by their Section 2.7 ghosts).  Negative values mark
   vortex cores; solid cells hold 0.  Computed from the case's current u, v, w
   in its compute precision; written to host_out as nx*ny*nz doubles, x
   fastest (caller-owned, n = its capacity in doubles).  Runs on the case's
   stream and synchronises it; the fields are not changed.
   FVM_ERR_INVALID for a null case or buffer or n < nx*ny*nz. */
fvm_status fvm_lambda2(fvm_case* c, double* host_out, size_t n);

/* Vector-Jacobian product of the projection, the first piece of a
   differentiable step (an addition: Section 1 presents the method as
   differentiable but defines no discrete gradient).  The map is
   u* -> (u^{n+1}, p) of steps 4-6 above with an exact pressure solve:
   b = -div(u*)/dt (Eq. pc_residual), A p = b, u^{n+1} = u* - dt G p.  It is
   affine in u* (the inlets add constants), and this call returns
   xbar = J^T ybar for its Jacobian J:
       q = pbar + (d u^{n+1} / d p)^T (ubar, vbar, wbar),
       A lambda = q (A is symmetric on the fluid cells),
       xbar = (ubar, vbar, wbar) + (d b / d u*)^T lambda.
   The solve runs V-cycles of the case's own multigrid from zero until
   ||q - A lambda|| / ||q|| <= rel_tol or max_vcycles cycles (in chunks of
   four); the case's p and b are saved and restored, its fields are not
   touched.  dt: the time step of the projection being differentiated.
   host_ybar: 4 nx*ny*nz doubles (ubar, vbar, wbar, pbar; field-major, x
   fastest); host_xbar: 3 nx*ny*nz doubles out; n = the number of doubles
   host_ybar holds (>= 4 nx*ny*nz); host_xbar must hold 3 nx*ny*nz.
   *rel_out (may be NULL) gets the final relative residual.  A is
   nonsingular on the fluid cells: fvm_create_case rejects cases without a
   zero-value (outlet) face.  Fluid enclosed by obstacles with no path to an
   outlet would make A singular there; q then generally lies outside A's range
   and the solve ends with FVM_ERR_NOT_CONVERGED.  Each chunk of four cycles
   restarts the flexible-CG direction of krylov = 1 cases.  FP64 cases
   only.  FVM_ERR_NOT_CONVERGED if rel_tol was not reached (xbar is still
   written); FVM_ERR_INVALID for null pointers, dt <= 0, rel_tol <= 0,
   max_vcycles < 1, a short buffer or a reduced-precision case.
   Synchronises. */
fvm_status fvm_projection_vjp(fvm_case* c, double dt, const double* host_ybar, double* host_xbar, size_t n,
                              double rel_tol, int32_t max_vcycles, double* rel_out);

/* ---------------------------------------------------------------- batches
   Cases stepped together (uneven sizes allowed).  Every launch site of the
   step (each step kernel, and each multigrid kernel of each level) runs
   once for all cases: one launch over a table of per-case kernel arguments,
   each case's blocks laid end to end.  One time step of the whole batch is
   one CUDA graph; its V-cycle loop runs until no case is active, and each
   case stops on its own rule (a converged case's blocks return at once).
   The results are those of stepping each case alone (tested bitwise).

   Requirements: every case has the same precision, runs the default
   one-sweep level kernels and the single-CTA coarse levels, and has
   profiling off.  While a case belongs to a live batch, step it only
   through the batch.  Memory: the batch holds device tables of its launch
   arguments (kilobytes per case) per pointer parity; the cases keep their
   own fields. */
typedef struct fvm_batch fvm_batch;

typedef struct {
    int32_t n_cases;
    int32_t graphs;                  /* CUDA graphs captured (one per pointer parity) */
    int64_t steps;                   /* batch steps taken */
    int64_t kernel_launches;         /* kernels run by the batch since creation */
    int64_t cells;                   /* sum of the cases' cells */
    int64_t launches_per_step;       /* per step outside the V-cycle loop */
    int64_t launches_per_outer;      /* per outer V-cycle iteration (level-0 residual + V-cycle) */
} fvm_batch_info;

/* Group n cases (the array is copied; the cases stay owned by the caller,
   who must destroy the batch before any of its cases).  stream: the
   cudaStream_t the batch runs on, or NULL for a stream of its own.
   Errors: FVM_ERR_INVALID (null or repeated case, mixed precisions,
   profiling on), FVM_ERR_OOM, FVM_ERR_CUDA. */
fvm_status fvm_batch_create(fvm_case* const* cases, int32_t n, void* stream, fvm_batch** out);

/* Advance every case by nsteps.  stats (may be NULL): n entries, in the
   order of creation.  Returns the worst status over the cases
   (FVM_ERR_DIVERGED before FVM_ERR_NOT_CONVERGED); fields stay readable. */
fvm_status fvm_batch_step(fvm_batch* b, int32_t nsteps, fvm_step_stats* stats);

/* fvm_batch_step in two halves, so that the caller can do host work while
   the steps run: fvm_batch_launch enqueues nsteps steps on the batch's
   stream and returns; fvm_batch_wait waits for them and fills stats as
   fvm_batch_step does.  One launch at a time per batch (FVM_ERR_INVALID
   otherwise, and for a wait with nothing launched); the cases' fields are
   not to be read or written in between. */
fvm_status fvm_batch_launch(fvm_batch* b, int32_t nsteps);
fvm_status fvm_batch_wait(fvm_batch* b, fvm_step_stats* stats);

fvm_status fvm_batch_get_info(const fvm_batch* b, fvm_batch_info* out);

/* Profiling pass of a batch: nsteps steps run launch by launch (the merged
   launches of the batch's graph, the V-cycle loop driven from the host with
   one read of the cases' solve states per outer iteration), each launch
   bracketed by a pair of CUDA events on the batch's stream.  out receives
   up to cap per-site tallies (name = launch site such as "sweep_L0";
   launches; summed event time; algorithmic bytes summed over the cases);
   *n_out (may be NULL) = number of sites.  The steps advance the cases like
   fvm_batch_step. */
fvm_status fvm_batch_profile(fvm_batch* b, int32_t nsteps, fvm_kernel_stat* out, int32_t cap, int32_t* n_out);
void fvm_batch_destroy(fvm_batch* b);

/* One-shot form: a temporary batch of the n cases, advanced by nsteps, then
   released (the graphs are captured on every call; keep a fvm_batch for
   repeated stepping).  stats (may be NULL): n entries. */
fvm_status fvm_step_batch(fvm_case* const* cases, int n, int nsteps, fvm_step_stats* stats);

fvm_status fvm_case_get_info(const fvm_case* c, fvm_case_info* out);

/* ---------------------------------------------------------------- autotuning
   Picks the multigrid parameters for a case by measurement (no counterpart
   in the paper, whose solver runs a fixed scheme): on temporary copies of
   the case (own stream; the descriptor is not changed), graph-mode steps
   after two untimed ones, timed with CUDA events, `steps` steps each.
   Pass 1: V(nu, nu) for nu = 2, 3, 4 times the V-cycles per FP64 outer
   residual (1..4 with reduced-precision corrections, 1 in FP64) times the
   flexible-CG acceleration off / on times the constant / Chebyshev sweep
   weights (both off only with mg_variant 1); pass 2: the
   z planes per block of the four-cell level kernels (the rule, 1 .. 32)
   with the best pass-1 choice; pass 3: 1 and 2 sweeps on the levels below
   the finest (coarse_sweeps), where fewer than the finest level's.  Candidates that stop at max_vcycles above
   the tolerance are not eligible.  Copy the result into the descriptor's
   pre_sweeps, post_sweeps, inner_cycles, sweep_planes, krylov, coarse_sweeps and smoother.  Device memory: one
   temporary case at a time.  Errors: FVM_ERR_INVALID, FVM_ERR_NOT_CONVERGED
   (no candidate converged), FVM_ERR_CUDA. */
typedef struct {
    int32_t pre_sweeps, post_sweeps, inner_cycles, sweep_planes;
    double  ms_per_step;             /* of the choice, device time per step */
    int32_t candidates;              /* candidates timed */
    int32_t krylov;                  /* 0 / 1: the flexible-CG acceleration */
    int32_t coarse_sweeps;           /* sweeps on the levels below the finest (0: as the finest) */
    int32_t smoother;                /* 0 / 1: the constant or the Chebyshev sweep weights */
} fvm_tuning;

fvm_status fvm_autotune(const fvm_case_desc* desc, int32_t steps, fvm_tuning* out);

/* ---------------------------------------------------------------- serving
   A request loop over resident cases (continuous batching).  A request is a
   case description plus a number of steps.  fvm_server_poll runs one
   scheduling round:
     1. launch the steps of every resident case together: one fvm_batch per
        precision, min(chunk, fewest remaining steps) steps;
     2. meanwhile admit, first come first served, the queued requests whose
        arrival time has passed while their device bytes (fvm_case_bytes)
        fit the HBM budget and a slot is free: each becomes a resident case
        that joins the next round, its creation overlapping the steps;
     3. wait for the steps, retire the finished requests (their memory is
        freed at once, or kept for fvm_server_read_fields until
        fvm_server_release when keep_results is set) and report them.
   Times are seconds on the server's steady clock (fvm_server_now, zero at
   creation); a request's latency is t_done - t_arrive.  The paper serves
   no requests: this is an addition for many concurrent cases.  Not
   thread-safe: drive a server from one thread. */
typedef struct fvm_server fvm_server;

typedef struct {
    int64_t id;
    int32_t status;                  /* FVM_OK, or the status that ended the request */
    int32_t steps;                   /* steps run */
    int64_t cells;
    int64_t device_bytes;
    int32_t vcycles_total;
    int32_t reserved;
    double  rel_residual;            /* after the last solve */
    double  t_arrive, t_admit, t_done;
} fvm_request_result;

typedef struct {
    int64_t queued, running, done;
    int64_t bytes_in_use;            /* device bytes of the resident cases */
    int64_t rounds;                  /* scheduling rounds that stepped cases */
    int64_t batch_rebuilds;          /* batches (re)built after admissions or retirements */
    int64_t cell_steps;              /* summed over retired and running requests */
    double  t_admit_s;               /* host seconds in admission (case creation) */
    double  t_rebuild_s;             /* host seconds building batches (recording, graph capture) */
    double  t_step_s;                /* seconds in batched steps (launch to completion) */
} fvm_server_info;

/* budget_bytes: device bytes the resident cases may hold; max_cases: most
   resident cases (0: no limit); stream: cudaStream_t or NULL (own stream);
   keep_results: keep retired cases for reading.  Errors: FVM_ERR_INVALID. */
fvm_status fvm_server_create(int64_t budget_bytes, int32_t max_cases, void* stream, int32_t keep_results,
                             fvm_server** out);
double fvm_server_now(const fvm_server* s);
/* Queue a request (the descriptor and its vent and box arrays are copied;
   desc->stream is ignored).  FVM_ERR_BUDGET when the case alone exceeds the
   budget, FVM_ERR_INVALID for a bad descriptor. */
fvm_status fvm_server_submit(fvm_server* s, const fvm_case_desc* desc, int32_t nsteps, double t_arrive,
                             int64_t* id_out);
/* One scheduling round (see above); done receives up to cap retired
   requests, *n_done their number (may be NULL).  Returns FVM_OK unless the
   server itself failed; a request's own failure is in its result. */
fvm_status fvm_server_poll(fvm_server* s, int32_t chunk, fvm_request_result* done, int32_t cap, int32_t* n_done);
fvm_status fvm_server_get_info(const fvm_server* s, fvm_server_info* out);
/* Fields of a retired request (keep_results), as fvm_read_fields. */
fvm_status fvm_server_read_fields(fvm_server* s, int64_t id, unsigned field_mask, double* host_out, size_t n);
fvm_status fvm_server_release(fvm_server* s, int64_t id);
void fvm_server_destroy(fvm_server* s);

/* Options (fvm_set_option).  FVM_OPT_GRAPH (default 1): run each time
   step as one CUDA graph, the V-cycle loop being a device-side while node;
   0 runs the same kernels launch by launch with one host synchronisation
   per V-cycle.  Results are identical either way. */
enum { FVM_OPT_GRAPH = 1 };
fvm_status fvm_set_option(fvm_case* c, int option, int64_t value);

/* Profiling hook.  While enabled, every kernel the case launches is
   bracketed by a pair of CUDA events on the case's stream, and its class,
   device time and algorithmic bytes are tallied; steps then run launch by
   launch (not as graphs).  Enabling or disabling clears the tallies. */
fvm_status fvm_profile_enable(fvm_case* c, int enable);

/* Copy up to cap per-class tallies into out (n_out = classes seen), and
   clear them.  Synchronises the case's stream. */
fvm_status fvm_profile_read(fvm_case* c, fvm_kernel_stat* out, int cap, int* n_out);

/* Pressure residual without any device allocation (the paper has no
   counterpart; this serves callers that cannot call cudaMalloc, e.g. a
   program whose device memory belongs to a pooling allocator, a control
   loop that must not take an allocation's latency or implicit
   synchronisation, or a plug-in that must keep its device footprint fixed).
   Computes r = b - A p on an nx x ny x nz box without obstacles, A the same
   7-point negative Laplacian the pressure solve uses (one ghost per domain
   face: zero-gradient for p where dirichlet[face] = 0, zero-value where it
   is 1; a one-cell axis contributes no term), and norms[0] = ||r||^2,
   norms[1] = ||b||^2.
     p, b, r : device pointers to nx*ny*nz doubles, x fastest (caller-owned)
     norms   : device pointer to 2 doubles (caller-owned)
     h       : host array, cell sizes along x, y, z; dirichlet: host array of 6
     stream  : cudaStream_t or NULL; the call only enqueues work
   The kernel's scratch (per-block partial sums and a counter, about 1 MB) is a
   static device array that every GPU loading the library keeps until exit;
   grids above 65,536 blocks of 32 x 4 x 2 cells (16,777,216 cells), or above
   65,535 blocks along y or z, are rejected with FVM_ERR_INVALID.  The first call on a device looks up that
   array's address (with the device current); make that first call before any
   stream capture.  All calls share the array: calls that overlap on the GPU
   (other streams, other threads) race and must be serialised by the caller. */
fvm_status fvm_poisson_residual_static(const double* p, const double* b, int32_t nx, int32_t ny, int32_t nz,
                                       const double h[3], const int32_t dirichlet[6], double* r,
                                       double* norms, void* stream);

/* Vector-Jacobian product of one destruction half step (the k and omega
   updates of Section 2.5, Eqs. k_des_step and o_des_step, Algorithm 4) over
   dt, linearised at the case's current u, v, w, k, omega.  The step maps
   (u, v, w, k, omega) to (u, v, w, k', omega'); host_ybar holds cotangents of
   its output (u, v, w, k', omega': 5 nx*ny*nz doubles, field-major, x
   fastest) and host_xbar receives the cotangents of its input (same layout).
   The partial derivatives of the pointwise formulas (beta*, f_beta*, chi_k,
   chi_omega, f_beta) are written out and sent back through the transposed
   cell-gradient stencils with the Section 2.7 ghosts.  FP64 cases only; the
   case is not changed.  n = capacity of each buffer in doubles (>= 5 N).
   Synchronises.  FVM_ERR_INVALID for null pointers, dt <= 0, short buffers
   or a reduced-precision case. */
fvm_status fvm_destruction_vjp(fvm_case* c, double dt, const double* host_ybar, double* host_xbar, size_t n);

/* Vector-Jacobian product of the forward-Euler explicit stage (Algorithms 2
   and 3, Section A.4: upwind convection, central diffusion, the -(2/3) k
   face term, production G_k, G_omega and buoyancy) over dt, linearised at
   the case's current u, v, w, T, k, omega.  host_ybar: cotangents of the
   stage's output (u, v, w, T, k, omega: 6 N doubles); host_xbar: cotangents
   of its input (6 N).  Clamped k, omega and the wall omega pass no
   derivative, and at u_face = 0 the upwind side is the lower cell, as in
   the forward.  FP64, forward-Euler cases only (rk_stages 0 or 1); the case
   is not changed.  n >= 6 N.  Synchronises.  FVM_ERR_INVALID as above. */
fvm_status fvm_explicit_vjp(fvm_case* c, double dt, const double* host_ybar, double* host_xbar, size_t n);

/* Vector-Jacobian product of one whole time step (Section 2.6) with a fixed
   dt and the pressure solve taken as exact: the first destruction half step,
   the explicit stage, the second half step, the right-hand side, the solve
   and the projection, composed in reverse.  host_ybar: cotangents of the
   step's output u, v, w, p, T, k, omega (7 N doubles, in field id order);
   host_xbar: cotangents of the step's input u, v, w, T, k, omega (6 N).  The
   adjoint pressure solve runs the case's V-cycles to rel_tol (as
   fvm_projection_vjp); *rel_out (may be NULL) gets its final relative
   residual.  FP64, forward-Euler cases only; the case's fields, p and b are
   not changed.  n >= 7 N.  Synchronises.  FVM_ERR_NOT_CONVERGED if rel_tol
   was not reached (xbar is still written); FVM_ERR_INVALID as above or for
   rel_tol <= 0, max_vcycles < 1. */
fvm_status fvm_step_vjp(fvm_case* c, double dt, const double* host_ybar, double* host_xbar, size_t n,
                        double rel_tol, int32_t max_vcycles, double* rel_out);

/* sizeof of the public structs, for binding checks: out[0..10] = fvm_patch,
   fvm_vent, fvm_box, fvm_case_desc, fvm_step_stats, fvm_case_info,
   fvm_kernel_stat, fvm_batch_info, fvm_request_result, fvm_server_info,
   fvm_tuning.  Needs no GPU. */
void fvm_struct_sizes(size_t out[11]);

/* Message of the last failed call on this thread ("" if none). */
const char* fvm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
