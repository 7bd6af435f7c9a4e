/*
 * rafem.h — C-ABI of librafem: per-time-step reassembly and sparse solve of the coupled electric-potential /
 * Pennes-bioheat P1-tetrahedral finite-element model of radiofrequency ablation (RAFEM), on one B300 GPU.
 *
 * What the library computes follows the paper's statement of the problem (arXiv 2409.13036):
 *   - Sec. II-A "Main application loop": time advances step by step; each corrector pass recomputes the
 *     element equations from updated values, assembles them into a global sparse matrix (structurally
 *     symmetric, fixed pattern) and solves it.
 *   - Sec. III-A: element equations assembled into a CSR global matrix without races; Sec. III-B: the fixed
 *     pattern lets analysis work be reused across steps; residual tolerance 1e-10.
 *   - Sec. II-B: CG for symmetric positive-definite systems, preconditioning to accelerate convergence.
 * The PDE pair and constants (the paper defers them to its cited formulation) are read as
 *     div(sigma(T) grad V) = 0,  sigma_e = sigma0_e (1 + alpha (mean_e T - 37)),
 *     rho_c dT/dt = div(k grad T) + sigma |grad V|^2 - perf (T - T_a),
 * discretised with P1 tetrahedra, consistent mass and backward Euler, solved staggered (V then T), each
 * system Dirichlet-lifted symmetrically so that both are SPD.
 *
 * Conventions (all entry points):
 *   - Return value: 0 = RAFEM_OK; positive = soft outcome (RAFEM_NOT_CONVERGED); negative = error.
 *   - Inputs passed to rafem_create are copied; the caller keeps ownership of every pointer it passes.
 *   - A pointer documented as "device" must be a CUDA device pointer valid on the context's device; "host"
 *     pointers are ordinary host memory (pinned or pageable).
 *   - All work is issued on the stream given at create (NULL = a non-blocking stream the context creates and
 *     owns) and every entry point synchronises that stream before returning, unless stated otherwise.
 *   - There is no global state: calls on different contexts are independent; calls on one context must not
 *     overlap (not thread-safe).
 *   - Units are SI; coordinates in metres, temperatures in degrees Celsius, potentials in volts.
 */
#ifndef RAFEM_H
#define RAFEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------------------------------- */
#define RAFEM_OK                 0
#define RAFEM_NOT_CONVERGED      1   /* iteration cap reached; fields hold the last iterate, stats are filled  */
#define RAFEM_ERR_BAD_INPUT     -1   /* a NULL pointer, a size out of range, an index outside the mesh         */
#define RAFEM_ERR_BAD_MESH      -2   /* a tetrahedron with non-positive volume                                  */
#define RAFEM_ERR_OOM           -3   /* device or host allocation failed                                       */
#define RAFEM_ERR_NONFINITE     -4   /* NaN or Inf met in a residual, a coefficient or a field                  */
#define RAFEM_ERR_TIMEOUT       -5   /* a bounded device wait ran out (not expected in normal use; see
                                        rafem_set_wait_limit)                                                  */
#define RAFEM_ERR_CUDA          -6   /* a CUDA runtime call failed                                              */
#define RAFEM_ERR_INTERNAL      -7   /* an internal consistency check failed                                   */
#define RAFEM_ERR_BREAKDOWN     -8   /* Krylov breakdown: p^T A p <= 0 (matrix not SPD) or a zero denominator  */

/* ---- options ---------------------------------------------------------------------------------------------- */
#define RAFEM_SYS_V 1                /* the electric-potential system                                          */
#define RAFEM_SYS_T 2                /* the thermal system                                                     */

#define RAFEM_PRECOND_JACOBI 0       /* diagonal preconditioner                                               */
#define RAFEM_PRECOND_ILU0   1       /* incomplete LU(0) on the fixed pattern (single instance; FP64 or mixed)  */

#define RAFEM_ILU_MULTICOLOR 0       /* ILU(0) ordering: greedy colours of the matrix graph, levels = colours  */
#define RAFEM_ILU_NATURAL    1       /* ILU(0) ordering: the mesh numbering, levels = dependency levels        */

#define RAFEM_PRECISION_FP64  0      /* every Krylov operation in FP64                                        */
#define RAFEM_PRECISION_MIXED 1      /* FP32 inner Krylov (FP32 values, vectors, dots) + FP64 residual refinement */

#define RAFEM_SOLVER_PCG      0      /* conjugate gradients (SPD systems)                                      */
#define RAFEM_SOLVER_BICGSTAB 1      /* BiCGSTAB (general nonsymmetric systems): FP64, Jacobi, SELL-32 layout,
                                        single instance                                                        */

#define RAFEM_SOLVER_GMRES    2      /* restarted GMRES(m), the paper's iterative method (Sec. III-B): FP64, right
                                        Jacobi, classical Gram-Schmidt (repeated once when the first pass
                                        cancels more than 99% of the vector's squared norm), SELL-32 layout, single
                                        instance; m = gmres_restart, adaptive between gmres_min_restart and m
                                        when that is set; two full-length cycles in a row that each reduce the
                                        residual by less than 0.1% (stagnation) end the solve NOT_CONVERGED   */
#define RAFEM_SOLVER_PIPECG   3      /* pipelined Jacobi-PCG (Ghysels-Vanroose): CG's iterates with one grid
                                        barrier per iteration instead of two, at the cost of 20 vector touches
                                        instead of 14; for small systems and batches of small instances. FP64,
                                        Jacobi, symmetric lift; the solve ends with the true residual and
                                        restarts from x (at most 3 times) while the recurrences have drifted   */

#define RAFEM_PREDICT_PROJECT 4      /* predictor: for the potential, A-orthogonal projection of the new
                                        solution onto the span of its last proj_basis (default 4) solutions
                                        (difference basis, free rows; one extra pass over the matrix per
                                        solve; needs the symmetric lift, any solver); quadratic extrapolation
                                        otherwise and for T                                                    */

#define RAFEM_COUPLING_STAGGERED   0 /* V then T per pass (lagged sigma; corrector passes when n_corrector > 1) */
#define RAFEM_COUPLING_MONOLITHIC  1 /* the paper's 2N x 2N system: V and T of a step solved together by Newton's
                                        method (Jacobian with the sigma(T) and Joule couplings, unknowns
                                        interleaved per node, 2 x 2 blocks on the node pattern, row-only
                                        Dirichlet rows; linear solver: coupled_solver) until max |dT| <
                                        corrector_tol or n_corrector iterations, starting from the lagged
                                        staggered step; each linear solve is inexact (forcing terms of Eisenstat
                                        and Walker, within [tol, 1e-2]); FP64, SELL-32 layout, single instance;
                                        the iterations run on the device like corrector passes                 */

/* Linear solver of the monolithic step's Newton iterations (rafem_params.coupled_solver). */
#define RAFEM_COUPLED_FGMRES   0     /* flexible GMRES, at most 8 iterations per Newton iteration, right-
                                        preconditioned by one block Gauss-Seidel sweep (potential block, then
                                        thermal block with the coupling term) whose block solves are mixed-
                                        precision Jacobi-PCG solves of the split systems to a relative residual
                                        of 0.4; forcing terms within [max(tol, 1e-6), 1e-2] (default)           */
#define RAFEM_COUPLED_BICGSTAB 1     /* BiCGSTAB with 2 x 2 block-Jacobi preconditioning                        */

#define RAFEM_LIFT_SYMMETRIC  0      /* Dirichlet rows and columns of the matrix zeroed, unit diagonal, known
                                        values moved to the right-hand side: the systems stay SPD              */
#define RAFEM_LIFT_ROW        1      /* Dirichlet rows replaced by identity rows, columns kept: the same solution
                                        from a nonsymmetric system (BiCGSTAB or GMRES; no adjoint)              */

#define RAFEM_ASSEMBLY_GATHER 0      /* row-owner assembly: one thread per matrix row sums the element
                                        contributions of its entries (SELL-32 layout only); for the monolithic
                                        step's 2 x 2 block Jacobian as well (an element pass writes per-element
                                        records, a row pass sums them per entry)                              */
#define RAFEM_ASSEMBLY_COLOR  1      /* element-owner scatter, one launch per element colour, no atomics     */

#define RAFEM_ARITH_AUTO      0      /* element and node passes of the gather assembly in double-word arithmetic
                                        when the mesh's scales allow it (element volumes in [2^-90, 2^60] m^3,
                                        coefficients and boundary values below 2^60 in magnitude), FP64
                                        otherwise                                                              */
#define RAFEM_ARITH_FP64      1      /* FP64 element and node passes                                           */
#define RAFEM_ARITH_DW        2      /* double-word element and node passes (pairs of floats, 48 significant
                                        bits, on the FP32 pipes; FP64 only to write FP64 results): B300 issues
                                        FP64 at 1/64 of its FP32 rate, which bounds the FP64 passes. Gather
                                        assembly only; BAD_INPUT at create when the scales are out of range    */

/* Mesh and boundary data of one instance. All pointers are host pointers, read only during rafem_create. */
typedef struct rafem_mesh {
    int32_t n_nodes;                 /* N >= 4                                                                 */
    int32_t n_tets;                  /* E >= 1                                                                 */
    const double*  coords;           /* [N*3] x,y,z per node, metres                                           */
    const int32_t* tets;             /* [E*4] node ids per tetrahedron (any orientation; volume must be != 0)  */
    const uint8_t* bc_V;             /* [N] 1 = Dirichlet node of the potential system                         */
    const double*  g_V;              /* [N] prescribed potential where bc_V = 1                                */
    const uint8_t* bc_T;             /* [N] 1 = Dirichlet node of the thermal system                           */
    const double*  g_T;              /* [N] prescribed temperature where bc_T = 1                              */
    const double*  sigma0;           /* [E] electrical conductivity at 37 degC, S/m                            */
    const double*  k;                /* [E] thermal conductivity, W/m/K                                        */
} rafem_mesh;

/* Physics, time stepping and solver parameters. rafem_default_params fills the liver defaults. */
typedef struct rafem_params {
    double  alpha_sigma;             /* 1/degC, temperature coefficient of sigma (0.015)                      */
    double  rho_c;                   /* J/m^3/K (3.6e6)                                                        */
    double  perf;                    /* W/m^3/K, perfusion coefficient (2.4e4)                                 */
    double  T_a;                     /* degC, arterial temperature (37)                                        */
    double  dt;                      /* s, time step (1)                                                       */
    double  tol;                     /* relative residual ||b - A x|| / ||b|| to reach (1e-10)                 */
    double  inner_tol;               /* mixed precision: relative reduction of each FP32 inner solve (1e-4)    */
    double  corrector_tol;           /* degC, max |T^{k+1} - T^k| ending the corrector passes (1e-6)           */
    int32_t max_iter;                /* cap on Krylov iterations per solve, FP64 and inner together (20000)    */
    int32_t max_refine;              /* mixed precision: cap on FP64 refinements per solve (30)                */
    int32_t n_corrector;             /* corrector passes per step; 1 = lagged coefficients (1, at most 50)     */
    int32_t precond;                 /* RAFEM_PRECOND_*                                                        */
    int32_t precision;               /* RAFEM_PRECISION_*                                                      */
    int32_t solver;                  /* RAFEM_SOLVER_*                                                         */
    int32_t lanes_per_row;           /* matrix layout: 0 or 1 = SELL-32 (one thread per row), 4/8/16/32 = CSR
                                        with that many lanes per row                                          */
    int32_t rows_per_tile;           /* rows per work tile of the persistent solver: 0 = automatic            */
    int32_t assembly;                /* RAFEM_ASSEMBLY_GATHER (default with SELL-32) or RAFEM_ASSEMBLY_COLOR      */
    int32_t predictor;               /* initial guess of each solve (the predictor of the predictor-corrector
                                        loop): polynomial extrapolation in time of order 0..3 (0 = x^n,
                                        1 = 2 x^n - x^{n-1}, 2 = 3 x^n - 3 x^{n-1} + x^{n-2},
                                        3 = 4 x^n - 6 x^{n-1} + 4 x^{n-2} - x^{n-3}), or
                                        RAFEM_PREDICT_PROJECT (default)                                       */
    int32_t ilu_order;               /* RAFEM_PRECOND_ILU0 only: RAFEM_ILU_MULTICOLOR (0) or RAFEM_ILU_NATURAL  */
    int32_t lift;                    /* RAFEM_LIFT_SYMMETRIC (0) or RAFEM_LIFT_ROW (nonsymmetric: BiCGSTAB or
                                        GMRES)                                                                 */
    int32_t gmres_restart;           /* GMRES restart length m, 1..64 (0 = 30)                                  */
    int32_t coupling;                /* RAFEM_COUPLING_STAGGERED (0) or RAFEM_COUPLING_MONOLITHIC               */
    int32_t arith;                   /* RAFEM_ARITH_AUTO (0), RAFEM_ARITH_FP64 or RAFEM_ARITH_DW                 */
    int32_t proj_basis;              /* RAFEM_PREDICT_PROJECT: solutions in the basis, 1..8 (0 = 4)             */
    int32_t gmres_min_restart;       /* RAFEM_SOLVER_GMRES: 0 = every cycle has gmres_restart steps; 1..m = the
                                        cycle length adapts between this and gmres_restart from each cycle's
                                        residual reduction (shorter while convergence is moderate, back to the
                                        full length on stagnation); every solve starts at the full length      */
    int32_t coupled_solver;          /* RAFEM_COUPLING_MONOLITHIC: RAFEM_COUPLED_FGMRES (0) or
                                        RAFEM_COUPLED_BICGSTAB                                                 */
} rafem_params;

/* Per-step statistics, filled on the device and copied back when requested. */
typedef struct rafem_step_stats {
    int32_t status;                  /* RAFEM_OK, RAFEM_NOT_CONVERGED or a negative error                     */
    int32_t iters_V;                 /* Krylov iterations of the potential solve (all refinements); monolithic
                                        step: BiCGSTAB iterations, or with RAFEM_COUPLED_FGMRES the inner CG
                                        iterations on the potential block, over all Newton iterations          */
    int32_t iters_T;                 /* Krylov iterations of the thermal solve (monolithic step with
                                        RAFEM_COUPLED_FGMRES: inner CG iterations on the thermal block)        */
    int32_t refine_V;                /* FP64 refinements of the potential solve (mixed precision), restart
                                        cycles (GMRES), outer flexible-GMRES iterations (monolithic step with
                                        RAFEM_COUPLED_FGMRES), else 0                                          */
    int32_t refine_T;                /* FP64 refinements of the thermal solve                                  */
    int32_t correctors;              /* corrector passes (monolithic step: Newton iterations) in this step     */
    double  relres_V;                /* final relative residual of the potential solve (FP64)                 */
    double  relres_T;                /* final relative residual of the thermal solve (FP64)                   */
    int64_t step;                    /* steps completed by the context                                         */
} rafem_step_stats;

typedef struct rafem_ctx rafem_ctx;

/* Liver defaults: alpha 0.015, rho_c 3.6e6, perf 2.4e4, T_a 37, dt 1, tol 1e-10, inner_tol 1e-4, FP64, Jacobi,
 * PCG, one corrector pass, automatic SpMV schedule, projection predictor, symmetric lift. */
void rafem_default_params(rafem_params* p);

/* Build a context: validates the mesh (ids in range, non-degenerate tetrahedra), builds the fixed CSR pattern,
 * the element-to-slot map and the element colouring on the host, uploads everything, precomputes element
 * geometry on the device, assembles the constant thermal matrix and sets T = T_a, V = 0 (Dirichlet values
 * applied). stream: a cudaStream_t or NULL. On failure *out is NULL. Ownership of *out passes to the caller,
 * released with rafem_destroy. Errors: BAD_INPUT, BAD_MESH, OOM, CUDA. */
int rafem_create(const rafem_mesh* mesh, const rafem_params* params, void* stream, rafem_ctx** out);

/* Assemble one system into the context's device buffers (Sec. II-A, element equations from updated values;
 * Sec. III-A race-free assembly): which = RAFEM_SYS_V builds A_V(sigma(T)) and its lifted right-hand side
 * from the current temperature; which = RAFEM_SYS_T builds the thermal right-hand side from the current
 * potential and temperature (the thermal matrix is constant and assembled at create). Errors: BAD_INPUT, CUDA. */
int rafem_assemble(rafem_ctx* ctx, int which);

/* Solve the assembled system `which` in place (warm start from the current field), with the context's
 * solver settings; fills *stats (nullable) for that system. Returns OK, NOT_CONVERGED or an error. */
int rafem_solve(rafem_ctx* ctx, int which, rafem_step_stats* stats);

/* One backward-Euler time step (the corrector pass of Sec. II-A): assemble V, solve V, assemble T, solve T.
 * With n_corrector > 1 the pass repeats on the device (sigma at the newest temperature iterate, mass term at T^n)
 * until max |T^{k+1} - T^k| < corrector_tol (status NOT_CONVERGED when n_corrector passes did not get there);
 * stats->correctors holds the passes taken. stats: nullable. */
int rafem_solve_step(rafem_ctx* ctx, rafem_step_stats* stats);

/* n_steps time steps, each launched as one captured CUDA graph, with no host<->device traffic between steps
 * (only the statistics of the last step are copied back). last: nullable, receives the statistics of the
 * last step and, in status, the worst status met over all steps. */
int rafem_run(rafem_ctx* ctx, int32_t n_steps, rafem_step_stats* last);

/* One time step with its state in host memory (as rafem_set_state at the current step, rafem_solve_step and
 * rafem_get_field in one call): T_in and V_in (N doubles each, nullable) replace the state before the step, T_out
 * and V_out (nullable, may be the same buffers as the inputs) receive the fields after it; the predictor history
 * is kept. The copies overlap the step where the data allows: V goes in while the potential is assembled and
 * comes out while the thermal system is assembled and solved, on a second stream; T goes in first and out last.
 * Pinned host buffers let the whole step (copies included) run as one captured graph, rebuilt when the buffers
 * change; pageable buffers work with direct launches. Returns like rafem_solve_step. */
int rafem_step_host(rafem_ctx* ctx, const double* T_in, const double* V_in, double* T_out, double* V_out,
                    rafem_step_stats* stats);

/* Copy a field (RAFEM_SYS_V = potential, RAFEM_SYS_T = temperature) of N doubles to dst.
 * dst_on_device: 0 = host pointer, 1 = device pointer. */
int rafem_get_field(rafem_ctx* ctx, int which, double* dst, int dst_on_device);

/* Replace the state: T and V (either may be NULL to keep it) of N doubles each; on_device as above. The step
 * counter is set to `step`. Dirichlet values are not re-imposed (the caller passes consistent fields). When
 * `step` differs from the context's current step count the predictor's history is cleared (the next step starts
 * its solves from the given fields); when it is equal the run continues and the history is kept. */
int rafem_set_state(rafem_ctx* ctx, const double* T, const double* V, int on_device, int64_t step);

/* Reverse Cuthill-McKee node order of a mesh (host only, no device work): perm [n_nodes] receives perm[new] = old.
 * Meshes whose node numbering has no locality (exported from unstructured generators, shuffled) lose the
 * coalescing of the solver's gathers and the 16-bit column deltas; renumbering them by this order before
 * rafem_create restores both. Per connected component (in order of its lowest node): start at its smallest-degree
 * node (lowest index on ties), move to the smallest-degree node of the last breadth-first level while that
 * increases the eccentricity, number breadth first with unvisited neighbours in increasing (degree, index), and
 * reverse the whole order. tets: [n_tets*4] host. Errors: BAD_INPUT (index out of range), OOM. */
int rafem_reorder_rcm(int32_t n_nodes, int32_t n_tets, const int32_t* tets, int32_t* perm);

/* Sizes of the fixed CSR pattern: n_rows (= N), nnz, number of element colours. Any out pointer may be NULL. */
int rafem_pattern_info(rafem_ctx* ctx, int32_t* n_rows, int64_t* nnz, int32_t* n_colors);

/* ---- batching form ----------------------------------------------------------------------------------------
 * Many independent instances (meshes of different sizes, electrode settings and tissue properties, one set of
 * physics/solver parameters) in one context: every step assembles all instances and solves all of them in one
 * persistent launch per system, each instance with its own Krylov scalars and convergence test (an instance
 * that has converged stops iterating while the others continue). The paper simulates one case per run
 * (Sec. II-A); the batch is this library's answer to evaluating many treatment cases.
 * The instances' nodes are laid out one after the other, each starting at a multiple of 32 (the nodes in
 * between are isolated and carry zero potential / T_a), so rafem_get_field, rafem_set_state and
 * rafem_get_system address the concatenated fields; rafem_batch_info gives each instance's first node. */
#define RAFEM_MAX_BATCH 96

/* n in [1, RAFEM_MAX_BATCH]; meshes[i] as for rafem_create (host pointers, copied). Errors as rafem_create. */
int rafem_batch_create(int32_t n, const rafem_mesh* const* meshes, const rafem_params* params, void* stream,
                       rafem_ctx** out);
/* n_inst (nullable) and node_offsets [n_inst + 1] (nullable): first node of each instance, then the total. */
int rafem_batch_info(rafem_ctx* ctx, int32_t* n_inst, int32_t* node_offsets);
/* Statistics of the last step per instance, per_instance [n_inst] (host). The step statistics returned by
 * rafem_solve_step / rafem_run summarise all instances (worst status, largest iteration counts and residuals). */
int rafem_batch_stats(rafem_ctx* ctx, rafem_step_stats* per_instance);
/* n_steps time steps of every instance of a batch context (rafem_run on that context: one captured step graph per
 * step, each system solved for all instances in one persistent launch), then the statistics of the last step per
 * instance into per_instance [n_inst] (host, nullable) as rafem_batch_stats. Returns the worst status over all
 * steps and instances (OK, NOT_CONVERGED or an error). Also valid on a single-instance context (n_inst = 1). */
int rafem_batch_run(rafem_ctx* ctx, int32_t n_steps, rafem_step_stats* per_instance);

/* Work schedule of the persistent solvers: rows per work tile (tiles never straddle batch instances; rounded up
 * to a multiple of 32 for SELL-32). 0 = automatic. Rebuilds only the tile arrays (cheap) and drops the captured
 * step graph; used by the autotuner. rafem_get_schedule reports the tile size, tile count and solver grid. */
int rafem_set_schedule(rafem_ctx* ctx, int32_t rows_per_tile);
int rafem_get_schedule(rafem_ctx* ctx, int32_t* rows_per_tile, int32_t* n_tiles, int32_t* grid);

/* Storage actually used by the solver: kernel_code 1 = SELL-32 with 32-bit columns, 2 = SELL-32 with 16-bit
 * column deltas, 3 = SELL-32 whose 32-row slices each share one column pattern (chosen at create when that adds
 * at most 2% of stored entries, as on lattice-numbered meshes: the ring solvers then stream matrix values only),
 * 4/8/16/32 = CSR with that many lanes per row; nnz_stored includes slice padding; column_bytes is the size of the
 * per-entry columns, 2 or 4 (read by the other passes, and by the solvers unless kernel_code is 3); assembly is the
 * RAFEM_ASSEMBLY_* in use; arith is RAFEM_ARITH_FP64 or RAFEM_ARITH_DW (what RAFEM_ARITH_AUTO resolved to). Any out
 * pointer may be NULL. */
int rafem_layout_info(rafem_ctx* ctx, int32_t* kernel_code, int64_t* nnz_stored, int32_t* column_bytes,
                      int32_t* assembly, int32_t* arith);

/* Copy the current lifted system `which` to host buffers: row_ptr [N+1], col [nnz], vals [nnz], rhs [N].
 * Any pointer may be NULL to skip it. For inspection and tests. */
int rafem_get_system(rafem_ctx* ctx, int which, int32_t* row_ptr, int32_t* col, double* vals, double* rhs);

/* Solve A x = b for an arbitrary right-hand side on the context's lifted system `which` with the context's
 * solver settings, without touching the fields: b and x are device pointers to N doubles, x holds the
 * initial guess on entry. */
int rafem_solve_rhs(rafem_ctx* ctx, int which, const double* b_dev, double* x_dev, rafem_step_stats* stats);

/* Monolithic contexts only: assemble the coupled Newton system at the current state (T_old = T) and copy it out
 * (host): blocks [4 nnz] = the 2 x 2 block of each entry of the CSR node pattern, row-major (dR_V/dV, dR_V/dT,
 * dR_T/dV, dR_T/dT); residual [2N] interleaved (R_V, R_T per node). Either may be NULL. BAD_INPUT otherwise. */
int rafem_get_coupled_system(rafem_ctx* ctx, double* blocks, double* residual);

/* y = A x with the current lifted system `which` (FP64). x, y: device pointers to N doubles. */
int rafem_spmv(rafem_ctx* ctx, int which, const double* x_dev, double* y_dev);

/* Region timing (the paper's trace regions of Sec. III-C: Assembly, Solve, memcpyH2D, memcpyD2H, plus Predict),
 * measured
 * with CUDA events on the context's stream. While tracing is on, rafem_solve_step and rafem_run launch each
 * region directly (no graph) with an event on each side and NVTX ranges of the same names. */
typedef struct rafem_trace {
    int64_t steps;                   /* traced steps accumulated                                              */
    int64_t iters_V, iters_T;        /* Krylov iterations over the traced steps                              */
    int64_t solves;                  /* traced solves of each system                                          */
    int64_t refine_V;                /* FP64 refinements of the potential solves (mixed precision)           */
    double  ms_assemble_V;           /* "Assembly" of the potential system (matrix + lifted rhs)             */
    double  ms_solve_V;              /* "Solve" of the potential system (one persistent solver launch)       */
    double  ms_assemble_T;           /* "Assembly" of the thermal rhs (Joule + mass term)                     */
    double  ms_solve_T;              /* "Solve" of the thermal system                                         */
    double  ms_memcpy_h2d;           /* rafem_set_state copies                                                */
    double  ms_memcpy_d2h;           /* rafem_get_field copies                                                */
    double  ms_predict_V;            /* "Predict": initial guess of the potential solve (extrapolation or
                                        projection)                                                            */
    double  ms_predict_T;            /* "Predict" of the thermal solve                                        */
} rafem_trace;

/* enable: 1 = on (accumulators cleared), 0 = off. */
int rafem_set_tracing(rafem_ctx* ctx, int enable);
/* Copy the accumulated region timings to *out. */
int rafem_get_trace(rafem_ctx* ctx, rafem_trace* out);

/* Solve A x = b with the library's persistent FP64 Jacobi-PCG for a CSR system the caller already holds on the
 * device, without allocating any memory. The paper has no counterpart: it exists for callers that cannot call
 * cudaMalloc when they need a solve, such as code inside a framework whose caching allocator already owns the
 * device's memory (a cudaMalloc there can fail, or force the allocator to release its cache), or a latency-bound
 * loop that cannot absorb the device-wide synchronisation of cudaMalloc/cudaFree. It calls no allocation routine;
 * the caller passes only its inputs and outputs.
 *
 * Working memory comes from one fixed device array of RAFEM_NOALLOC_SCRATCH_BYTES (7 MiB) inside the library,
 * present on every device that loads the library until the process exits. Hence:
 *   - n_rows must be in [1, RAFEM_NOALLOC_MAX_ROWS]; larger systems are rejected with RAFEM_ERR_BAD_INPUT
 *     before any device work.
 *   - Every call on a device shares that array and leaves its contents behind; the entry point clears what must
 *     start at zero itself. Calls whose GPU work overlaps in time (different streams, or different host threads
 *     on the same device) race on the array and give wrong results: serialise them.
 *   - The first call on each device looks up the array's device address (cudaGetSymbolAddress, with that device
 *     current) and keeps it for the life of the process. After cudaDeviceReset the kept address is stale: do not
 *     call this entry point on a device after resetting it.
 * The call is synchronous: it waits on the stream twice (after the input check, and after the solve) and reads
 * the check's result and the solver's statistics back into host memory before it returns.
 * Arguments (device pointers unless stated): row_ptr [n_rows+1] and col [row_ptr[n_rows]] int32 CSR pattern,
 * every row storing its diagonal entry and every column in [0, n_rows) (else RAFEM_ERR_BAD_INPUT, with x left
 * untouched); vals [row_ptr[n_rows]] FP64 values of a symmetric positive-definite matrix; b [n_rows]; x [n_rows]
 * initial guess on entry, solution on exit. tol: relative residual ||b - A x|| / ||b||; max_iter: iteration cap.
 * stream: cudaStream_t or NULL (legacy default stream). stats (host, nullable): status, iters_V = iterations,
 * relres_V = final relative residual, other fields 0. Returns OK, NOT_CONVERGED, BAD_INPUT, BREAKDOWN, NONFINITE,
 * TIMEOUT or CUDA. */
#define RAFEM_NOALLOC_MAX_ROWS 131072
#define RAFEM_NOALLOC_SCRATCH_BYTES 7340032
int rafem_pcg_csr_noalloc(int32_t n_rows, const int32_t* row_ptr, const int32_t* col, const double* vals,
                          const double* b, double* x, double tol, int32_t max_iter, void* stream,
                          rafem_step_stats* stats);

/* ---- dynamic step size ---------------------------------------------------------------------------------------
 * The main loop advances in dynamically sized steps (Sec. II-A); a step whose corrector passes do not converge
 * within the maximum number of passes is not accepted and the step size is halved, so the simulation still ends
 * at the requested time (Sec. IV). */

/* Which step graphs are in use: 1 = captured and instantiated, 0 = capture failed (direct launches / host loop),
 * -1 = not built yet (built at the first step). corrector_graph is the conditional-loop graph of n_corrector > 1.
 * step_kernels: kernel launches per step of the captured step graph (0 when there is none). Any out pointer may
 * be NULL. */
int rafem_graph_info(rafem_ctx* ctx, int32_t* step_graph, int32_t* corrector_graph, int32_t* step_kernels);

/* Change the step size: reassembles the thermal matrix (and its ILU(0) factors) for the new dt. Ends any tape. */
int rafem_set_dt(rafem_ctx* ctx, double dt);

/* Change the solver tolerances of a live context (the state and the predictor history are kept): tol, the
 * relative residual to reach (> 0), and, when inner_tol > 0, the mixed solver's inner reduction (< 1); inner_tol
 * <= 0 keeps the current one. The captured step graphs are rebuilt at the next step. Errors: BAD_INPUT. */
int rafem_set_tol(rafem_ctx* ctx, double tol, double inner_tol);

/* Bounded device waits. Every wait inside a persistent solver kernel (the grid barriers between its phases and the
 * shared-memory copy slots of the matrix stream) gives up after limit_ns nanoseconds of wall-clock time, records
 * RAFEM_ERR_TIMEOUT and lets the kernel return, so a wait that cannot end costs at most that long and leaves the
 * context usable (its fields hold whatever the interrupted solve left; rafem_reset or rafem_set_state restores a
 * defined state). limit_ns <= 0 restores the default of 5 s. missing_arrivals (for testing the timeout path; 0 in
 * normal use, at most 1024): the following solver launches start their grid-barrier counter that many arrivals
 * short, so their first barrier cannot complete, its waits run out after limit_ns and the solve returns
 * RAFEM_ERR_TIMEOUT, without a fault. The captured step graphs are rebuilt at the next step. Errors: BAD_INPUT. */
int rafem_set_wait_limit(rafem_ctx* ctx, int64_t limit_ns, int32_t missing_arrivals);

typedef struct rafem_advance_stats {
    int32_t status;                  /* worst status of the accepted steps                                     */
    int32_t accepted;                /* steps accepted                                                        */
    int32_t rejected;                /* steps rejected (corrector not converged) and retried with dt / 2      */
    int32_t passes;                  /* corrector passes over the accepted steps (0 for lagged steps)         */
    double  dt;                      /* step size at the end (halvings persist; the last step may be shorter) */
    double  time;                    /* simulated time advanced (= duration)                                  */
} rafem_advance_stats;

/* Advance the state by `duration` seconds in steps of the current dt, the last one shortened to end exactly at
 * `duration`. With n_corrector > 1 each step runs its corrector passes on the device (one CUDA graph whose
 * conditional loop repeats the pass until max |T^{k+1} - T^k| < corrector_tol or n_corrector passes are done); a
 * step that did not converge is discarded (fields and statistics restored) and retried with half the step size,
 * kept for later steps. When half the size would fall below dt_min the step is accepted unconverged (status
 * NOT_CONVERGED). One small read-back per attempted step decides acceptance. Lagged steps (n_corrector = 1) are
 * always accepted. Ends any tape. stats: nullable. */
int rafem_advance(rafem_ctx* ctx, double duration, double dt_min, rafem_advance_stats* stats);

/* ---- preconditioner inspection ----------------------------------------------------------------------------
 * ILU(0) (Sec. II-B preconditioning): the factors are those of P A P^T, where P sorts the rows by level (greedy
 * colour or dependency level, stable within a level; rafem_params.ilu_order) so that rows of one level never
 * depend on each other; levels are solved one after the other. The potential system is refactored after every
 * assembly, the constant thermal system once (and again when k changes). */

/* n_levels, padded_rows (rows of the level-ordered layout, each level padded to a multiple of 32), nnz_stored
 * (entries of its SELL-32 storage of P A P^T, padding included), order [N] (host): the original row of the k-th
 * row in factor order; factor_stored: entries of the solver's SELL-32 layouts of L and of the strictly upper part
 * of U (padding included); column_bytes: column bytes the ILU(0) solver streams per stored entry, 0 when its
 * layouts share one column pattern per 32-row slice, else 4. Any out pointer may be NULL. Returns BAD_INPUT unless
 * the context uses RAFEM_PRECOND_ILU0. */
int rafem_precond_info(rafem_ctx* ctx, int32_t* n_levels, int32_t* padded_rows, int64_t* nnz_stored,
                       int32_t* order, int64_t* factor_stored, int32_t* column_bytes);

/* ILU(0) factors of system `which` mapped back onto the original CSR pattern (host, [nnz]): the entry of (i, j)
 * holds L_ij (below the diagonal of P A P^T, unit diagonal implied) or U_ij (diagonal and above), where "below"
 * refers to the factor order. BAD_INPUT unless ILU(0) is in use. */
int rafem_get_precond(rafem_ctx* ctx, int which, double* factors);

/* z = M^-1 r with the context's preconditioner for system `which` (ILU(0): forward and backward level sweeps;
 * Jacobi: r / diag(A)). r_dev, z_dev: device pointers to N doubles (distinct). */
int rafem_precond_apply(rafem_ctx* ctx, int which, const double* r_dev, double* z_dev);

/* ---- differentiation form ----------------------------------------------------------------------------------
 * Gradients of a loss on the final fields with respect to the per-element conductivities sigma0 and k (and the
 * initial temperature), by the discrete adjoint of the lagged time step (n_corrector = 1): back-propagating
 * through step n solves A_T mu = dL/dT^{n+1} and K(sigma(T^n)) nu = h (both systems are symmetric, so the
 * transposed solves use the same solver), then accumulates the element terms. The forward states the backward
 * pass needs are recomputed segment by segment from checkpoints written every `checkpoint_every` steps. The
 * paper runs the forward model only (Sec. II-A); this form exists for calibrating tissue properties. */

/* Reset the state to the initial condition of rafem_create (T = T_a, V = 0, Dirichlet values applied), step 0,
 * predictor history cleared; ends any tape. */
int rafem_reset(rafem_ctx* ctx);

/* Replace the per-element sigma0 [E] and/or k [E] (either may be NULL to keep it; mesh element order; for a batch
 * the instances' elements one after the other). on_device: 0 = host pointers (checked for finite values),
 * 1 = device pointers (not checked). The constant thermal matrix is reassembled when k changes. Ends any tape. */
int rafem_set_params(rafem_ctx* ctx, const double* sigma0, const double* k, int on_device);
/* The same from FP32 device arrays (the usual storage of trainable per-element parameters, e.g. torch tensors):
 * sigma0_dev [E] and/or k_dev [E] (either may be NULL to keep it), widened to FP64 by the library on its stream.
 * Values are not checked for finiteness. Ends any tape. Errors: BAD_INPUT, OOM, CUDA. */
int rafem_set_params_device(rafem_ctx* ctx, const float* sigma0_dev, const float* k_dev);

/* Start recording: the current state is the tape's origin (checkpoint 0); every later time step taken by
 * rafem_run or rafem_solve_step stores a checkpoint of the state (fields, predictor history, statistics) each time
 * (step - origin) is a multiple of checkpoint_every (>= 1). Checkpoint memory: 8 N doubles each, kept for reuse
 * until rafem_destroy. Requires n_corrector = 1. rafem_set_state, rafem_reset, rafem_set_params and rafem_solve end
 * the tape. Errors: BAD_INPUT. */
int rafem_tape_begin(rafem_ctx* ctx, int32_t checkpoint_every);

typedef struct rafem_adjoint_stats {
    int32_t status;                  /* worst status of the adjoint solves                                   */
    int32_t forward_status;          /* worst status of the recomputed forward steps                          */
    int32_t steps;                   /* steps back-propagated (current step - tape origin)                    */
    int32_t segments;                /* checkpoint segments recomputed                                         */
    int64_t iters_V, iters_T;        /* Krylov iterations of the adjoint potential / thermal solves           */
    double  ms;                      /* wall time of the call                                                  */
} rafem_adjoint_stats;

/* Back-propagate from the current state to the tape origin. Inputs (N doubles each; in_on_device 0 = host,
 * 1 = device): dL_dT = dL/dT at the current step (required), dL_dV = dL/dV at the current step (nullable; the
 * potential of the last step). Outputs (nullable; out_on_device as above): dL_dsigma0 [E] and dL_dk [E] in mesh
 * element order, dL_dT0 [N] = dL/dT at the tape origin with respect to every entry of that state vector (Dirichlet
 * entries included: they enter the first step through sigma(mean T) and the mass term); out_on_device = 2 writes
 * dL_dsigma0 and dL_dk as FP32 device arrays (float* passed through the double* arguments; dL_dT0 stays FP64 on the
 * device), the gradients of rafem_set_params_device's parameters. Entries of dL_dT and dL_dV
 * on Dirichlet nodes are ignored for steps after the origin (those values are fixed). The forward state of the
 * context is left exactly as it was. Returns the worse of the adjoint and recomputation statuses (OK or
 * NOT_CONVERGED), or BAD_INPUT (no tape), OOM, CUDA. stats: nullable. */
int rafem_adjoint(rafem_ctx* ctx, const double* dL_dT, const double* dL_dV, int in_on_device, double* dL_dsigma0,
                  double* dL_dk, double* dL_dT0, int out_on_device, rafem_adjoint_stats* stats);

/* Release every device and host resource of the context. NULL is accepted. */
void rafem_destroy(rafem_ctx* ctx);

/* Human-readable name of a status code (static storage). */
const char* rafem_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* RAFEM_H */
