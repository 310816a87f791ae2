/*
 * cgp.h -- C ABI of the GB300 (sm_103a) coarse-grid-projection (CGP) pressure-correction library.
 *
 * The library advances the incompressible Navier-Stokes equations by the IFE-CGP scheme of
 * Kashefi & Staples, "A Finite-Element Coarse-Grid Projection Method" (Sect. 2.2, Eqs. 19-23):
 * a semi-implicit P1 momentum solve on a fine triangle mesh, injection of the intermediate
 * velocity onto the coarse mesh, a coarse pressure Poisson solve, prolongation of the pressure
 * through parent/child tables (Eq. 29) and a consistent-mass velocity correction.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Return value: CGP_OK (0) or one of the CGP_ERR_* codes below; cgp_status_str() names it.
 * - Pointers named *_host are host memory; pointers named *_dev are device memory on the device
 *   that was current when the context was created. All of them are owned by the caller; the
 *   library copies what it keeps and never frees caller memory.
 * - Layouts: node fields are float64, contiguous; velocity-like fields are interleaved
 *   [n][2] = (x, y) pairs; triangles are int32 [t][3] counter-clockwise.
 * - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream). Calls that
 *   take a stream are asynchronous and stream-ordered: they enqueue kernels and return; errors
 *   found on the device (no convergence, NaN, a device wait that ran out) are recorded in the
 *   context's device status and read back by cgp_get_stats().
 * - Ordering: the fine mesh numbering is fixed by the refinement rule of cgp_mesh_create().
 * - A context is not thread-safe; use one context per host thread or serialise calls.
 */
#ifndef CGP_H
#define CGP_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------------- */
#define CGP_OK                 0
#define CGP_ERR_ARG            1  /* a NULL pointer, a size out of range or an unknown option      */
#define CGP_ERR_MESH           2  /* bad orientation, index out of range, non-manifold edge        */
#define CGP_ERR_CUDA           3  /* a CUDA runtime call failed                                    */
#define CGP_ERR_NOT_CONVERGED  4  /* a solve hit max_iter; its result is still written             */
#define CGP_ERR_NAN            5  /* a non-finite residual or inner product                        */
#define CGP_ERR_TIMEOUT        6  /* a bounded device-side wait gave up (grid barrier)             */
#define CGP_ERR_NOMEM          7  /* device or host allocation failed                              */
#define CGP_ERR_STATE          8  /* call out of order (e.g. a step before cgp_set_bc)             */

/* ---- precision modes --------------------------------------------------------------------- */
#define CGP_FP64   0  /* every Krylov iteration in FP64                                            */
#define CGP_MIXED  1  /* FP32 inner Krylov iterations inside FP64 iterative refinement for the     */
                      /* momentum, Poisson and mass-matrix solves; true residuals, refinement      */
                      /* updates and the velocity correction itself stay FP64                      */

/* ---- boundary masks ------------------------------------------------------------------------ */
#define CGP_BC_U   1  /* bit 0 of a fine-node velocity mask: x-velocity prescribed (Eqs. 3, 10)   */
#define CGP_BC_V   2  /* bit 1: y-velocity prescribed                                             */

typedef struct cgp_ctx_s* cgp_ctx;

/* Physical and solver parameters. rho, mu, dt: density, dynamic viscosity and time step of the
 * semi-implicit BDF1 scheme (Eqs. 5-8). levels: number l of 1:4 refinements from the pressure
 * (coarse) mesh to the velocity (fine) mesh (Sect. 2.2); l = 0 is the standard scheme.
 * rtol: every solve stops when ||b - A x||_2 <= rtol ||b||_2 for each right-hand side (the
 * paper's Sect. 2.3 uses 1e-8); for the momentum system ||b|| is that of the row-scaled system
 * in which a Dirichlet row reads A_ii x_i = A_ii g_i. inner_rtol: CGP_MIXED only, the FP32 inner solve's reduction of
 * the FP64 residual per refinement pass (0 = default 1e-4). max_iter: cap on the total number of
 * Krylov iterations of one solve. max_outer: cap on refinement passes (0 = default 30).
 * spmv_lanes: lanes per CSR row in the SpMV inner loops (0 = let cgp_autotune()/default decide;
 * otherwise 1, 2, 4, 8, 16 or 32). block_threads: threads per block of the generic persistent
 * kernels (0 = default 512, else 256..512, a multiple of 32). coarse_solver: 0 = automatic (kernel 3 whenever the
 * coarse matrix slice of a block fits in shared memory, else the generic kernel), 1 = the generic
 * Jacobi-preconditioned classical CG kernel, 2 = the on-chip Jacobi-preconditioned pipelined CG
 * kernel in CGP_FP64 (CGP_MIXED falls back to kernel 5), 3 = on-chip classical CG with a
 * two-level additive Schwarz preconditioner applied in FP32 (one subdomain per block of a
 * Hilbert-curve renumbering of the nodes; local solver: a Chebyshev polynomial of degree
 * precond_degree in D^-1 A on the subdomain; coarse space: the constant and the two linear
 * functions on every subdomain, Galerkin matrix inverted on the host), 4 = kernel 3 with the
 * preconditioner in the iteration precision, 5 = the on-chip Jacobi-preconditioned classical CG
 * kernel. Explicit choices 2..5 fall back to the generic kernel when the slice does not fit.
 * precond_degree: 0 = default 6. precond_ratio: lambda_max / lambda_min of the Chebyshev
 * interval (0 = default 30). */
typedef struct {
    double rho, mu, dt;
    int levels;
    int precision;
    double rtol;
    double inner_rtol;
    int max_iter;
    int max_outer;
    int spmv_lanes;
    int block_threads;
    int coarse_solver;
    int spmv_format;   /* stand-alone fine SpMV (cgp_spmv): 0 = CSR until cgp_autotune picks the faster of
                          CSR and sliced ELL, 1 = sliced ELL, 2 = CSR */
    int precond_degree;
    double precond_ratio;
    int warm_start;    /* initial guesses of the solves of a step: 0 = u^n (momentum), p^n, w^n
                          (coarse Poisson, mass); 1 = u^n + (u~^n - u^(n-1)) (the last converged
                          momentum increment, repeated) and the linear extrapolations
                          2 v^n - v^(n-1) of p and w; 2 = the same with the quadratic
                          extrapolations 3 v^n - 3 v^(n-1) + v^(n-2) once three values exist; 3
                          (default) = the cubic extrapolations 4 v^n - 6 v^(n-1) + 4 v^(n-2) -
                          v^(n-3) once four exist and the momentum guess u^n + 2 dx^n - dx^(n-1)
                          (dx the converged increments) once two exist; lower orders until the
                          history is long enough; history kept by the
                          context (cgp_step, the batched step, cgp_momentum_solve,
                          cgp_prolong_correct for w, cgp_predict_pressure for p). cgp_set_bc clears
                          the history */
    int mass_degree;   /* preconditioner of the consistent-mass solve (Eq. 23): 1 = Jacobi, k >= 2 = the
                          degree-k Chebyshev polynomial in D^-1 M on [1/2, 2] (its spectrum for P1
                          triangles), applied in FP32 inside the CG; 0 (default) = 4, except Jacobi
                          for CGP_MIXED on fine meshes of more than 2048 rows per block */
    int momentum_degree; /* preconditioner of the momentum BiCGStab (Eq. 19): 1 = Jacobi, k >= 2 = the
                          degree-k Chebyshev polynomial in D^-1 A on [1/2, G], G the Gershgorin bound
                          of D^-1 A taken by each cgp_assemble, applied in FP32; 0 (default) = 3
                          for CGP_FP64, Jacobi for CGP_MIXED */
    int solver_format; /* matrix layout of the fine-mesh solvers' products (momentum and mass, Eqs. 19
                          and 23): 0 (default) = automatic (CSR until cgp_autotune times the
                          alternatives), 1 = sliced ELL of the natural row order (32-row slices, slot
                          k of a slice's rows contiguous, so each warp load is coalesced), 2 = CSR
                          with spmv_lanes lanes per row. Batched steps always use CSR */
    int restrict_mode; /* coarse right-hand side of the Poisson solve (Eq. 21): 0 (default) = the
                          paper's injection u~_c = u~_f[xi] (Eqs. 20, 30) and b_c = -(rho/dt) D_c u~_c;
                          1 = Galerkin restriction of the fine divergence, b_c = -(rho/dt) P^T D_f u~_f
                          with P the prolongation of Eq. 29 (the coarse test functions integrated
                          against div u~_f); not in the paper */
    int projection;    /* pressure-correction form: 0 (default) = the paper's non-incremental scheme
                          (Eqs. 9-15); 1 = incremental: the momentum right-hand side carries
                          -dt G_f P p_c^n, the Poisson solve of Eq. 21 gives the increment phi, the
                          correction applies phi and p_c^{n+1} = p_c^n + phi; 2 = rotational: as 1 with
                          p_c^{n+1} = p_c^n + phi - mu chi, chi = -(dt/rho) b_c / (lumped coarse mass).
                          The paper's Sect. 4 names these forms as future work; with restrict_mode 0
                          they drift as dt falls (the coarse Laplacian does not match the injected
                          divergence), with restrict_mode 1 they are stable. Single contexts only:
                          cgp_batch_create rejects contexts with projection != 0 */
    int fine_order;    /* storage order of the fine nodes inside the library (levels >= 1): 0 (default)
                          = along a Hilbert curve of their coordinates, so that neighbouring rows and
                          the columns they gather lie close together in memory; 1 = the refinement
                          order. Every fine-mesh array crossing this interface (cgp_fine_mesh,
                          cgp_set_bc, velocities, pf, gp) is in the refinement order either way; the
                          library permutes on the way in and out */
    double momentum_rtol; /* tolerance of the momentum solve (Eq. 19) alone: 0 (default) = rtol / 10
                          (at least 1e-14, at most rtol) with CGP_MIXED, rtol with CGP_FP64. The
                          momentum solve's error reaches the coarse right-hand side and the histories
                          the extrapolated guesses of the later solves are built from; with cheap FP32
                          inner iterations a ten times tighter solve saves more coarse and mass
                          iterations than it costs */
} cgp_params;

/* A coarse mesh: n_nodes points xy_host[n][2] and n_tris counter-clockwise triangles
 * tri_host[t][3] (0-based). The coarse mesh is the pressure mesh V_{4-k} of Sect. 2.2. */
typedef struct {
    int n_nodes, n_tris;
    const double* xy_host;
    const int* tri_host;
} cgp_mesh_desc;

/* Sizes of a context. n_fine/n_coarse: velocity/pressure nodes; nnz_*: CSR entries of the P1
 * pattern (node i couples to itself and its edge neighbours); n_colours: element colours of the
 * fine mesh used by the assembly; grid_blocks: blocks of the persistent solver kernels. */
typedef struct {
    int n_fine, n_coarse, tris_fine, tris_coarse, nnz_fine, nnz_coarse, levels;
    int n_colours, grid_blocks, block_threads, spmv_lanes;
    int coarse_kernel;   /* 0 generic classical CG, 1 on-chip classical CG, 2 on-chip pipelined CG,
                            3 on-chip two-level Schwarz CG, preconditioner in FP32,
                            4 the same, preconditioner in the iteration precision */
    int solver_format;   /* layout of the fine solvers' products: 1 sliced ELL, 2 CSR */
    int fine_order;      /* storage order of the fine nodes: 0 a Hilbert curve, 1 the refinement order
                            (always 1 when levels = 0, where the fine mesh is the coarse one) */
} cgp_info;

/* Per-solve statistics of the most recent step (read back by cgp_get_stats, which synchronises
 * the stream). iters: total inner Krylov iterations; outer: refinement passes; rel_res: final
 * FP64 true relative residual ||b - A x|| / ||b|| (max over the right-hand sides); status: the
 * CGP_* code of that solve. */
typedef struct {
    int momentum_iters, momentum_outer, momentum_status;
    int poisson_iters, poisson_outer, poisson_status;
    int mass_iters, mass_status;
    int barrier_status;
    double momentum_rel_res, poisson_rel_res, mass_rel_res;
} cgp_stats;

/* Fill *p with the defaults: rho = 1, mu = 0.01, dt = 0.01, levels = 1, CGP_FP64, rtol = 1e-8,
 * inner_rtol = 1e-4, max_iter = 20000, max_outer = 30, spmv_lanes = 0, block_threads = 0,
 * coarse_solver = 0, spmv_format = 0, precond_degree = 0, precond_ratio = 0, warm_start = 3, mass_degree = 0,
 * momentum_degree = 0, solver_format = 0, restrict_mode = 0, projection = 0, fine_order = 0,
 * momentum_rtol = 0 (rtol / 10 with CGP_MIXED, else rtol). p NULL: nothing is written. */
void cgp_default_params(cgp_params* p);

/* Preprocessing (the paper's C_pre, Sect. 2.4): validates the coarse mesh, refines it
 * prm->levels times by conforming 1:4 splits (Sect. 2.2) with the numbering
 *   parents keep 0..N_k-1; one midpoint per edge, appended in order of first visit
 *   (triangles in order, local edges (a,b), (b,c), (c,a)); triangle t = (a,b,c) becomes
 *   4t: (a,m_ab,m_ca), 4t+1: (m_ab,b,m_bc), 4t+2: (m_ca,m_bc,c), 4t+3: (m_ab,m_bc,m_ca),
 * builds the s^p tables of Eq. 29 and the s^u table of Eq. 30, the CSR patterns, the element
 * colouring, uploads them and assembles the constant P1 matrices (Eqs. 16-18) on the device.
 * Host arrays are copied. On success *out owns device memory until cgp_mesh_destroy().
 * Errors: CGP_ERR_ARG (NULL, n <= 0, levels outside 0..4), CGP_ERR_MESH (index out of range,
 * non-positive area, an edge shared by more than two triangles), CGP_ERR_CUDA, CGP_ERR_NOMEM. */
int cgp_mesh_create(const cgp_mesh_desc* coarse, const cgp_params* prm, cgp_ctx* out);

/* Host-only preprocessing query (no device calls): refine the coarse mesh `levels` times with
 * the same rule as cgp_mesh_create() (Sect. 2.2) and report the fine mesh. Call once with NULL
 * outputs to learn *n_fine / *n_tris_fine, then again with buffers: xy_host [n_fine][2],
 * tri_host [n_tris_fine][3], sp_host [n_fine][2] (the s^p pairs of Eq. 29 from level l-1 to
 * level l; for levels = 0 the identity pairs), colour_host [n_tris_fine] (the element colour of
 * the fine assembly). Any output may be NULL. Errors: CGP_ERR_ARG, CGP_ERR_MESH. */
int cgp_refine(const cgp_mesh_desc* coarse, int levels, int* n_fine, int* n_tris_fine, double* xy_host,
               int* tri_host, int* sp_host, int* colour_host);

/* Host-only query (no device calls): the order in which cgp_mesh_create() stores the fine nodes
 * with fine_order = 0 (a data layout of this library, not a step of the paper): the nodes sorted
 * by their position along a Hilbert curve of 2^16 x 2^16 cells spanning the larger side of the
 * mesh's bounding box (ties in the refinement order). perm_host[n_fine] receives, for each stored
 * node i, its index in the refinement order of cgp_refine (the identity when levels = 0): the
 * permutation cgp_fine_order() reports for such a context. Errors: CGP_ERR_ARG, CGP_ERR_MESH. */
int cgp_refine_order(const cgp_mesh_desc* coarse, int levels, int* perm_host);

/* Coarse-pressure predictor for time stepping: pc <- 2 pc - pc_prev (warm_start = 1, or the second
 * call), pc <- 3 pc - 3 pc_prev + pc_prev2 (warm_start = 2, or the third call) or
 * pc <- 4 pc - 6 pc_prev + 4 pc_prev2 - pc_prev3 (warm_start = 3, from the fourth call on), where
 * pc_prev, pc_prev2, pc_prev3 are the pc the context saw at its previous calls (the previous steps'
 * pressures when pc holds the latest one); then the history shifts by the incoming pc. The first
 * call after cgp_set_bc only records pc. pc_dev: [n_coarse] float64, device. Stream-ordered;
 * cgp_step calls it when warm_start >= 1. Errors: CGP_ERR_ARG, CGP_ERR_STATE, CGP_ERR_CUDA. */
int cgp_predict_pressure(cgp_ctx ctx, double* pc_dev, void* stream);

/* Sizes and launch shapes of the context. Host-side; errors: CGP_ERR_ARG (NULL). */
int cgp_mesh_info(cgp_ctx ctx, cgp_info* info);

/* Copy the fine (velocity) mesh out: xy_host[n_fine][2], tri_host[tris_fine][3] and
 * on_boundary_host[n_fine] (1 where the node lies on an edge with a single triangle). Any of
 * the three may be NULL. The coarse mesh is the caller's input. Host-side, in the refinement
 * numbering whatever fine_order is. Errors: CGP_ERR_ARG (NULL context). */
int cgp_fine_mesh(cgp_ctx ctx, double* xy_host, int* tri_host, unsigned char* on_boundary_host);

/* Boundary classes. vel_mask_host[n_fine]: CGP_BC_U / CGP_BC_V bits of velocity-Dirichlet
 * nodes (Eqs. 3, 10); nodes without bits are natural (Eq. 11; nothing is assembled there).
 * p_mask_host[n_coarse]: 1 where the coarse pressure is held at 0 (Eq. 14 on the open boundary,
 * plus one pinned node for enclosed flows whose pure-Neumann problem of Eq. 13 is singular);
 * those rows and columns are eliminated symmetrically. g_host[n_fine][2]: prescribed velocity
 * values (read only where a bit is set). Synchronous. The momentum system must be assembled
 * again afterwards (cgp_momentum_solve and cgp_solver_spmv return CGP_ERR_STATE until then).
 * Errors: CGP_ERR_ARG. */
int cgp_set_bc(cgp_ctx ctx, const unsigned char* vel_mask_host, const unsigned char* p_mask_host,
               const double* g_host);

/* Replace the prescribed velocity values (e.g. time-dependent data at t^{n+1}) from a device
 * array g_dev[n_fine][2] in the refinement numbering (read only where a mask bit is set);
 * stream-ordered copy into the context. Errors: CGP_ERR_ARG (NULL), CGP_ERR_CUDA. */
int cgp_set_dirichlet_values(cgp_ctx ctx, const double* g_dev, void* stream);

/* Step 1 set-up, Eq. 19: A = rho M + dt (rho N(u^n) + mu K) written into the fixed fine CSR
 * pattern from per-element contributions gathered per entry (no atomics, deterministic), the Jacobi diagonal
 * per component, and the right-hand side b = rho M u^n with Dirichlet rows set to the prescribed
 * values. u_dev: [n_fine][2] velocity u^n, read (with fine_order = 0 gathered into the library's
 * stored order; with fine_order = 1 or levels = 0 this buffer is what a later NULL u^n in
 * cgp_momentum_solve reads).
 * Stream-ordered. Errors: CGP_ERR_ARG (NULL), CGP_ERR_STATE (before cgp_set_bc), CGP_ERR_CUDA. */
int cgp_assemble(cgp_ctx ctx, const double* u_dev, void* stream);

/* Step 1, Eq. 19: solve A u~ = b (per component, Dirichlet rows replaced by identity rows) by
 * BiCGStab on both components at once, preconditioned by Jacobi or by the FP32 Chebyshev
 * polynomial of cgp_params.momentum_degree (CGP_MIXED: FP32 BiCGStab inside FP64 iterative
 * refinement). Requires an assembly on the same u^n first (else CGP_ERR_STATE). u_dev: u^n, the initial
 * guess, plus the previous converged increment when warm_start >= 1, or NULL for the velocity of
 * the last assembly (cgp_assemble, cgp_assemble_incremental, cgp_step or a batched step; no second
 * copy into the library's fine order) while a buffer still holds it: with fine_order = 1 or
 * levels = 0 that buffer is the caller's, and once cgp_step, a batched step or cgp_prolong_correct
 * has written u^{n+1} into it (with fine_order = 0: once cgp_body_force or cgp_reattachment has
 * reused the library's copy), NULL returns CGP_ERR_STATE; ut_dev: [n_fine][2]
 * output u~^{n+1}, or NULL to keep u~^{n+1} inside the context for cgp_restrict and
 * cgp_prolong_correct (no copy out of the library's fine order). */
int cgp_momentum_solve(cgp_ctx ctx, const double* u_dev, double* ut_dev, void* stream);

/* Steps 2-3 right-hand side, Eqs. 20-21 with Eq. 30: u~_c = u~_f[xi] (injection), then
 * b_c = -(rho/dt) (Dx_c u~_c,x + Dy_c u~_c,y) with D_ij = int psi_i d phi_j on the coarse mesh,
 * zero at p-masked nodes; with restrict_mode = 1, b_c = -(rho/dt) P^T (Dx_f u~_x + Dy_f u~_y)
 * instead (P^T level by level through inverse child lists of the s^p tables of Eq. 29).
 * ut_dev: [n_fine][2], or NULL for the context's u~ of the last cgp_momentum_solve; bc_dev:
 * [n_coarse] output. Stream-ordered. Errors: CGP_ERR_ARG (NULL context or bc_dev),
 * CGP_ERR_STATE (before cgp_set_bc), CGP_ERR_CUDA. */
int cgp_restrict(cgp_ctx ctx, const double* ut_dev, double* bc_dev, void* stream);

/* Step 3, Eq. 21: solve K_c p_c = b_c (K_c = coarse stiffness, +(-Laplacian), after symmetric
 * elimination of masked nodes) by conjugate gradients in a single persistent kernel, preconditioned
 * as cgp_params.coarse_solver selects (default: two-level additive Schwarz; 5: Jacobi) (CGP_MIXED:
 * FP32 CG inside FP64 iterative refinement). pc_dev [n_coarse] is
 * the initial guess on entry (warm start) and the solution on exit. bc_dev [n_coarse], or NULL
 * for the context's own right-hand side of its latest cgp_step. Stream-ordered. Errors:
 * CGP_ERR_ARG (NULL context or pc_dev), CGP_ERR_STATE (before cgp_set_bc), CGP_ERR_CUDA; the
 * solve's own outcome (CGP_ERR_NOT_CONVERGED, CGP_ERR_NAN, CGP_ERR_TIMEOUT) through cgp_get_stats. */
int cgp_poisson_solve(cgp_ctx ctx, const double* bc_dev, double* pc_dev, void* stream);

/* Steps 4-5, Eqs. 22-23 with Eq. 29: p_f = P p_c level by level, g = G p_f (G_ij = int phi_i
 * d psi_j), w = M^{-1} g by CG on the consistent mass matrix (FP64, or FP32 inside FP64 refinement
 * with CGP_MIXED), preconditioned by Jacobi or the FP32 Chebyshev polynomial of
 * cgp_params.mass_degree, then
 * u = u~ - (dt/rho) w and Dirichlet nodes reset to their prescribed values.
 * pc_dev [n_coarse], ut_dev [n_fine][2] inputs (ut_dev NULL: the context's u~ of the last
 * cgp_momentum_solve); u_dev [n_fine][2] output (may equal ut_dev);
 * pf_dev [n_fine] and gp_dev [n_fine][2] optional outputs (NULL to skip): p_f and w. All fine
 * arrays in the refinement numbering. Stream-ordered. Errors: CGP_ERR_ARG (NULL context, pc_dev or
 * u_dev), CGP_ERR_STATE (before cgp_set_bc), CGP_ERR_CUDA; the mass solve's outcome through
 * cgp_get_stats. */
int cgp_prolong_correct(cgp_ctx ctx, const double* pc_dev, const double* ut_dev, double* u_dev,
                        double* pf_dev, double* gp_dev, void* stream);

/* One whole time step (Eqs. 19-23): assemble, momentum, restrict, Poisson (warm-started from
 * pc_dev), prolong-correct. u_dev [n_fine][2] holds u^n on entry and u^{n+1} on exit; pc_dev
 * [n_coarse] holds p_c^n on entry and p_c^{n+1} on exit. With projection = 1 or 2 the step is
 * cgp_assemble_incremental with p_c^n, the momentum solve, the restriction, the Poisson solve for
 * the increment (warm-started from the extrapolated previous increments), prolong-correct with
 * the increment and cgp_pressure_update. Stream-ordered, no host sync. Errors: CGP_ERR_ARG (NULL),
 * CGP_ERR_STATE (before cgp_set_bc), CGP_ERR_CUDA; the solves' outcomes (CGP_ERR_NOT_CONVERGED,
 * CGP_ERR_NAN, CGP_ERR_TIMEOUT) through cgp_get_stats. */
int cgp_step(cgp_ctx ctx, double* u_dev, double* pc_dev, void* stream);

/* Many coarse Poisson solves (Eq. 21) with the context's matrix in one call: nrhs right-hand
 * sides b_dev [nrhs][n_coarse] and initial guesses / solutions x_dev [nrhs][n_coarse], each solved
 * to the context's rtol by the two-level preconditioned CG of the batched step (Jacobi plus three
 * coarse functions per 256-row subdomain of a Hilbert-curve renumbering), one block per right-hand
 * side, as many right-hand sides per cooperative launch as the GPU holds blocks of that kernel
 * (about two per SM; larger counts go in successive launches). For independent solves of one mesh:
 * the learned warm start's evaluation, or many instances that share a coarse mesh. iters_dev,
 * rel_dev, status_dev [nrhs] (optional): per right-hand side iteration count, final FP64 relative
 * residual and CGP_* status. The first call builds the two-level structures and workspace
 * (synchronously). Coarse meshes of at most 131,072 nodes (else CGP_ERR_ARG). Not in the paper. */
int cgp_poisson_solve_many(cgp_ctx ctx, int nrhs, const double* b_dev, double* x_dev, int* iters_dev, double* rel_dev,
                           int* status_dev, void* stream);

/* Incremental forms, step 1: as cgp_assemble, with the momentum right-hand side
 * rho M u^n - dt G_f P p_c^n (the previous pressure prolonged by Eq. 29 and its fine gradient)
 * at rows that are not velocity-Dirichlet. pc_dev: [n_coarse] p_c^n. Stream-ordered. Not in the
 * paper (its Sect. 4 names the incremental form as future work). Errors: CGP_ERR_ARG (NULL),
 * CGP_ERR_STATE (before cgp_set_bc), CGP_ERR_CUDA. */
int cgp_assemble_incremental(cgp_ctx ctx, const double* u_dev, const double* pc_dev, void* stream);

/* Incremental forms, last step: pc_dev += phi_dev (projection 1), and for projection 2 also
 * - mu chi with chi = -(dt/rho) bc_dev / (lumped coarse mass) (the restricted divergence of u~
 * that the right-hand side bc_dev of the increment's Poisson solve was built from). bc_dev,
 * phi_dev, pc_dev: [n_coarse]. Stream-ordered. Errors: CGP_ERR_ARG, CGP_ERR_STATE (projection 0). */
int cgp_pressure_update(cgp_ctx ctx, const double* bc_dev, const double* phi_dev, double* pc_dev, void* stream);

/* y = A x with the FP32 copy of the momentum matrix of Eq. 19 of the last assembly (cgp_assemble,
 * cgp_assemble_incremental, cgp_step or a batched step)
 * (the full operator rows, Dirichlet rows included), for two interleaved right-hand sides x_dev,
 * y_dev [n_fine][2] (float) in the stored fine order: the product of the fine solvers' FP32
 * iterations as a launch of its own, in their launch shape and layout (solver_format, lanes), for
 * measuring it. Requires CGP_MIXED or momentum_degree >= 2 (else CGP_ERR_STATE) and a prior
 * assembly. Stream-ordered. */
int cgp_solver_spmv(cgp_ctx ctx, const float* x_dev, float* y_dev, void* stream);

/* The library's storage order of the fine nodes: perm_host[n_fine] receives, for each stored node
 * i, its index in the refinement order of cgp_fine_mesh (the identity with fine_order = 1 or
 * levels = 0). Errors: CGP_ERR_ARG. */
int cgp_fine_order(cgp_ctx ctx, int* perm_host);

/* y = A0 x with A0 = rho M + dt mu K (the constant part of the momentum matrix of Eq. 19) on the
 * fine mesh, for two interleaved right-hand sides: x_dev, y_dev [n_fine][2] in the library's
 * stored fine order (cgp_fine_order), the layout the Krylov solvers multiply in. The sliced-ELL
 * or CSR SpMV kernel (cgp_autotune picks) as a stand-alone launch. Stream-ordered. Errors:
 * CGP_ERR_ARG (NULL), CGP_ERR_CUDA. */
int cgp_spmv(cgp_ctx ctx, const double* x_dev, double* y_dev, void* stream);

/* Copy the coarse right-hand side b_c of the context's latest cgp_step (or batched step) to
 * bc_dev [n_coarse] (e.g. to log (b_c, p_c) pairs). Stream-ordered. Errors: CGP_ERR_ARG (NULL),
 * CGP_ERR_CUDA. */
int cgp_copy_coarse_rhs(cgp_ctx ctx, double* bc_dev, void* stream);

/* The same step on host buffers: copies u_host [n_fine][2] and pc_host [n_coarse] to the
 * context's device staging buffers, runs cgp_step, copies both back and synchronises the
 * stream. For best copy speed the host buffers should be page-locked. Errors: CGP_ERR_ARG (NULL),
 * the errors of cgp_step, CGP_ERR_CUDA (a copy). */
int cgp_step_host(cgp_ctx ctx, double* u_host, double* pc_host, void* stream);

/* Synchronise the stream and read the statistics of the latest solves. Returns the first
 * non-OK status among them (CGP_ERR_NOT_CONVERGED, CGP_ERR_NAN, CGP_ERR_TIMEOUT) or CGP_OK. */
int cgp_get_stats(cgp_ctx ctx, void* stream, cgp_stats* st);

typedef struct cgp_batch_s* cgp_batch;
/* ---- batched instances (many independent meshes advanced together) ------------------------
 * A batch advances n contexts (same precision and device, each after cgp_set_bc) by the step of
 * cgp_step, with one cooperative launch per persistent stage for all instances: the grid (up to
 * two blocks per SM) is cut into per-instance block groups, sized by the instance's fine nnz for
 * the fine-mesh solves and by nnz_c * sqrt(n_c) for the coarse CG; barriers and reductions stay
 * inside a group. The coarse solve uses the batched two-level CG (Jacobi plus three coarse
 * functions per 256-row subdomain) when every instance has coarse_solver 0 and fits it, else the
 * generic Jacobi CG. The gathers between stages (restriction, prolongation, gradient, correction)
 * are one launch per stage for all instances (per instance when one uses restrict_mode 1). Not in
 * the paper: a systems pattern for many small problems.
 * u_devs[i] [n_fine_i][2] and pc_devs[i] [n_coarse_i] are the instances' state, caller-owned
 * device buffers that must stay valid until cgp_batch_destroy. Contexts with projection != 0 are
 * rejected (CGP_ERR_ARG). Errors: CGP_ERR_ARG (NULL, n <= 0, mixed precisions or devices, a
 * context with projection != 0), CGP_ERR_STATE (a context before cgp_set_bc), CGP_ERR_NOMEM,
 * CGP_ERR_CUDA. */
int cgp_batch_create(cgp_ctx* ctxs, int n, double* const* u_devs, double* const* pc_devs, cgp_batch* out);
/* Launch shape: total blocks and each instance's group sizes (arrays of n, may be NULL).
 * Host-side; errors: CGP_ERR_ARG (NULL batch). */
int cgp_batch_info(cgp_batch b, int* blocks, int* group_fine, int* group_coarse);
/* One step of every instance, stream-ordered. Errors: CGP_ERR_ARG (NULL), CGP_ERR_CUDA; the
 * instances' solver outcomes through cgp_batch_get_stats. */
int cgp_batch_step(cgp_batch b, void* stream);
/* `steps` steps of every instance by replaying a CUDA graph of one step (captured on an internal
 * stream at the first call; make the first call outside any other stream capture).
 * Errors: CGP_ERR_ARG (NULL batch, steps < 0), CGP_ERR_CUDA (capture, instantiation or launch). */
int cgp_batch_run(cgp_batch b, int steps, void* stream);
/* Only the coarse Poisson stage (Eq. 21) of every instance, one batched launch: instance i solves
 * its context's last coarse right-hand side (from the latest step or cgp_restrict into the
 * context) into pc_devs[i], which is also the initial guess. Stream-ordered. Errors:
 * CGP_ERR_ARG (NULL), CGP_ERR_CUDA. */
int cgp_batch_poisson_solve(cgp_batch b, void* stream);
/* Synchronise and read every instance's statistics into per_instance[n]; returns the first
 * non-OK status (an instance's solver or barrier status, or CGP_ERR_CUDA), CGP_ERR_ARG for NULL. */
int cgp_batch_get_stats(cgp_batch b, void* stream, cgp_stats* per_instance);
/* Free the batch (not the contexts); synchronises the device first. NULL is accepted. Returns
 * CGP_OK. */
int cgp_batch_destroy(cgp_batch b);

/* ---- learned warm start for the coarse solve (not in the paper) -----------------------------
 * A BF16 network n -> H -> H -> n with GELU (tanh form) maps a coarse right-hand side b to an
 * initial guess p = ||b|| NN(b / ||b||) for the Poisson solve of Eq. 21 (the solve is linear in b);
 * PCG still runs to the same tolerance, so the network only changes the iteration count. Products
 * run on tcgen05 tensor cores (BF16 operands, FP32 accumulation); training uses Adam on FP32
 * master weights. Weights are row-major [out][in]. */
typedef struct cgp_ws_s* cgp_ws;

/* C[M][N] (float32, row-major) = A[M][K] * B[N][K]^T with A, B bfloat16 row-major device arrays
 * (K contiguous, 16-byte aligned). Requires M % 128 == 0, N % 128 == 0, K % 64 == 0 (else
 * CGP_ERR_ARG). Stream-ordered. The tensor-core product the network is built from. */
int cgp_gemm_bf16(int M, int N, int K, const void* A_dev, const void* B_dev, float* C_dev, void* stream);
/* Network for n unknowns, hidden width H (H % 128 == 0), up to batch_max right-hand sides per call.
 * Errors: CGP_ERR_ARG (NULL out, n, H or batch_max out of range), CGP_ERR_NOMEM, CGP_ERR_CUDA. */
int cgp_ws_create(int n, int hidden, int batch_max, cgp_ws* out);
/* Host float32 weights: W1 [H][n], b1 [H], W2 [H][H], b2 [H], W3 [n][H], b3 [n]; resets Adam.
 * Synchronous. Errors: CGP_ERR_ARG (NULL), CGP_ERR_CUDA. */
int cgp_ws_set_params(cgp_ws w, const float* W1, const float* b1, const float* W2, const float* b2, const float* W3,
                      const float* b3);
/* Copy the FP32 master weights out (host arrays of the same shapes; NULL skips one). Synchronous.
 * Errors: CGP_ERR_ARG (NULL network), CGP_ERR_CUDA. */
int cgp_ws_get_params(cgp_ws w, float* W1, float* b1, float* W2, float* b2, float* W3, float* b3);
/* Gradients of the latest cgp_ws_train_step (same shapes as the weights; NULL skips one).
 * Synchronous. Errors: CGP_ERR_ARG (NULL network), CGP_ERR_CUDA. */
int cgp_ws_get_grads(cgp_ws w, float* dW1, float* db1, float* dW2, float* db2, float* dW3, float* db3);
/* held_host[n]: 1 for pressure-held entries (output forced to 0, excluded from the loss).
 * Synchronous. Errors: CGP_ERR_ARG (NULL, or every entry held), CGP_ERR_CUDA. */
int cgp_ws_set_mask(cgp_ws w, const unsigned char* held_host);
/* Inference: p_dev [B][n] float64 = ||b|| NN(b / ||b||) for b_dev [B][n] float64, B <= batch_max.
 * Stream-ordered. Errors: CGP_ERR_ARG (NULL, B outside 1..batch_max), CGP_ERR_CUDA; a device wait
 * of the tensor-core pipeline that ran out through cgp_ws_status. */
int cgp_ws_forward(cgp_ws w, const double* b_dev, int B, double* p_dev, void* stream);
/* One training step on B pairs (b_dev, p_dev) [B][n] float64: loss L = 1/(B n_free) sum over
 * unmasked entries of (NN(b/s) - p/s)^2, gradients by back-propagation, then Adam with step size
 * lr (lr = 0: gradients only). loss_dev (device float, may be NULL) receives L. Stream-ordered.
 * Errors: CGP_ERR_ARG (NULL, B outside 1..batch_max, lr negative or NaN), CGP_ERR_CUDA; a device
 * wait that ran out through cgp_ws_status. */
int cgp_ws_train_step(cgp_ws w, const double* b_dev, const double* p_dev, int B, float lr, float* loss_dev,
                      void* stream);
/* Synchronise and return the network's device error word (CGP_ERR_TIMEOUT if a bounded
 * tensor-core pipeline wait gave up), else CGP_OK. */
int cgp_ws_status(cgp_ws w, void* stream);
/* Free the network and its device buffers. NULL is accepted. Returns CGP_OK. */
int cgp_ws_destroy(cgp_ws w);

/* Residual form of the learned warm start: the network corrects a base guess x_base (for example
 * the previous step's pressure or its extrapolation) instead of predicting p itself. Inference:
 * r = b - K_c x_base (the coarse matrix of Eq. 21 after elimination, from ctx), then
 * p = x_base + ||r|| NN(r / ||r||). Training on pairs (b, p): the same r as input and the
 * correction p - x_base as target (loss as in cgp_ws_train_step). b_dev, base_dev, p_dev: [B][n]
 * float64 with n = the context's n_coarse (else CGP_ERR_ARG). The first call allocates two
 * [batch_max][n] buffers. Stream-ordered. Errors: CGP_ERR_ARG (NULL, B outside 1..batch_max,
 * n mismatch), CGP_ERR_STATE (context before cgp_set_bc), CGP_ERR_NOMEM, CGP_ERR_CUDA. */
int cgp_ws_forward_residual(cgp_ws w, cgp_ctx ctx, const double* b_dev, const double* base_dev, int B, double* p_dev,
                            void* stream);
/* Training step of the residual form above, on pairs (b_dev, p_dev) with base guesses base_dev.
 * Stream-ordered. Errors: as cgp_ws_forward_residual, plus CGP_ERR_ARG for a negative or NaN lr. */
int cgp_ws_train_step_residual(cgp_ws w, cgp_ctx ctx, const double* b_dev, const double* p_dev, const double* base_dev,
                               int B, float lr, float* loss_dev, void* stream);

/* out = the extrapolation in time of order 0..3 through the values v0 (newest) .. v3 of n doubles:
 * v0, 2 v0 - v1, 3 v0 - 3 v1 + v2, 4 v0 - 6 v1 + 4 v2 - v3 (the initial-guess predictors of
 * warm_start, without a history); unused inputs may be NULL. Stream-ordered. Errors: CGP_ERR_ARG
 * (n <= 0, order outside 0..3, a needed input NULL), CGP_ERR_CUDA. */
int cgp_extrapolate(long long n, int order, const double* v0_dev, const double* v1_dev, const double* v2_dev,
                    const double* v3_dev, double* out_dev, void* stream);

/* Project-written autotuner (not in the paper). Times the SpMV lane counts {1, 2, 4, 8, 16, 32} on the
 * fine and coarse matrices and keeps the fastest for the solver kernels; the stand-alone SpMV's
 * layout (CSR or sliced ELL, spmv_format 0); and, for the fine-mesh solvers (solver_format 0 and/or
 * block_threads 0), the product layout (CSR or sliced ELL) and the threads per block of their
 * persistent kernels (the default or 256, i.e. rows per thread), by timing the consistent-mass CG
 * on a fixed right-hand side and, after cgp_set_bc, the momentum BiCGStab on the matrix of a fluid
 * at rest (the default is left only for a 5 % gain). Overwrites the statistics, the momentum
 * matrix and right-hand side (after cgp_set_bc they count as not assembled: rebuilt by the next
 * assembly) and the context's intermediate-
 * velocity, staging and gradient buffers (not the solution histories). Synchronous. Errors:
 * CGP_ERR_ARG (NULL), CGP_ERR_CUDA. */
int cgp_autotune(cgp_ctx ctx, void* stream);

/* Allocation-free conjugate-gradient solve of one symmetric positive definite CSR system
 * A x = b (no counterpart in the paper: it exists for callers that must not allocate device
 * memory, such as code embedded in a host program whose allocator owns every device byte, or code
 * running where a cudaMalloc would synchronise or fail). It runs the same persistent
 * Jacobi-preconditioned CG kernel inside FP64 refinement that cgp_poisson_solve uses for its
 * generic coarse solver (CSR products with 4 lanes per row, at most 30 FP64 refinement passes),
 * but takes its scratch from a fixed static device array of about 3.6 MB instead of a context.
 * Arguments: n rows (1 <= n <= 65536; larger n returns CGP_ERR_ARG), rp_dev [n+1], ci_dev [nnz]
 * (0-based columns), val_dev [nnz] float64, all device memory; b_dev [n]; x_dev [n] initial
 * guess in, solution out; stop at ||b - A x|| <= rtol ||b||; max_iter caps CG iterations.
 * status_dev, iters_dev, rel_res_dev: optional device outputs (NULL to skip) receiving the
 * CGP_* status, the iteration count and the final true relative residual. Device-side statuses:
 * CGP_ERR_ARG when a row has no positive finite stored diagonal (that row's preconditioner entry
 * is taken as 0); CGP_ERR_NOT_CONVERGED when max_iter or the 30 refinement passes run out (x and
 * the residual are still written, so a caller seeing fewer than max_iter iterations knows the
 * pass cap ended the solve); CGP_ERR_NAN on a non-finite residual or inner product;
 * CGP_ERR_TIMEOUT when a grid barrier gave up (then rel_res reads NaN, iters holds what the
 * solver had recorded, and x is unspecified).
 * The call is stream-ordered and asynchronous and allocates nothing (no cudaMalloc, no
 * cudaFree). The first call on each device looks up the scratch array's device address with that
 * device current; make that first call before any stream capture. All calls share the one
 * scratch array, so calls whose kernels overlap on the GPU race with each other: serialise them
 * (one stream, or events). Host-side errors (returned): CGP_ERR_ARG, CGP_ERR_CUDA. */
int cgp_cg_solve_noalloc(int n, const int* rp_dev, const int* ci_dev, const double* val_dev, const double* b_dev,
                         double* x_dev, double rtol, int max_iter, int* status_dev, int* iters_dev,
                         double* rel_res_dev, void* stream);

/* ---- diagnostics of the benchmark flows (Sect. 3.2 reattachment length, Sect. 3.3 drag and lift) ----
 * Standard definitions (the paper prints none for the forces): the force on a body is the sum over
 * its boundary edges of int sigma n_b, sigma = -p I + mu (grad u + grad u^T), n_b the unit normal
 * from the body into the fluid, p = P p_c on the fine mesh (Eq. 29, trapezoid rule along the edge),
 * grad u the P1 gradient of the fluid triangle owning the edge; C_D = 2 F_x / (rho u_inf^2 d),
 * C_L = 2 F_y / (rho u_inf^2 d). Wall shear tau = mu t . (grad u) n_f per wall edge (t the unit
 * tangent towards larger x, n_f the unit normal into the fluid). */

/* Surface of a diagnostic: which = 0 the body of cgp_body_force, 1 the wall of cgp_reattachment;
 * node_mask_host [n_fine]: nonzero on the surface's fine nodes; the surface is every boundary edge
 * of the fine mesh whose two end nodes are marked (wall edges are kept sorted by midpoint x).
 * *n_edges (optional) receives the edge count. Synchronous. Errors: CGP_ERR_ARG, CGP_ERR_NOMEM,
 * CGP_ERR_CUDA. */
int cgp_set_surface(cgp_ctx ctx, int which, const unsigned char* node_mask_host, int* n_edges);

/* Force on the body for velocity u_dev [n_fine][2] and coarse pressure pc_dev [n_coarse]:
 * force_dev [4] = pressure force (x, y), viscous force (x, y). One block, fixed-order sums
 * (deterministic). Stream-ordered. Errors: CGP_ERR_ARG, CGP_ERR_STATE (no body set). */
int cgp_body_force(cgp_ctx ctx, const double* u_dev, const double* pc_dev, double* force_dev, void* stream);

/* Reattachment point on the wall: the first x >= x_start at which the wall shear turns from
 * negative to non-negative, linear between edge midpoints; *xr_dev = NaN if there is none.
 * x_dev, tau_dev [n_edges] (optional): each wall edge's midpoint x and shear. Stream-ordered.
 * Errors: CGP_ERR_ARG, CGP_ERR_STATE (no wall set). */
int cgp_reattachment(cgp_ctx ctx, const double* u_dev, double x_start, double* xr_dev, double* x_dev, double* tau_dev,
                     void* stream);

/* Check of the bounded device waits (not in the paper; for tests of failure detection): launches,
 * on the context's persistent launch shape (grid_blocks blocks, cooperative), one grid barrier
 * whose target is grid_blocks + missing_blocks arrivals, with a wait bound of limit_ms
 * (0 < limit_ms <= 10000) instead of the library's 250 ms. With missing_blocks = 0 every block
 * passes and *status_dev receives CGP_OK; with missing_blocks > 0 (at most 1024) the barrier can
 * never complete, every block gives up after limit_ms and *status_dev receives CGP_ERR_TIMEOUT.
 * The context's own statistics are not touched and it stays usable. status_dev: one int of
 * device memory. Stream-ordered. Errors: CGP_ERR_ARG, CGP_ERR_CUDA. */
int cgp_wait_probe(cgp_ctx ctx, int missing_blocks, double limit_ms, int* status_dev, void* stream);

/* Free everything the context owns; synchronises the device first. NULL is accepted. Returns
 * CGP_OK. */
int cgp_mesh_destroy(cgp_ctx ctx);

/* Name of a status code (static string, never NULL; unknown codes get a generic name). */
const char* cgp_status_str(int status);

#ifdef __cplusplus
}
#endif
#endif /* CGP_H */
