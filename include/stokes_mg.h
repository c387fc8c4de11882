/*
 * stokes_mg.h -- C-ABI of the GB300 coupled multigrid solver for the generalized Stokes system
 *
 *     -Lap u + beta u + grad p = f,   div u = g   in (0,1)^2,   u = 0 on the boundary,  int p = 0
 *
 * (Takacs, "A robust multigrid method for the time-dependent Stokes problem", SINUM 53(6), 2015:
 * problem statement Sec. 1, eq. stokes; variational form Sec. 2, eq. gen:bil; matrix form
 * eq. gen:bil:mv).  Discretisation: Taylor-Hood P2 velocity / P1 pressure on the unit square split
 * into 8 triangles around its centre (level 0) and refined uniformly k times (Sec. 6), so level k
 * has N = 2^(k+1) element legs per side.
 *
 * DATA LAYOUT (all arrays are caller-owned DEVICE memory of the current CUDA device, float64,
 * dense, row-major with y outer and x inner):
 *   u : 2 x (2N+1) x (2N+1)   velocity nodal values on the P2 lattice (spacing 1/(2N)),
 *                             component x first.  Boundary lattice points hold 0 on output and
 *                             are ignored (treated as 0) on input.
 *   p : (N+1) x (N+1)         pressure nodal values at the vertices (spacing 1/N).  The paper's
 *                             weak form carries +(p, div v) (Sec. 2), so p approximates -p of the
 *                             strong form written in Sec. 1.  Returned with zero mean int p = 0.
 *   f : 2 x (2N+1) x (2N+1)   the velocity right-hand side as a LOAD VECTOR (f, phi_i) (the
 *                             underlined f_k of eq. gen:bil:mv); boundary entries ignored.
 *   g : (N+1) x (N+1)         the pressure load vector (g, psi_i); its entries must sum to 0
 *                             (solvability, Sec. 1); stokes_load_vectors() produces such g.
 * Use stokes_load_vectors() to turn nodal values of f, g into load vectors.
 *
 * STREAMS: every call is asynchronous on the stream given to stokes_setup() unless it returns a
 * host-side result (stokes_solve, stokes_residual_norm), which synchronises that stream.
 *
 * ERRORS: every call returns a stokes_status; no call aborts or exits the process.  After
 * STOKES_ERR_CUDA the handle should be destroyed.
 *
 * ENVIRONMENT: STOKES_MG_PDL=0 (read once per process) launches the cycle's kernels without
 * programmatic dependent launch; by default a kernel's CTAs may be scheduled while the tail of
 * its predecessor runs.  Results do not depend on it.  STOKES_MG_FUSE_PROLONG=0 (read once per
 * process) prolongates on the planar float32 levels with a separate kernel; by default the
 * coarse-grid correction is added to the staged tiles of the first post-smoothing step (results
 * differ in float32 rounding only).
 */
#ifndef STOKES_MG_H
#define STOKES_MG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum stokes_status {
    STOKES_OK = 0,
    STOKES_ERR_BAD_ARG = 1,      /* null pointer, levels out of range, beta < 0 or NaN, ... */
    STOKES_ERR_OOM = 2,          /* device allocation failed */
    STOKES_ERR_CUDA = 3,         /* a CUDA runtime call failed */
    STOKES_NOT_CONVERGED = 4,    /* solve reached max_cycles above tol (result still returned) */
    STOKES_DIVERGED = 5,         /* residual became NaN/Inf or grew in 8 consecutive cycles */
    STOKES_ERR_TIMEOUT = 6       /* a bounded device-side wait gave up (about a second): the tile
                                    copies of the planar levels' kernels, or a grid barrier of the
                                    cooperative small-level cycle; reported by the next solve, cycle,
                                    float32 smoothing or batch call after it; results are not valid */
} stokes_status;

typedef enum stokes_smoother {
    STOKES_UZAWA = 0,            /* Uzawa-type smoother, Sec. 4 (default, tau = sigma = 0.8) */
    STOKES_NORMAL_EQ = 1         /* preconditioned normal-equation smoother, Sec. 4 (tau = 0.35) */
} stokes_smoother;

typedef enum stokes_domain {
    STOKES_UNIT_SQUARE = 0,      /* the unit square of Sec. 6 */
    STOKES_L_SHAPE = 1           /* the unit square without [1/2, 1]^2 (a non-convex domain, Sec. 1) */
} stokes_domain;

typedef enum stokes_precision {
    STOKES_FP64 = 0,             /* every level and every step in float64 */
    STOKES_MIXED = 1             /* float32 cycles inside float64 iterative refinement */
} stokes_precision;

typedef struct stokes_params {
    int levels;        /* number of grid levels; the finest is k = levels-1; 1 <= levels <= 13 */
    double beta;       /* >= 0 (Sec. 1 assumes beta > 0; beta = 0 is the stationary Stokes case) */
    int nu_pre;        /* pre-smoothing steps  (Sec. 6 uses 3) */
    int nu_post;       /* post-smoothing steps (Sec. 6 uses 3) */
    double tau;        /* smoother damping tau   (Sec. 6: 0.8 Uzawa, 0.35 normal equation) */
    double sigma;      /* Uzawa pressure damping (Sec. 6: 0.8) */
    int smoother;      /* stokes_smoother */
    int gamma;         /* 1 = V-cycle, 2 = W-cycle (Sec. 3) */
    int precision;     /* stokes_precision */
    int inner_cycles;  /* STOKES_MIXED: float32 cycles per refinement step (>= 1) */
    int coarse_level;  /* coarsest level of the iteration, 0 <= coarse_level <= min(levels - 1, 3): the
                          coarse problem is solved exactly there (Sec. 3) -- on level 0 by a 27 x 27
                          inverse, on level c > 0 by a dense float64 inverse of its bordered system
                          (2212 unknowns at c = 3) computed on the device at setup and set_beta; a
                          finer coarse level shortens the W-cycle's recursion */
    int domain;        /* stokes_domain.  STOKES_L_SHAPE keeps the square's lattice and layouts: the
                          L's level j is the square's level j + 1 with the velocity nodes in the closed
                          removed quadrant (the re-entrant sides x = 1/2, y >= 1/2 and y = 1/2,
                          x >= 1/2 and beyond) Dirichlet nodes and the vertices strictly inside it not
                          unknowns; entries of u, p, f, g there are ignored on input and zero on output,
                          and the zero-mean pressure is over the L.  It needs the Uzawa smoother,
                          coarse_level = 1 (the L's level 0) and levels >= 2; with STOKES_MIXED its
                          float32 levels keep the compact layout and the per-phase step; load vectors,
                          Euler right-hand sides and mass products are square-only (they return
                          STOKES_ERR_BAD_ARG on an L handle) */
    int tma_level;     /* STOKES_MIXED with the Uzawa smoother on the unit square: the float32 levels
                          k >= tma_level are held in a padded layout whose rows start on 16-byte
                          boundaries and smoothed by a one-kernel step whose tiles arrive by
                          tensor-memory-access box copies (the other levels as set by
                          stokes_set_step_variant).  0 selects the default (level 6, N = 128); otherwise
                          tma_level >= 5, and a value above the finest level keeps every level on the
                          other variants.  Internal layout only: every array a caller passes keeps the
                          layout above.  The step needs the register tile's coefficient structure
                          (stokes_step_tables_match): setup and set_beta return STOKES_ERR_BAD_ARG for
                          a beta without it on such a level */
    int coop_level;    /* STOKES_MIXED with the Uzawa smoother on the unit square: a visit of a float32
                          level l <= coop_level (and above the coarsest level, below tma_level) runs the
                          whole V- or W-cycle from l down, the coarsest solve included, as ONE
                          cooperative launch whose phases meet at grid barriers, instead of one launch
                          per phase.  0 or -1: off (the default; on a GB300 a phase of that launch
                          costs about as much as a launch of its own); at most 6 */
} stokes_params;

/* Paper defaults: Uzawa, nu = 3+3, tau = sigma = 0.8, V-cycle, float64, one inner cycle, coarsest
 * level 0. */
void stokes_default_params(stokes_params* prm, int levels, double beta);

typedef struct stokes_handle_t stokes_handle;

typedef struct stokes_report {
    int cycles;              /* cycles (FP64) or refinement steps (MIXED) performed */
    double rel_residual;     /* final ||F - A x||_2 / ||F||_2 over the unknowns (float64) */
    double mean_rate;        /* geometric mean of the per-cycle residual reduction (Sec. 6 q) */
    double initial_residual; /* ||F - A x0||_2 */
    double rhs_norm;         /* ||F||_2 */
} stokes_report;

/* Device memory for the internal buffers of handles and batches.  alloc returns a pointer to at
 * least `bytes` bytes of device memory of the current device, 256-byte aligned and usable on
 * `stream` (the handle's cudaStream_t), or NULL on failure (the setup then returns STOKES_ERR_OOM);
 * release frees a block that alloc returned, with the same bytes and stream.  ctx is passed through.
 * The callbacks are called only inside stokes_setup, stokes_batch_setup, stokes_euler_rhs (its first
 * call) and the destroy calls, on the calling thread. */
typedef void* (*stokes_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*stokes_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);

/* Registers the allocator that every later stokes_setup and stokes_batch_setup uses for its device
 * buffers (process-wide; both NULL restores cudaMalloc / cudaFree, one of them NULL is
 * STOKES_ERR_BAD_ARG).  A handle keeps the allocator it was set up with and releases its buffers
 * through it in stokes_destroy, so the allocator must outlive the handles set up with it.  This lets
 * a framework's caching allocator (PyTorch's, for one) own the solver's level buffers.  Pinned host
 * mirrors of a few scalars are always cudaMallocHost. */
stokes_status stokes_set_allocator(stokes_alloc_fn alloc, stokes_free_fn release, void* ctx);

/* Builds the level hierarchy (Sec. 2 nesting), the per-level diagonals Ahat = diag A_k and
 * Shat = diag(B_k Ahat^{-1} B_k^T) (Sec. 6, eq. numintroduc) and the coarsest level's factorisation
 * (Sec. 3: exact coarsest solve).  `stream` is a cudaStream_t (NULL = a stream the library creates).
 * The library owns the handle and all internal buffers (from the registered allocator, else
 * cudaMalloc); free with stokes_destroy. */
stokes_status stokes_setup(const stokes_params* prm, void* stream, stokes_handle** out);

/* Changes beta: rebuilds the diagonals and the coarse factorisation only (synchronises the stream). */
stokes_status stokes_set_beta(stokes_handle* h, double beta);

void stokes_destroy(stokes_handle* h);

const char* stokes_status_str(stokes_status s);

/* N and array lengths of the finest level: n_vel = 2 (2N+1)^2, n_p = (N+1)^2, ndof = number of
 * unknowns 2 (2N-1)^2 + (N+1)^2. */
stokes_status stokes_sizes(const stokes_handle* h, int* N, size_t* n_vel, size_t* n_p, size_t* ndof);

/* One multigrid iteration on the finest level (Sec. 3; V or W by params.gamma), in place on
 * (u, p), followed by the zero-mean projection of p.  Under STOKES_MIXED it is one refinement
 * step: float64 residual, params.inner_cycles float32 cycles on the correction, float64 update. */
stokes_status stokes_cycle(stokes_handle* h, double* u, double* p, const double* f, const double* g);

/* Iterates stokes_cycle from the given (u, p) until ||F - A x||_2 <= tol ||F||_2 or max_cycles.
 * Returns STOKES_OK, STOKES_NOT_CONVERGED or STOKES_DIVERGED; `rep` (caller-owned, may be NULL)
 * receives the statistics; `history` (caller-owned host array of max_cycles+1 doubles, may be
 * NULL) receives the residual norm before the first and after every cycle. */
stokes_status stokes_solve(stokes_handle* h, double* u, double* p, const double* f, const double* g,
                           double tol, int max_cycles, stokes_report* rep, double* history);

/* r = F - A x on the finest level (eq. gen:bil:mv), float64; ru / rp have the layouts of u / p
 * (boundary entries of ru set to 0).  Asynchronous. */
stokes_status stokes_residual(stokes_handle* h, const double* u, const double* p, const double* f,
                              const double* g, double* ru, double* rp);

/* ||F - A x||_2 over the unknowns, float64; synchronises the stream. */
stokes_status stokes_residual_norm(stokes_handle* h, const double* u, const double* p, const double* f,
                                   const double* g, double* norm);

/* nu steps of the configured smoother (Sec. 4) on the finest level, in place on (u, p), with the
 * float64 arithmetic of the FP64 path.  Exposed for verification of the smoother alone. */
stokes_status stokes_smooth(stokes_handle* h, double* u, double* p, const double* f, const double* g, int nu);

/* nu steps of the float32 smoother used inside STOKES_MIXED refinement, with the step variant
 * currently set for the finest level (stokes_step_variant: a one-kernel tile, the three-kernel step
 * or a pair tile), on float32 arrays of the finest-level layouts; requires a STOKES_MIXED handle.
 * Exposed for verification of the float32 path alone. */
stokes_status stokes_smooth_f32(stokes_handle* h, float* u, float* p, const float* f, const float* g, int nu);
/* Verification of the float32 transfer path (Sec. 3): (fc, gc) = I^T (F - A x) from the finest level of
 * a STOKES_MIXED handle to the level below, float32, on the caller's arrays in the layout above
 * (u, f: 2 (2N+1)^2, p, g: (N+1)^2 of the finest level; fc: 2 (N+1)^2, gc: (N/2+1)^2).  On a planar
 * finest level (stokes_params.tma_level) this is the kernel the cycles run, defect and restriction in
 * one pass over tiles staged by tensor-memory-access copies; the caller's arrays are copied into the
 * handle's finest and coarse float32 buffers (their contents are overwritten).  Asynchronous on the
 * handle's stream.  STOKES_ERR_BAD_ARG for a float64 handle or levels < 2. */
stokes_status stokes_residual_restrict_f32(stokes_handle* h, const float* u, const float* p, const float* f,
                                           const float* g, float* fc, float* gc);

/* Canonical transfers (Sec. 3) between finest level k and level k-1 (requires levels >= 2):
 * restriction  (fc, gc) = I_k^{k-1} (fu, fp)   with coarse layouts of level k-1,
 * prolongation (uf, pf) += I_{k-1}^k (uc, pc). */
stokes_status stokes_restrict(stokes_handle* h, const double* fu, const double* fp, double* fc, double* gc);
stokes_status stokes_prolong_add(stokes_handle* h, const double* uc, const double* pc, double* uf, double* pf);

/* Load vectors of nodal data: f = (f_h, phi_i) on interior P2 nodes (the P2 interpolant f_h of the
 * nodal values on the FULL lattice, boundary values included) and g = (g_h, psi_i) on all
 * vertices.  With project_g != 0 the P1 function g_h is first shifted to zero mean
 * (g_h <- g_h - int g_h), the solvability condition of Sec. 1. */
stokes_status stokes_load_vectors(stokes_handle* h, const double* f_nodal, const double* g_nodal,
                                  int project_g, double* f, double* g);

/* Host-only views of the operator tables the kernels use (no device work; callable without a GPU).
 * stokes_stencil_class: the stencil class (0..6) of cell (i, j), 0 <= i, j <= N = 2^levels, by the
 * orientations of its four squares (Sec. 6 mesh: 0 / 1 off the mid-lines, 2..6 on them).
 * stokes_stencil_rows: for class cls of a level with N = 2^levels and the given beta, the rows of the
 * matrix of eq. gen:bil:mv at the cell's four velocity nodes s = V (2i, 2j), H (2i+1, 2j),
 * E (2i, 2j+1), C (2i+1, 2j+1), as written by the library:
 *   ma[s*25 + (dy+2)*5 + dx+2]  = (K + beta M)(node s, lattice node (2i+dx, 2j+dy))   (caller array of 100)
 *   mbtx[s*9 + (dj+1)*3 + di+1] = Bx(vertex (i+di, j+dj), node s), mbty likewise        (36 each)
 *   mbx[(dy+2)*5 + dx+2]        = Bx(vertex (i, j), lattice node (2i+dx, 2j+dy)), mby likewise (25 each)
 *   midg[s]                     = 1 / (K + beta M)(node s, node s)                       (4)
 * with B_ij = (div phi_j, psi_i) split by component.  STOKES_ERR_BAD_ARG on out-of-range input. */
stokes_status stokes_stencil_class(int levels, int i, int j, int* cls);
stokes_status stokes_stencil_rows(int levels, double beta, int cls, double* ma, double* mbtx, double* mbty,
                                  double* mbx, double* mby, double* midg);

/* Host-only (no device work): the canonical P2 embedding weights of Sec. 3 that the transfer kernels
 * use, w[((o*9 + L)*5 + fb)*5 + fa] = value of the local basis function L = 3*b + a (local lattice
 * node (a, b) in {0,1,2}^2) of a coarse square of orientation o at its fine lattice point (fa, fb) in
 * {0..4}^2 (caller array of 450); and the inverse of the level-0 system (N = 2) of eq. gen:bil:mv
 * bordered with the zero-mean pressure condition, first 27 x 27 block, row-major, unknowns u_x at the
 * interior lattice points (X, Y) in [1, 3]^2 (Y outer), then u_y, then p at the 3 x 3 vertices
 * (caller array of 729).  STOKES_ERR_BAD_ARG on bad input or a singular system. */
stokes_status stokes_transfer_weights(double* w);
/* Host-only: the embedding weights compiled into the planar float32 smoothing kernel, which adds
 * the coarse-grid correction P x_c (Sec. 3) to the tiles of a planar level's first post-smoothing
 * step: w[((o * 9 + L) * 4 + fb) * 4 + fa] for orientation o, coarse local node L and the fine
 * lattice points (fa, fb) in {0..3}^2 that a coarse square owns (caller array of 288).
 * STOKES_ERR_BAD_ARG if w is NULL. */
stokes_status stokes_embed_weights(double* w);
stokes_status stokes_coarse_inverse(double beta, double* inv);

/* Host-only (no device work): tables for the L-shaped domain, the unit square without [1/2, 1]^2
 * (Sec. 1: the method applies to non-convex domains).  For a pressure vertex on a re-entrant side
 * of a level with N = 2^levels (levels >= 2): kind 0 = vertex (N/2, j), N/2 < j < N (side x = 1/2);
 * kind 1 = vertex (i, N/2), N/2 < i < N (side y = 1/2); kind 2 = the corner (N/2, N/2); kinds 3, 4 =
 * the ends (N/2, N) and (N, N/2) of the two sides on the outer boundary.  Writes the
 * vertex's B row over its 5 x 5 lattice window, mbx[(dy+2)*5 + dx+2] = Bx(vertex, lattice node
 * (2i+dx, 2j+dy)) and mby likewise (25 each), summed over the squares around the vertex that lie in
 * the L, and its pressure-mass weight w = (1, psi_vertex) over the L.  STOKES_ERR_BAD_ARG on bad
 * input. */
stokes_status stokes_lshape_vertex_rows(int levels, int kind, double* mbx, double* mby, double* w);
/* Host-only: S_hat = diag(B Ahat^-1 B^T) (eq. numintroduc) on the L at the re-entrant vertices of a
 * level with N = 2^levels, the sum over the velocity unknowns (nodes strictly inside the L) of the
 * vertex's masked B row squared over diag A: s0[t] at (N/2, N/2 + 1 + t) and s1[t] at
 * (N/2 + 1 + t, N/2), t = 0 .. N/2 - 1 (the last entries are the ends on the outer boundary; caller
 * arrays of N/2), s2[0] at the corner. */
stokes_status stokes_lshape_schur(int levels, double beta, double* s0, double* s1, double* s2);
/* Host-only: the inverse of level 0 of the L-shaped hierarchy (the square's N = 4 level without the
 * upper-right quadrant) for eq. gen:bil:mv bordered with the zero-mean pressure condition, first
 * block, row-major, unknowns u_x at the interior nodes of the L in lattice order (Y outer), then
 * u_y, then p at the vertices of the L in lattice order; *nunk receives the size (87; caller array
 * of 87 * 87).  STOKES_ERR_BAD_ARG on bad input or a singular system. */
stokes_status stokes_lshape_coarse_inverse(double beta, double* inv, int* nunk);

/* Right-hand side of one implicit Euler step of the time-dependent Stokes problem
 *     u_t - Laplace u + grad p = f,  div u = g,  u = 0 on the boundary      (unit viscosity),
 * whose step with length dt is the generalized Stokes system of Sec. 1 with beta = 1/dt (the
 * handle's current beta; another viscosity is a rescaling the caller applies to beta, f and p):
 *     f = (f_h + beta u_prev, phi_i) on interior P2 nodes,  g = (g_h, psi_i) with g_h shifted to
 * zero mean, where f_nodal, g_nodal are the nodal data of the new time level (layouts and
 * interpolants as in stokes_load_vectors) and u_prev the velocity of the previous level (layout of
 * u, zero on the boundary).  The first call allocates one velocity-sized scratch array owned by
 * the handle.  f and g must not alias f_nodal or g_nodal.  Asynchronous on the handle's stream. */
stokes_status stokes_euler_rhs(stokes_handle* h, const double* u_prev, const double* f_nodal, const double* g_nodal,
                               double* f, double* g);

/* A sequence of `steps` implicit Euler steps (as in stokes_euler_rhs, beta = 1/dt the handle's beta)
 * in ONE CUDA-graph launch.  For n = 0 .. steps-1: the right-hand side of the step from the nodal data
 * f_nodal[n], g_nodal[n] of the new time level and the current velocity, then multigrid cycles from the
 * current (u, p) (a warm start) in a device-side loop until the TRUE float64 relative residual
 * ||F - A x|| / ||F|| <= tol or max_cycles cycles.  u, p (device, layouts above) hold the initial state
 * and receive the state after the last step; f_nodal, g_nodal are host arrays of `steps` device
 * pointers (repeat a pointer for constant forcing).  cycles, rel_residual (caller-owned host arrays of
 * `steps`, may be NULL) receive each step's cycle count and final relative residual.  The graph is kept
 * and replayed while the pointers, tol and max_cycles are the same.  Returns STOKES_NOT_CONVERGED if
 * some step missed tol (the trajectory is still written).  Synchronises the stream. */
stokes_status stokes_euler_run(stokes_handle* h, double* u, double* p, const double* const* f_nodal,
                               const double* const* g_nodal, int steps, double tol, int max_cycles, int* cycles,
                               double* rel_residual);

/* g <- g - (1^T g) w,  w = M_P 1 (w sums to 1): makes a pressure right-hand side orthogonal to the
 * constant pressure, the kernel of the matrix of eq. gen:bil:mv (Sec. 1: int g = 0).  Needed for
 * adjoint right-hand sides whose pressure part does not sum to zero.  In place, asynchronous. */
stokes_status stokes_make_consistent(stokes_handle* h, double* g);

/* dot = a^T M_U b for two velocity arrays a, b (layout of u, boundary entries ignored), where M_U
 * is the velocity mass matrix (the beta-part of A_k = K + beta M_U, Sec. 2); float64, synchronises
 * the stream.  Gives the beta-derivative of a loss through the adjoint: dL/dbeta = -lambda_u^T M_U u. */
stokes_status stokes_mass_dot(stokes_handle* h, const double* a, const double* b, double* dot);

/* ||F - A x||_2^2 of the finest level, like stokes_residual_norm, but without a handle and without
 * allocating any device memory.  The paper has no counterpart: this exists for callers that cannot
 * call cudaMalloc -- code that lives inside a fixed memory budget handed out by another framework
 * (which owns the rest of the device), code on a device that is already full, or code that has no
 * way to release memory later.
 *   levels, beta : as in stokes_params; levels <= 11 (N <= 2048), larger sizes return
 *                  STOKES_ERR_BAD_ARG before any GPU work
 *   u, p, f, g   : caller-owned device arrays with the layouts described at the top of this file
 *   norm2        : caller-owned device double that receives the squared norm (not synchronised)
 *   stream       : cudaStream_t to run on (NULL = legacy default stream)
 * The per-block partial sums live in one fixed array inside the library (about 131 KB of device
 * memory on every GPU that loads the library, kept until the process exits).  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress); the first call in a process
 * may also build the host-side element tables.  Make that first call before any stream capture.
 * Every call overwrites the whole
 * part of the array it reads, so nothing needs clearing, but all calls share the one array: calls
 * whose GPU work overlaps (different streams or threads without ordering) race and give wrong
 * results. */
stokes_status stokes_residual_norm2_noalloc(int levels, double beta, const double* u, const double* p,
                                            const double* f, const double* g, double* norm2, void* stream);

/* Chooses, for every level of a STOKES_MIXED handle whose size has not been tuned in this process,
 * the fastest float32 Uzawa step variant (one-kernel tiles of several kinds and shapes, or the
 * three-kernel step with several block shapes; on planar levels the planar step variants) by timing
 * each on the handle's buffers; the choice is kept process-wide per level size.  Untuned levels use the three-kernel step below N = 128 and
 * the 32 x 16 fused tile above.  Synchronises the stream. */
stokes_status stokes_autotune(stokes_handle* h);
/* The step variant currently used for a float32 level with `levels` levels (N = 2^levels), -1 if
 * out of range: 0-3 fused tiles 32x16, 32x8, 64x8, 16x16; 4-6 three-kernel step, blocks 32x8, 16x8, 8x8;
 * 7-9 fused step on component-pair tiles (packed FP32x2 arithmetic), 28 cells wide: 8 or 4 warps with the
 * tile height chosen per level, or 12 warps on 8 rows; 10-11 fused step with the operator's coefficients
 * in registers and asynchronous staging, 28 cells wide, 8 warps, tile height chosen per level for at least
 * 2 or at least 4 resident CTAs per SM. */
int stokes_step_variant(int levels);
/* Host-only (no device work): STOKES_OK if the merged stencils of the two orientation classes on a
 * level with N = 2^levels and this beta have exactly the compile-time structure that step variants
 * 10-11 assume (which coefficients vanish, which are equal, B and B^T entries +-b and +-b/2 for one
 * b); STOKES_ERR_BAD_ARG otherwise (those variants then run the pair tile of variant 7 instead). */
stokes_status stokes_step_tables_match(int levels, double beta);
/* Sets the step variant (0-11, as above) for float32 levels with `levels` levels (N = 2^levels),
 * process-wide, and marks that size as tuned (stokes_autotune keeps it).  Takes effect for direct
 * smoothing calls (stokes_smooth_f32) and for cycle graphs captured afterwards; graphs a handle has
 * already captured keep their variant.  Not thread-safe against concurrent setup or capture.
 * Returns STOKES_ERR_BAD_ARG for levels outside 2..31 or an unknown variant. */
stokes_status stokes_set_step_variant(int levels, int variant);
/* The same for the planar float32 levels (stokes_params.tma_level), whose step stages its tiles by
 * tensor-memory-access box copies, one tile per CTA of 8 warps: 0 tile height for 3 resident CTAs per
 * SM, 2 for 4 (fewer registers, shorter tiles); 1 and 3 the same, each CTA also prefetching into L2
 * the tiles of a tile one wave of resident CTAs ahead; 4 and 5 two cell rows per warp pass (window
 * rows shared by the two loaded once), 2 or 3 CTAs per SM, with the prefetch.
 * stokes_autotune times them on the handle's planar levels; untuned sizes use 0.  Same scope and
 * rules as stokes_set_step_variant; -1 / STOKES_ERR_BAD_ARG out of range. */
int stokes_planar_step_variant(int levels);
stokes_status stokes_set_planar_step_variant(int levels, int variant);

/* ---- batches: many independent solves (right-hand sides, beta values, mesh levels) in one launch.
 * stokes_batch_setup builds `count` solvers; instance i has levels[i] levels and beta betas[i], the
 * other parameters from `base` (STOKES_MIXED is the intended precision).  With autotune != 0 the
 * tile shape of the float32 Uzawa kernel is chosen per level size by timing the candidates on the
 * instances' own buffers (the choice is kept process-wide).  The library owns all buffers. */
typedef struct stokes_batch_t stokes_batch;
stokes_status stokes_batch_setup(int count, const int* levels, const double* betas, const stokes_params* base,
                                 void* stream, int autotune, stokes_batch** out);

/* Solves every instance from its (u[i], p[i]) to ||F - A x|| <= tol ||F|| (at most max_cycles steps)
 * in ONE launch of a CUDA graph: per instance a prologue, a conditional WHILE node whose body is one
 * cycle (MIXED: one refinement step) followed by a device-side convergence test, and an epilogue that
 * checks the true float64 residual and writes (u[i], p[i]).  Instances run concurrently.  u, p, f, g
 * are host arrays of `count` device pointers with the per-instance layouts above.  The graph is
 * rebuilt only when the pointers, tol or max_cycles change.  An instance whose true residual misses
 * tol after the graph (not expected) continues through stokes_solve.  cycles / rel_residual
 * (caller-owned host arrays of `count`, may be NULL) receive the steps taken and the final relative
 * residuals.  Synchronises the batch's stream. */
stokes_status stokes_batch_solve(stokes_batch* b, double* const* u, double* const* p, const double* const* f,
                                 const double* const* g, double tol, int max_cycles, int* cycles,
                                 double* rel_residual);
void stokes_batch_destroy(stokes_batch* b);
/* Independent implicit Euler trajectories, one per instance of the batch (instance i: its own level
 * and beta = 1/dt_i), each a chain of `steps` steps as in stokes_euler_run, all instances concurrent in
 * one CUDA-graph launch.  u, p: host arrays of `count` device pointers (state in, state out);
 * f_nodal, g_nodal: host arrays of count * steps device pointers, instance-major (entry i * steps + n
 * is step n of instance i); cycles, rel_residual (may be NULL): host arrays of count * steps, likewise.
 * Returns STOKES_NOT_CONVERGED if some step of some instance missed tol.  Synchronises the stream. */
stokes_status stokes_batch_euler_run(stokes_batch* b, double* const* u, double* const* p, const double* const* f_nodal,
                                     const double* const* g_nodal, int steps, double tol, int max_cycles, int* cycles,
                                     double* rel_residual);
/* Kernels executed by stokes_batch_solve calls so far (loop bodies counted per executed step). */
unsigned long long stokes_batch_kernel_launches(const stokes_batch* b);

/* Timing of the hot kernels inside the captured cycle: with enable != 0, the cycle graph is
 * rebuilt with CUDA event records (cudaEventRecordExternal) around every finest-level smoothing
 * step and around the float64 finest-level residual, and stokes_solve accumulates their durations
 * (milliseconds, counts) until the next stokes_set_timing call, which also resets the totals.
 * stokes_get_timing_fused: the finest-level smoothing steps that also add the coarse-grid
 * correction to their staged tiles (the first post-smoothing step of a planar level, Sec. 3),
 * which stokes_get_timing's smoothing totals leave out.  Any output pointer may be NULL. */
stokes_status stokes_set_timing(stokes_handle* h, int enable);
stokes_status stokes_get_timing(const stokes_handle* h, double* smooth_ms, long long* smooth_count,
                                double* resid_ms, long long* resid_count);
stokes_status stokes_get_timing_fused(const stokes_handle* h, double* ms, long long* count);

/* Number of CUDA kernels this handle has launched so far (kernel nodes of replayed graphs
 * included); for accounting in benchmarks. */
unsigned long long stokes_kernel_launches(const stokes_handle* h);

#ifdef __cplusplus
}
#endif
#endif
