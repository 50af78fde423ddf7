/*
 * gbmg.h -- C ABI of the GB300 multigrid solver for the variable-density
 * pressure Poisson equation
 *
 *     div( (1/rho) grad p ) = S                                       (Eq. 9)
 *
 * of Shin, Chergui & Juric, "A solver for massively parallel direct numerical
 * simulation of three-dimensional multiphase flows" (arXiv 1410.8568), Sec. 2.3,
 * discretised with cell-centred second-order differences on a uniform
 * staggered (MAC) grid (Eq. 10) with face coefficients alpha = 1/rho (harmonic
 * averages, Eqs. 11-12), solved by V-cycle multigrid with red-black relaxation.
 *
 * One process, one GPU.  All compute runs in the CUDA kernels of libgbmg.so;
 * there is no CPU fallback.  Every call returns an int status (MG_OK = 0).
 *
 * ---------------------------------------------------------------------------
 * Layout.  A grid has nx*ny*nz cells; cell (i,j,k) is element i + nx*(j + ny*k)
 * of every cell array (x fastest).  A face array ax (likewise ay, az) has one
 * entry per cell: the coefficient alpha of that cell's LOW face along x, i.e.
 * the face between cells (i-1,j,k) and (i,j,k).  On a Neumann (wall) axis the
 * entries at i = 0 are the wall and are ignored (zero flux), and the high wall
 * of the last cell carries no entry.  On a periodic axis the entry at i = 0 is
 * the face shared with cell nx-1.  All arrays are FP64 unless stated.
 *
 * Operator.  (A p)_c = sum over the faces f of c of alpha_f / h_d^2 (p_nb - p_c)
 * with h_d = l_d / n_d; A is symmetric negative semidefinite with A 1 = 0.
 * Because every boundary is a wall or periodic, A p = b is solvable only for
 * sum(b) = 0 and p is defined up to a constant: the library removes the mean of
 * the right-hand side (reported in mg_stats.rhs_mean) and returns the solution
 * with zero mean.
 *
 * Size rule.  Every axis has n >= 2 cells and the grid fewer than 2^31 cells.
 * All axes are coarsened together while every axis is even and larger than 2.
 * A coarsest grid of at most MG_MAX_COARSE cells is solved exactly (dense
 * inverse); a larger one, up to MG_MAX_COARSE_GMRES cells, by restarted GMRES
 * (Sec. 2.3 item 6).  Every n = m * 2^k with m in {1, 2, 3, 4} has an exact
 * coarsest solve (2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256,
 * 384, 512, 768, 1024, ...); sizes with a larger odd factor (e.g. 100 = 25 * 4)
 * take GMRES.
 *
 * Ownership.  The caller owns every buffer it passes.  Device pointers are
 * device memory of the current CUDA device.  A handle owns its hierarchy (all
 * levels, FP32 copies, the coarsest-grid inverse, reduction scratch) until
 * mg_destroy.  No host<->device copy happens inside the device-pointer calls
 * except the small statistics record.  The *_host calls take host pointers and
 * do their own copies on the handle's stream.
 *
 * Errors.  MG_EINVAL for bad arguments (unsupported size, null pointer,
 * non-positive or non-finite coefficients or density, bad parameters);
 * MG_ENOMEM when device memory cannot be allocated; MG_ECUDA for a CUDA error;
 * MG_ENOTCONV when max_iters cycles did not reach the tolerance (p holds the
 * last iterate); MG_EDIVERGED when the residual became NaN/Inf; MG_ESINGULAR
 * when the coarsest-grid matrix could not be inverted (a grid cut into pieces
 * by zero coefficients); MG_EBUSY, MG_EAGAIN, MG_EBUDGET, MG_ENOTFOUND for the
 * serving calls; MG_ETIMEOUT when a bounded device wait expired.
 */
#ifndef GBMG_H
#define GBMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MG_OK 0
#define MG_EINVAL 1
#define MG_ENOMEM 2
#define MG_ECUDA 3
#define MG_ENOTCONV 4
#define MG_EDIVERGED 5
#define MG_ETIMEOUT 6
#define MG_EBUSY 7
#define MG_EAGAIN 8
#define MG_EBUDGET 9
#define MG_ESINGULAR 10
#define MG_ENOTFOUND 11
#define MG_ETOOBIG 12 /* larger than the fixed scratch area of mg_coarse_solve_static */

#define MG_BC_NEUMANN 0  /* walls at both ends of the axis: zero normal flux */
#define MG_BC_PERIODIC 1 /* the axis wraps around */

#define MG_PREC_FP64 0  /* every level in FP64 */
#define MG_PREC_MIXED 1 /* FP32 V-cycles inside FP64 iterative refinement */

#define MG_SOLVER_MG 0   /* multigrid iteration: V-cycles inside FP64 iterative refinement */
#define MG_SOLVER_PCG 1  /* conjugate gradients on -A (FP64), preconditioned by V-cycles */

#define MG_PROLONG_TRILINEAR 0 /* prolongation weights 27/9/3/1 over 64 */
#define MG_PROLONG_FLUX 1      /* Sec. 2.3 item 4, Eqs. 13-14: cell flux conservation */

#define MG_FACE_HARMONIC 0   /* Eqs. 11-12: 2 a_L a_R / (a_L + a_R), a = 1/rho */
#define MG_FACE_ARITHMETIC 1 /* (a_L + a_R) / 2 */

#define MG_MAX_COARSE 512 /* most cells of a coarsest grid solved by the dense inverse */
#define MG_MAX_COARSE_GMRES 32768 /* most cells of any coarsest grid (GMRES above MG_MAX_COARSE) */
#define MG_GMRES_RESTART 30 /* Krylov vectors per GMRES cycle on the coarsest grid */

#define MG_COARSE_AUTO 0  /* coarsest solve: dense inverse up to MG_MAX_COARSE cells, else GMRES */
#define MG_COARSE_GMRES 1 /* coarsest solve: restarted GMRES whatever the size */
/* outer iteration of the mixed-precision multigrid iteration (mg_params.outer) */
#define MG_OUTER_FP64 0 /* FP64 residual and FP64 update p += e (Sec. 2.3 with FP32 V-cycles) */
#define MG_OUTER_XP 1   /* the same steps in extended precision from FP32 arithmetic: p held as a
                           sum of three floats (72 bits), b and the finest faces as float pairs,
                           the residual by error-free transformations with exact face differences
                           (about 2^-48 relative per term, FP64: 2^-53); FP64 only in the set-up
                           of a solve and its final conversion.  Ignored for FP64 cycles and CG */
#define MG_STATIC_MAX_CELLS 512 /* most cells of a grid solved by mg_coarse_solve_static */
#define MG_MAX_LEVELS 16

#define MG_TILES_AUTO (-1)   /* mg_params.tiles: time every launch shape per level, keep the fastest */
#define MG_TILES_ROWS 0      /* one grid row per warp, 8 rows per block (no tuning) */
#define MG_TILE_VARIANTS 7   /* launch shapes 0 .. 6 (see mg_tile_shape) */
#define MG_TILE_HALF 0       /* kernels with a tunable launch shape: red-black half-sweep, */
#define MG_TILE_RESTRICT 1   /* residual + restriction, */
#define MG_TILE_PROLONG 2    /* prolongation + correction, */
#define MG_TILE_SWEEP 3      /* finest-level full red-black sweep (0 = two half-sweep launches) */
#define MG_SWEEP_AUTO (-1)   /* mg_params.sweep: timed at create */
#define MG_SWEEP_HALF 0      /* mg_params.sweep: two half-sweep launches per sweep */
#define MG_SWEEP_VARIANTS 11 /* one-pass sweep shapes 1 .. 10 (see mg_sweep_shape) */

typedef struct {
    int nx, ny, nz;     /* cells per axis */
    double lx, ly, lz;  /* domain lengths (h_d = l_d / n_d) */
    int bc[3];          /* MG_BC_NEUMANN or MG_BC_PERIODIC, per axis x, y, z */
} mg_grid;

typedef struct {
    int nu1, nu2;      /* pre- and post-relaxation sweeps (one sweep = red then black), nu1 >= 1 */
    double omega;      /* SOR factor of the red-black relaxation, 0 < omega < 2 */
    int max_iters;     /* most V-cycles per solve */
    int precision;     /* MG_PREC_FP64 or MG_PREC_MIXED */
    int use_graph;     /* 1: run each solve as one CUDA-graph launch; 0: host-driven loop */
    int inner_cycles;  /* most V-cycles per FP64 refinement step (residual evaluation), >= 1;
                          0 (default) = 6 in MIXED precision, 8 in FP64, 1 with MG_SOLVER_PCG */
    int solver;        /* MG_SOLVER_MG (default) or MG_SOLVER_PCG: FP64 conjugate gradients on -A,
                          each step preconditioned by inner_cycles V-cycles from zero (in the
                          V-cycle precision), the preconditioned residual projected to zero mean;
                          beta in the Polak-Ribiere form; iters counts V-cycles */
    int prolongation;  /* MG_PROLONG_TRILINEAR (default) or MG_PROLONG_FLUX: the coarse error
                          at a coarse face, edge or node is the mean of the coarse cells meeting
                          there weighted by their cell coefficient (flux continuity, Eq. 13), a
                          fine cell takes the mean of its octant's 8 corner values; the cell
                          coefficient is the mean alpha of the cell's non-wall faces */
    int tiles;         /* launch shapes of the V-cycle kernels: MG_TILES_AUTO (autotuned per
                          level), MG_TILES_ROWS, or a variant 1 .. MG_TILE_VARIANTS - 1 for
                          every level whose rows are a multiple of 4 cells */
    int coarse_solver;     /* MG_COARSE_AUTO (default) or MG_COARSE_GMRES */
    int coarse_max_iters;  /* GMRES: most Arnoldi steps per coarsest solve (default 300) */
    double coarse_tol;     /* GMRES: relative residual of the coarsest solve (default 1e-8); FP64 */
    int adaptive_cycles;   /* 1 (default): after the first refinement step, each step runs as many
                              V-cycles (1 .. inner_cycles) as the last step's measured reduction
                              rate predicts the tolerance needs, with a 10% margin on the rate;
                              0: always inner_cycles.  Either way a solve stops at max_iters cycles */
    int outer;             /* MG_OUTER_FP64 (default) or MG_OUTER_XP */
    int sweep;             /* finest-level red-black sweep: MG_SWEEP_AUTO (default: the faster of
                              two half-sweep launches per sweep and the one-pass sweep shapes that
                              fit, timed at create), MG_SWEEP_HALF, or a one-pass shape
                              1 .. MG_SWEEP_VARIANTS - 1 (used where it fits, else MG_SWEEP_HALF).
                              The one-pass sweep needs even nu1 and nu2 and a second iterate buffer
                              on the finest level (4 B per cell mixed, 8 B FP64); the staged shapes
                              (tile_x of mg_sweep_shape nonzero) run in FP32 cycles only.  Every
                              choice gives bitwise the same result */
} mg_params;

typedef struct {
    int iters;          /* V-cycles performed (nc of Eq. 15) */
    int status;         /* MG_OK, MG_ENOTCONV or MG_EDIVERGED */
    double rel_res;     /* ||b - A p||_2 / ||b||_2 at exit (b with its mean removed) */
    double res0;        /* R_0: ||b - A p0||_2 for the starting iterate */
    double res;         /* R_nc: final ||b - A p||_2 */
    double gamma;       /* average reduction rate (R_nc / R_0)^(1/nc), Eq. 15 */
    double bnorm;       /* ||b - mean(b)||_2 */
    double rhs_mean;    /* mean of the right-hand side that was removed */
    double ms;          /* device time of the solve (stream events), milliseconds */
    int steps;          /* FP64 refinement steps (residual evaluations after the first) */
    /* served solves only (zero for the other calls): */
    int64_t admit_tick;    /* the server's count of refinement-step launches when the request was admitted */
    int64_t finish_tick;   /* ... when it finished: two requests overlapped on the GPU when their
                              [admit_tick, finish_tick] intervals intersect */
    int inflight_at_admit; /* requests already on the GPU when this one was admitted */
    int lane;              /* size lane that ran it (see mg_server_create) */
} mg_stats;

typedef struct mg_handle mg_handle;
typedef struct mg_batch mg_batch;
typedef struct mg_server mg_server;
typedef int64_t mg_ticket;

/* Error text of a status code (static string). */
const char *mg_strerror(int status);

/* cudaError_t value of the most recent CUDA failure seen by this thread
 * (0 if none); explains an MG_ECUDA return. */
int mg_last_cuda_error(void);

/* Default parameters: V(2,2), omega = 1 (Gauss-Seidel), 100 cycles, mixed
 * precision, CUDA graph on, 2 V-cycles per refinement step. */
int mg_params_default(mg_params *params);

/* Face coefficients alpha = 1/rho of Eqs. 11-12 (mode MG_FACE_HARMONIC) or the
 * arithmetic mean of 1/rho (MG_FACE_ARITHMETIC) from the cell density rho
 * (DEVICE, nx*ny*nz, rho > 0), written to ax, ay, az (DEVICE, nx*ny*nz each,
 * the layout above; Neumann wall entries are written as 0).  Asynchronous on
 * `stream` (a cudaStream_t, NULL = the legacy default stream). */
int mg_faces_from_density(const mg_grid *grid, const double *rho, int mode,
                          double *ax, double *ay, double *az, void *stream);

/* Build a solver for `grid` with face coefficients ax, ay, az (DEVICE, the
 * layout above, alpha > 0 and finite off the walls).  The coefficients are
 * copied (scaled by 1/h^2, coarsened level by level as the mean of the 4 fine
 * faces tiling each coarse face, and the coarsest grid's inverse is formed),
 * so the caller may free them afterwards.  `params` may be NULL (defaults).
 * `stream` is the cudaStream_t all work of the handle runs on (NULL = the
 * legacy default stream).  Steps 1 (operator), 2 (Eqs. 11-12 input), 6
 * (coarsest grid) of Sec. 2.3. */
int mg_create(const mg_grid *grid, const double *ax, const double *ay, const double *az,
              const mg_params *params, void *stream, mg_handle **out);

/* Replace the face coefficients of an existing handle (same grid): the new
 * density of the next time step.  DEVICE pointers, same rules as mg_create.
 * Asynchronous on the handle's stream. */
int mg_set_faces(mg_handle *h, const double *ax, const double *ay, const double *az);

/* mg_faces_from_density followed by mg_set_faces, using the handle's own face
 * storage (no caller buffers besides rho, DEVICE).  Asynchronous. */
int mg_set_density(mg_handle *h, const double *rho, int mode);

/* Solve A p = rhs to ||rhs - A p|| <= tol ||rhs|| (after removing the mean of
 * rhs).  rhs and p are DEVICE arrays of nx*ny*nz doubles (p 16-byte aligned,
 * as every cudaMalloc/torch allocation is); p is the starting
 * iterate on entry (warm start; zeros for a cold start) and the zero-mean
 * solution on exit.  A starting p that is zero in every cell (+0 or -0) is
 * detected on the device and its starting residual taken as rhs - mean(rhs)
 * without the product A p (multigrid iteration; the result is bitwise that of
 * the full evaluation).  rhs is not modified.  Synchronous: returns when the
 * solve has finished on the handle's stream.  `st` may be NULL.  Returns MG_OK,
 * MG_ENOTCONV or MG_EDIVERGED (p then holds the last iterate) or an error.
 *
 * Consecutive kernels of a solve are launched with programmatic dependent
 * launch (each kernel's blocks are placed while the previous kernel runs and
 * wait for its completion before their first memory access); the environment
 * variable MG_DEP_LAUNCH=0, read once per process, turns that off. */
int mg_solve(mg_handle *h, const double *rhs, double *p, double tol, mg_stats *st);

/* Same as mg_solve with HOST arrays (pinned or pageable): copies rhs and the
 * warm start p to the device, solves, copies p back. */
int mg_solve_host(mg_handle *h, const double *rhs_host, double *p_host, double tol, mg_stats *st);

/* mg_set_density + mg_solve_host with HOST rho: one time step's pressure solve
 * from host data (density and right-hand side in, pressure out). */
int mg_step_host(mg_handle *h, const double *rho_host, int mode, const double *rhs_host,
                 double *p_host, double tol, mg_stats *st);

/* Release the handle and its device memory. */
int mg_destroy(mg_handle *h);

/* ---------------------------------------------------------------------------
 * Batched solves: many independent grids of uneven sizes advanced together,
 * one kernel launch per V-cycle stage for the whole batch, the whole solve one
 * CUDA-graph launch.  Each grid's arithmetic is independent of the others, so
 * its result is bitwise the same alone and in any batch.
 * --------------------------------------------------------------------------- */

/* Group `count` handles (all with the same precision and stream) into a batch.
 * The batch does not own the handles; destroy the batch before them. */
int mg_batch_create(mg_handle *const *handles, int count, mg_batch **out);

/* Solve every grid of the batch: rhs[g], p[g] DEVICE arrays as in mg_solve,
 * tol per grid; st (may be NULL) receives `count` records.  Returns MG_OK if
 * every grid converged, else the first failing status. */
int mg_batch_solve(mg_batch *b, const double *const *rhs, double *const *p, const double *tol,
                   mg_stats *st);

int mg_batch_destroy(mg_batch *b);

/* ---------------------------------------------------------------------------
 * Serving: a request loop on a host thread that admits queued solves as slots
 * and device memory (an HBM budget) allow, keeps hierarchies of finished
 * requests for reuse by later requests of the same size, and advances the
 * admitted requests of each size lane together one refinement step at a time
 * (continuous batching): requests join and leave their lane between steps.
 * --------------------------------------------------------------------------- */

/* hbm_budget_bytes: most device memory the server's hierarchies may hold;
 * max_slots: most requests on the GPU at once; params: precision etc. (NULL =
 * defaults); stream: NULL = the server's own streams, one per size lane (grids
 * of up to 64^3, 128^3, 256^3 cells and larger; smaller grids at a higher
 * stream priority), each lane stepping its requests one refinement step at a
 * time at its own pace; a cudaStream_t = every request in one lane on that
 * stream.  Test aid: with the environment variable MG_SERVER_FAIL_AT_STEP=n
 * (read here) the server's n-th step launch reports MG_ECUDA without launching
 * anything, a failure made on the host (see mg_server_drain). */
int mg_server_create(size_t hbm_budget_bytes, int max_slots, const mg_params *params,
                     void *stream, mg_server **out);

/* Queue a solve.  grid, the face coefficients ax/ay/az, rhs and p are as in
 * mg_create/mg_solve (DEVICE); they must stay valid and unmodified until
 * mg_poll reports the ticket finished.  Returns MG_EBUDGET if the request can
 * never fit in the budget. */
int mg_submit(mg_server *s, const mg_grid *grid, const double *ax, const double *ay,
              const double *az, const double *rhs, double *p, double tol, mg_ticket *out);

/* MG_EAGAIN while the ticket is queued or running; otherwise the solve's final
 * status (MG_OK, MG_ENOTCONV, ...) and its statistics, after which the ticket
 * is forgotten (MG_ENOTFOUND on a second poll).  st may be NULL; st->ms is the
 * latency from submission to completion. */
int mg_poll(mg_server *s, mg_ticket t, mg_stats *st);

/* Block until every submitted ticket has finished.  Returns MG_OK, or the
 * error of the first failed step since the server was created (the tickets
 * that failed report it too; the server keeps serving later submissions). */
int mg_server_drain(mg_server *s);

/* Statistics of the server: completed requests, bytes of hierarchies held,
 * peak bytes, most requests in flight at once. */
int mg_server_info(mg_server *s, int64_t *completed, size_t *bytes_in_use, size_t *peak_bytes,
                   int *max_in_flight);

/* Stops the loop; returns MG_EBUSY (and does nothing) if tickets are pending. */
int mg_server_destroy(mg_server *s);

/* ---------------------------------------------------------------------------
 * Single steps of the V-cycle, for unit checks of each kernel.  `level` 0 is
 * the finest grid.  Vectors are DEVICE arrays of the level's cell count, in
 * FP64 when prec = MG_PREC_FP64 and FP32 when prec = MG_PREC_MIXED (the
 * precision the V-cycle of a mixed handle runs in).  Synchronous.
 * --------------------------------------------------------------------------- */

int mg_num_levels(const mg_handle *h, int *levels);
int mg_level_shape(const mg_handle *h, int level, int *nx, int *ny, int *nz);

/* Scaled coefficients w_d = alpha_d / h_d^2 of `level` (FP64, DEVICE out). */
int mg_level_faces(const mg_handle *h, int level, double *wx, double *wy, double *wz);

/* The FP32 copies of the same coefficients that the V-cycles of a mixed-precision
 * handle use (each the FP64 value rounded to nearest, ties to even); DEVICE out,
 * n cells each.  MG_EINVAL for an FP64 handle.  Synchronous. */
int mg_level_faces32(const mg_handle *h, int level, float *wx, float *wy, float *wz);

/* Cell coefficients of `level` used by the flux-conserving prolongation
 * (MG_PROLONG_FLUX, Sec. 2.3 item 4): the mean alpha of each cell's faces that
 * are not walls, from the level's face coefficients; FP64, DEVICE buffer of the
 * level's cells.  Synchronous on the handle's stream.  Any prolongation mode. */
int mg_level_cell_alpha(const mg_handle *h, int level, double *alpha);

/* y = A_level x (Eq. 10 / h^2 on that level). */
int mg_apply(mg_handle *h, int level, int prec, const void *x, void *y);

/* `sweeps` red-black sweeps on x (each: red = (i+j+k) even cells, then black),
 * relaxation factor of the handle (Sec. 2.3 item 5). */
int mg_smooth(mg_handle *h, int level, int prec, const void *b, void *x, int sweeps);

/* coarse_b = mean over the 8 children of (b - A x) on `level` (item 3). */
int mg_restrict_residual(mg_handle *h, int level, int prec, const void *b, const void *x,
                         void *coarse_b);

/* `sweeps` red-black sweeps (item 5) in one launch each: both colours of a
 * sweep in one pass over the level, reading the iterate from one buffer and
 * writing the new iterate to the other: sweep 1 reads x and writes work, sweep
 * 2 reads work and writes x, and so on (after an even number the result is in
 * x, after an odd number in work).  Bitwise the result of mg_smooth.  variant:
 * a one-pass shape 1 .. MG_SWEEP_VARIANTS - 1, or 0 for the handle's tuned
 * choice on that level.  MG_EINVAL if the shape does not fit the level: an
 * even number of cells along a periodic y or z axis, and for a whole-row shape
 * rows of a multiple of 4 cells, at most a third of the shape's threads quads
 * per row; for a staged shape rows of a multiple of its tile_x cells and
 * prec = MG_PREC_MIXED. */
int mg_smooth_onepass(mg_handle *h, int level, int prec, const void *b, void *x, void *work, int sweeps,
                      int variant);

/* x += trilinear prolongation of the coarse error e of level+1 (item 4). */
int mg_prolong(mg_handle *h, int level, int prec, const void *coarse_e, void *x);

/* e = zero-mean solution of A e = r - mean(r) on the coarsest level (item 6). */
int mg_coarse_solve(mg_handle *h, int prec, const void *r, void *e);

/* Exact solve of a small grid without allocating any memory (the paper has no
 * counterpart).  For callers that cannot allocate device memory at the point
 * where they need a solve: a real-time loop whose device memory is budgeted
 * up front, or a host program whose own allocator has reserved the device
 * memory (cudaMalloc may then fail, and it can also synchronise the device).
 *
 * Writes e (DEVICE, nx*ny*nz doubles) = the zero-mean solution of
 * A e = r - mean(r) plus the constant -sum(r) / trace(-A), for the grid
 * `grid` (at most MG_STATIC_MAX_CELLS cells, any size per axis, walls or
 * periodic) with face coefficients ax, ay, az (DEVICE, alpha = 1/rho in the
 * layout above, > 0 off the walls) and right-hand side r (DEVICE), all in
 * FP64.  So e has zero mean exactly when sum(r) = 0.  It assembles
 * -A + c 1 1^T with c = trace(-A) / n^2, inverts it by Gauss-Jordan
 * elimination and applies the inverse, the arithmetic of the coarsest-grid
 * solve of a handle.
 *
 * Scratch: a 2 MiB array in the library's static device memory, held by every
 * device that loads the library until the process exits.  The first call on a
 * device looks up that array's device address; with CUDA's lazy module loading
 * that first call also loads this part of the library's device code (and its
 * static array), which can itself take device memory, so make the first call
 * on each device once at start-up, before any stream capture begins.  Later
 * calls allocate and free nothing.  Every call on a
 * device shares the array and each call rewrites what it reads: calls whose
 * kernels can overlap on the GPU (unordered streams) race and must be
 * serialised by the caller.  Synchronous on `stream` (a cudaStream_t, NULL =
 * legacy default stream): it reads a status word back before returning.
 * Returns MG_ETOOBIG above MG_STATIC_MAX_CELLS cells, MG_EINVAL for bad
 * arguments or coefficients, MG_ESINGULAR for a grid cut into pieces. */
int mg_coarse_solve_static(const mg_grid *grid, const double *ax, const double *ay,
                           const double *az, const double *r, double *e, void *stream);

/* ---------------------------------------------------------------------------
 * The projection step around the solve (Sec. 2.2: Chorin's projection on the
 * staggered MAC grid; S of Eq. 9 from the non-projected velocity).  Face
 * velocities are DEVICE FP64 arrays of the grid's cell count in the layout of
 * the face coefficients: u_d[c] is the normal velocity on the LOW face of cell
 * c along axis d; on a Neumann axis the low face of the first cell is a wall
 * (its entry is ignored: zero normal velocity) and the high wall of the last
 * cell carries none.  The face coefficients are the handle's current ones
 * (mg_create / mg_set_faces / mg_set_density).  Synchronous on the handle's
 * stream; MG_EINVAL for a null pointer or dt not > 0.
 * --------------------------------------------------------------------------- */

/* S = D u / dt: per cell, the sum over axes of (u on the high face - u on the
 * low face) / h_d, divided by dt (second-order centred differences). */
int mg_divergence(mg_handle *h, const double *ux, const double *uy, const double *uz, double dt,
                  double *S);

/* u -= dt alpha G p on every face that is not a wall: u_f -= dt alpha_f
 * (p_c - p_{c-1}) / h_d.  With the operator of Eq. 10 (A = D alpha G), the
 * projected field has D u = dt (S - A p): dt times the solve's residual. */
int mg_project(mg_handle *h, const double *p, double dt, double *ux, double *uy, double *uz);

/* One projection: S = D u / dt (written to the caller's DEVICE buffer S),
 * solve A p = S to tol (p = warm start in, solution out; as mg_solve), then
 * u -= dt alpha G p in place.  Returns the solve's status (MG_OK or
 * MG_ENOTCONV; u is projected with the last iterate) or an error. */
int mg_projection_step(mg_handle *h, double *ux, double *uy, double *uz, double dt, double *p,
                       double *S, double tol, mg_stats *st);

/* ---------------------------------------------------------------------------
 * Timing of individual kernels.  While enabled, every kernel launch of the
 * handle is bracketed by CUDA events on its stream (solves then run as a
 * host-driven loop, not a graph).  mg_profile_read returns, for kernel class
 * `kind` (see below) on `level`, the number of launches and their summed
 * duration in ms since the last reset.
 * --------------------------------------------------------------------------- */
#define MG_K_SMOOTH 0
#define MG_K_RESTRICT 1
#define MG_K_PROLONG 2
#define MG_K_COARSE 3
#define MG_K_RESIDUAL 4 /* the FP64 residual + norms (the update p += e is folded into the cycle) */
#define MG_K_OTHER 5
#define MG_K_TAIL 6 /* the levels of at most 4096 cells and the coarsest solve, one block per grid */
#define MG_K_RESIDUAL0 7 /* the starting residual of a solve (a zero starting iterate skips A p) */
#define MG_K_KINDS 8

int mg_profile_enable(mg_handle *h, int enable);
int mg_profile_read(mg_handle *h, int kind, int level, int64_t *launches, double *total_ms);

/* ---------------------------------------------------------------------------
 * Launch shapes of the V-cycle kernels (no counterpart in the paper, whose
 * solver is an MPI Fortran code; this is the GPU's tiling of Sec. 2.3's
 * relaxation, restriction and prolongation).  With mg_params.tiles =
 * MG_TILES_AUTO, mg_create times every shape that fits each level (half-sweep,
 * restriction, prolongation) on the handle's own work arrays and keeps the
 * fastest; choices are cached per process by kernel, precision, periodic axes
 * and level size.  A shape never changes a result, only its speed.  In a
 * batch, a table of grids takes the shape of its largest grid on that level
 * (the row shape if some grid's rows are not a multiple of 4 cells).
 * --------------------------------------------------------------------------- */

/* Shape chosen for kernel `kind` (MG_TILE_HALF, MG_TILE_RESTRICT,
 * MG_TILE_PROLONG) on `level` of h: 0 .. MG_TILE_VARIANTS - 1 (0 on the
 * coarsest level and on levels run by the bottom-of-cycle kernel); for
 * MG_TILE_SWEEP the finest level's sweep: 0 (two half-sweep launches) or a
 * one-pass shape 1 .. MG_SWEEP_VARIANTS - 1 (0 on every other level). */
int mg_tile_choice(const mg_handle *h, int kind, int level, int *variant);

/* Threads per block and items per thread of shape `variant`: an item is a
 * 4-cell quad of the half-sweep, or a coarse cell pair of the restriction and
 * prolongation (the quad of each of the 2 x 2 fine rows above it).  Variant 0
 * is the row tiling (a warp per row of up to 32 quads, 8 rows per block:
 * reports 256 threads, 1 item). */
int mg_tile_shape(int variant, int *threads, int *items_per_thread);

/* Threads per block, planes per block and tile width of one-pass sweep shape
 * `variant` (1 .. MG_SWEEP_VARIANTS - 1; 0 reports 0, 0, 0).  tile_x = 0: a
 * block owns a strip of full rows (as many as the threads allow at one thread
 * per 4-cell quad, less the two halo rows whose red cells it recomputes) of a
 * chunk of planes, and reads its operands from global memory.  tile_x > 0
 * (staged shapes, FP32 cycles): a block owns a tile of tile_x cells along x
 * and up to 14 rows of a chunk of planes, and copies each plane of its
 * operands (with the halo cells it recomputes) into shared memory two planes
 * ahead of the relaxation. */
int mg_sweep_shape(int variant, int *threads, int *planes, int *tile_x);

/* Forget every cached choice (the next mg_create times again). */
int mg_tune_cache_clear(void);

/* Write the cached choices to the text file `path` (one line per choice:
 * kind precision periodic-bits nx ny nz variant), replacing it. */
int mg_tune_cache_save(const char *path);

/* Add the choices in `path` to the cache (lines that do not parse, or name a
 * shape that does not fit the level, are skipped); *loaded (may be NULL) gets
 * the number of choices read.  MG_ENOTFOUND if the file cannot be opened.
 * When the environment variable MG_TUNE_CACHE names a file, the first tuning
 * of the process loads it and each new choice is appended to it. */
int mg_tune_cache_load(const char *path, int *loaded);

/* Number of cached choices. */
int mg_tune_cache_size(int *entries);

/* Test aid for the bounded device waits (no counterpart in the paper).  The
 * bottom-of-cycle kernel stages its levels by bulk asynchronous copies and
 * waits for them a bounded number of polls (default 2^20; the copies take
 * microseconds); if the wait gives up, the grid's solve reports MG_ETIMEOUT
 * and the kernel still lets the copies land before it exits.  This sets that
 * number of polls for h's later solves: 0 makes the first wait give up at
 * once, so a test can take the timeout path without a fault.  A later
 * mg_set_faces / mg_set_density clears the reported timeout.  Synchronous on
 * h's stream; MG_EINVAL for polls < 0. */
int mg_set_wait_limit(mg_handle *h, long long polls);

/* The parameters h was created with, defaults resolved (inner_cycles). */
int mg_handle_params(const mg_handle *h, mg_params *params);

/* Bytes of device memory the handle holds. */
int mg_memory_bytes(const mg_handle *h, size_t *bytes);

/* Bytes of device memory a handle for `grid` with `params` would hold. */
int mg_memory_estimate(const mg_grid *grid, const mg_params *params, size_t *bytes);

/* ---------------------------------------------------------------------------
 * Device FP64 rate (no counterpart in the paper: the denominator of the FP64
 * roofline of the outer-iteration kernels, whose bound on this GPU is the
 * lesser of the HBM bandwidth and the FP64 issue rate).  Runs a kernel of
 * independent FP64 fused multiply-add chains on every SM of the current
 * device `repeats` times (`iters` steps per chain), each timed with CUDA
 * events on `stream` (a cudaStream_t, NULL = legacy default stream), and
 * writes the best rate in FMA operations per second (an FMA counts once; 2
 * flops) to *fma_per_s.  Allocates one double of device memory for the call.
 * Synchronous.  MG_EINVAL for iters or repeats < 1 or a null output.
 * --------------------------------------------------------------------------- */
int mg_probe_fp64_rate(int iters, int repeats, double *fma_per_s, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GBMG_H */
