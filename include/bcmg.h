/*
 * bcmg.h -- C ABI of the GB300 (sm_103a) ghost-point Boundary Condition
 * MultiGrid solver.
 *
 * Method: Coco, Mazza and Semplice, "A ghost-point smoothing strategy for
 * geometric multigrid on curved boundaries" (arXiv 2207.14208).  The solver
 * treats -Lap u = f in Omega = {phi < 0} inside D = [-1,1]^d (d = 2 or 3)
 * with Dirichlet data g on the curved boundary by the ghost-point method of
 * Sec. 3.3 and relaxes every ghost equation with the distance-dependent
 * fictitious-time step Delta tau_OPT(theta~) of eq. DtauOptTheta.
 *
 * Grid and layout (Sec. 3 and Sec. 4 set-up): N cells per axis, n = N + 1
 * nodes per axis, x_i = -1 + i h, h = 2/N.  Every grid array passed through
 * this ABI is dense FP64 with n^d entries, x fastest: index i + n j + n^2 k.
 *
 * Node classes: INTERIOR (phi < 0, not on the box boundary), GHOST (phi >= 0
 * with an interior axis neighbour), BOXDIR (phi < 0 on the box boundary: an
 * eliminated Dirichlet node whose value is read from u), INACTIVE.
 *
 * Conventions of every entry point:
 *  - the return value is a status (BCMG_OK = 0 or one of the codes below);
 *    nothing throws across the ABI; bcmg_last_error() gives a message for
 *    the calling thread's last failure;
 *  - "_dev" pointers are CUDA device pointers, "_host" pointers host memory;
 *    the caller owns every pointer it passes; the handle owns everything else;
 *  - work is stream-ordered on the stream given at creation; entry points
 *    that return host data (counts, norms, host copies) synchronise it;
 *  - a call that reads or writes caller arrays must not overlap on the GPU
 *    with another call on the same handle (calls on one handle are ordered);
 *  - handles may be created and used from several threads at once; creation
 *    (opts.use_graph) records the solve graph by stream capture on the
 *    handle's own non-blocking stream, and while a capture is open CUDA
 *    rejects a device- or context-wide synchronisation (cudaDeviceSynchronize)
 *    from any thread: concurrent threads synchronise streams or events.
 */
#ifndef BCMG_H
#define BCMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BCMG_OK 0
#define BCMG_EINVAL 1     /* bad argument (null pointer, size, level) */
#define BCMG_ENOMEM 2     /* device or host allocation failed */
#define BCMG_ECUDA 3      /* a CUDA runtime call failed */
#define BCMG_EGEOM 4      /* no interior node, or singular / oversized coarsest system */
#define BCMG_ENOCONV 5    /* solve hit max_cycles before rtol */
#define BCMG_ENONFINITE 6 /* NaN or Inf in the residual */

#define BCMG_CLASS_INACTIVE 0
#define BCMG_CLASS_INTERIOR 1
#define BCMG_CLASS_GHOST 2
#define BCMG_CLASS_BOXDIR 3

#define BCMG_DTAU_EXP 0   /* G0 = exp(-p theta): Remark exptheta2D (default) */
#define BCMG_DTAU_POLY 1  /* G0 of eqs. G / G3D with coefficients eq. coeff */
#define BCMG_DTAU_CONST 2 /* one Delta tau for every ghost (Remark dtau) */

typedef struct bcmg_h *bcmg_handle;

typedef struct {
    int nu1;           /* pre-smoothing steps (Sec. 3.1: 2) */
    int nu2;           /* post-smoothing steps (Sec. 3.1: 1) */
    int dtau_mode;     /* BCMG_DTAU_* */
    double dtau_const; /* Delta tau (Neumann: Delta tau / h) when
                          dtau_mode == BCMG_DTAU_CONST */
    int ext_sweeps;    /* pseudo-time sweeps of the normal extension (4) */
    int min_coarse;    /* coarsening stops before N_l / 2 < min_coarse (8) */
    int max_levels;    /* upper bound on the number of levels (24) */
    int use_graph;     /* replay the V-cycle from a captured CUDA graph:
                          1 the solve graph is captured at creation
                          (default), 2 at the first bcmg_solve that needs
                          it (creation costs less when the handle is only
                          solved through the batched kernels of
                          bcmg_solve_batch), 0 never (host-driven loop) */
    int profile;       /* time every finest-level smoothing sweep with CUDA
                          events during bcmg_solve (0) */
    int precision;     /* BCMG_PREC_FP64 (default) or BCMG_PREC_MIXED */
    int bc;            /* boundary condition on Gamma: BCMG_BC_DIRICHLET
                          (default) or BCMG_BC_NEUMANN */
    double reaction;   /* c >= 0 of the interior equation c u - Lap u = f
                          (0: Poisson, the default; Sec. 4.2 Test2N: 1) */
    int cycle;         /* BCMG_CYCLE_V (gamma = 1, default), BCMG_CYCLE_W
                          (gamma = 2) or BCMG_CYCLE_TG (the two-grid
                          correction scheme: the level-1 problem solved by
                          tg_inner V-cycles), Sec. 2.1 */
    int ordering;      /* interior Gauss-Seidel order: BCMG_ORDER_RB
                          (red-black, default) or BCMG_ORDER_LEX
                          (lexicographic, the paper's GS-LEX, eq. GSLEX_2D,
                          run as a sweep over the hyperplanes i+j(+k) = p;
                          one launch per hyperplane, for comparisons) */
    int tg_inner;      /* V-cycles of the level-1 solve of BCMG_CYCLE_TG
                          (30: at the method's contraction the coarse
                          problem is then solved to rounding) */
} bcmg_opts;

#define BCMG_ORDER_RB 0
#define BCMG_ORDER_LEX 1

#define BCMG_CYCLE_V 0
#define BCMG_CYCLE_W 1
#define BCMG_CYCLE_TG 2

/* Boundary conditions on Gamma (Sec. 3): Dirichlet u = g; Neumann
 * grad u . n = g with n the ghost's outward unit normal (bcmg_ghost_normals),
 * the ghost row being the normal derivative at Q of the same interpolant
 * (Sec. 3.2.2, Sec. 4.1) relaxed with Delta tau = h (Delta tau / h)_OPT(theta)
 * (eqs. dtauoptLFA_Neumann, dtauoptLFA3D_Neumann; with BCMG_DTAU_CONST,
 * dtau_const is Delta tau / h).  Box-boundary nodes inside the domain stay
 * eliminated Dirichlet nodes (Test1N of Sec. 4.2). */
#define BCMG_BC_DIRICHLET 0
#define BCMG_BC_NEUMANN 1

#define BCMG_PREC_FP64 0  /* every cycle in FP64 */
#define BCMG_PREC_MIXED 1 /* FP64 iterative refinement: FP64 residual and
                             update, the V-cycle on the correction in FP32 */

/* Fill *opts with the defaults above. */
void bcmg_default_opts(bcmg_opts *opts);

/* The relaxation parameter the library gives a ghost at distance theta
 * (= |G - Q| / h, in [0, 1]): Delta tau_OPT(theta) of eqs. DtauOptTheta,
 * dtauoptLFA / dtauoptLFA3D (Dirichlet) or Delta tau_OPT / h of eqs.
 * dtauoptLFA_Neumann / dtauoptLFA3D_Neumann (Neumann), with the G0 form of
 * dtau_mode (BCMG_DTAU_EXP, BCMG_DTAU_POLY) or dtau_const for
 * BCMG_DTAU_CONST.  Host function; *out receives the value. */
int bcmg_dtau_opt(int dim, int bc, int dtau_mode, double dtau_const, double theta, double *out);

/* Build the level hierarchy (Sec. 2.1 re-discretisation, Sec. 3.3 geometry):
 * per level the node classes from phi injected to the level, the ghost list
 * with projection points Q = G - eta h n (phi(Q) = 0), upwind 3^d stencils,
 * quadratic interpolation weights and Delta tau_OPT(eta) (eq. DtauOptTheta),
 * the inactive band that receives normal extensions, and the inverse of the
 * coarsest system.
 *   dim      2 or 3
 *   N        cells per axis, N >= 4
 *   phi_dev  n^dim level-set values (read during the call only)
 *   f_dev    n^dim right-hand side of -Lap u = f (interior values are
 *            copied; may be NULL for f = 0)
 *   opts     NULL for the defaults
 *   stream   cudaStream_t (NULL = legacy default stream)
 *   out      receives the handle
 * Errors: EINVAL, ENOMEM, ECUDA, EGEOM (no interior node on the finest grid,
 * or the coarsest system is singular or has more than 4096 unknowns). */
int bcmg_create_grid_hierarchy(int dim, int64_t N, const double *phi_dev, const double *f_dev,
                               const bcmg_opts *opts, void *stream, bcmg_handle *out);

/* bcmg_create_grid_hierarchy on the box [lo, lo + N h]^dim with a caller's
 * device workspace (Sec. 3 and Sec. 4 set-up: a uniform grid of (N+1)^dim
 * nodes x_i = lo + i h on every axis; the paper's D = [-1, 1]^d is lo = -1,
 * h = 2 / N, which is what bcmg_create_grid_hierarchy passes).
 *   lo, h      node 0's coordinate and the finest spacing (h > 0, finite);
 *              level l has spacing h 2^l.  h scales the interior rows
 *              (1 / h^2), Neumann rows (1 / h) and the Neumann Delta tau
 *              (h (Delta tau / h)_OPT); classes, projections and stencils
 *              are index-space quantities and do not depend on lo or h.
 *              Projection points Q (bcmg_ghost_points) are returned in
 *              these coordinates.
 *   workspace  NULL: the library allocates (stream-ordered pool, with its
 *              own cache).  Otherwise a caller-owned device buffer, 256-byte
 *              aligned, of ws_bytes bytes, from which every device array of
 *              the hierarchy and all of its set-up scratch are carved (no
 *              library allocation of device memory); it must stay valid and
 *              untouched until bcmg_destroy, which does not free it.  If it
 *              is too small, creation fails with BCMG_ENOMEM and the
 *              message states the size reached; bcmg_workspace_size of a
 *              hierarchy of the same geometry and options gives the size
 *              that suffices, bcmg_footprint_estimate a guide.
 * Other arguments and errors as bcmg_create_grid_hierarchy; EINVAL also for
 * a non-finite lo, h <= 0, or a misaligned / empty workspace. */
int bcmg_create_grid_hierarchy_ex(int dim, int64_t N, double lo, double h, const double *phi_dev,
                                  const double *f_dev, const bcmg_opts *opts, void *workspace, size_t ws_bytes,
                                  void *stream, bcmg_handle *out);

/* Bytes of device memory the creation of h drew (its arrays and its set-up
 * scratch): a workspace of this size suffices to create a hierarchy of the
 * same dim, N, phi and options with bcmg_create_grid_hierarchy_ex.  (No
 * counterpart in the paper.) */
int bcmg_workspace_size(bcmg_handle h, int64_t *bytes);

/* Fixes the launch shape of the batched kernels of bcmg_solve_batch for the
 * calls that follow, in place of the autotuner's choice (no counterpart in
 * the paper; for tests and measurements):
 *   block      threads per block of the stage kernels: 64, 128 or 256; 0
 *              returns to the autotuner
 *   items      items per thread of the node-parallel stages: 1 or 4
 *   tail_rows  coarse levels whose lists all have at most this many entries
 *              run in one block per hierarchy (the block tail); 0: none
 * Results do not depend on the shape (the same per-node arithmetic in the
 * same order).  Process-wide.  EINVAL for other values. */
int bcmg_debug_batch_shape(int block, int items, int64_t tail_rows);

/* The launch shape (block size, items per thread, tail rows; see
 * bcmg_debug_batch_shape) the process's last batched solve used: the
 * autotuner's choice for that batch's shape, or the fixed one.  block = 0
 * when no batched solve has run.  (No counterpart in the paper.) */
int bcmg_batch_last_shape(int *block, int *items, int64_t *tail_rows);

/* Failure injection for tests of the callers' recovery paths (no
 * counterpart in the paper): after this call, the k-th device allocation the
 * library makes (counted over all handles and threads) fails as if the device
 * memory were exhausted, and the call that needed it returns BCMG_ENOMEM
 * after releasing what it had taken.  k = 0 disables.  Host-side only. */
int bcmg_debug_fail_allocation(int64_t k);

/* Device blocks (and their bytes) that live handles hold from the library's
 * allocator, outside its cache of returned blocks and outside caller
 * workspaces; 0 once every handle is destroyed (leak checks in tests; no
 * counterpart in the paper). */
int bcmg_debug_live_blocks(int64_t *blocks, int64_t *bytes);

/* Release every resource of the handle (NULL is accepted). */
int bcmg_destroy(bcmg_handle h);

/* Number of ghost points on the finest level. */
int bcmg_ghost_count(bcmg_handle h, int64_t *n);

/* Projection points Q of the finest-level ghosts (Sec. 3.3), ghost-list order
 * (increasing node index), written as count x dim FP64 (x, y[, z]) to Q: a
 * device buffer (stream-ordered) or host memory (pageable or page-locked;
 * filled when the call returns, which then synchronises the handle's
 * stream).  The caller evaluates its boundary data there. */
int bcmg_ghost_points(bcmg_handle h, double *Q);

/* Outward unit normals n (computed from phi at each ghost G, Sec. 3.3) of
 * the finest-level ghosts, ghost-list order, count x dim FP64 to the device
 * buffer n_dev: the direction of the Neumann data. */
int bcmg_ghost_normals(bcmg_handle h, double *n_dev);

/* Boundary data for the finest-level ghosts (eq. BCh right-hand side):
 * Dirichlet values g(Q), or Neumann values grad u(Q) . n with n from
 * bcmg_ghost_normals; count FP64 values in ghost-list order, from device
 * memory (stream-ordered) or host memory (read before the call returns). */
int bcmg_set_boundary_values(bcmg_handle h, const double *g);

/* Replace the interior right-hand side f (n^dim, device; NULL = 0). */
int bcmg_set_rhs(bcmg_handle h, const double *f_dev);

/* ncycles V(nu1, nu2) cycles (Sec. 2.1, gamma = 1) on u_dev (n^dim, device,
 * in/out).  Interior and ghost nodes are updated; BOXDIR values are read as
 * eliminated Dirichlet data; every other node of u is left untouched. */
int bcmg_vcycle(bcmg_handle h, double *u_dev, int ncycles);

/* V-cycles until ||r||_2 <= rtol ||r^(0)||_2 (r stacked over interior and
 * ghost rows, Sec. 2.2) or max_cycles.  cycles_done and final_rel_res may be
 * NULL.  Returns ENOCONV if max_cycles is reached, ENONFINITE on NaN/Inf. */
int bcmg_solve(bcmg_handle h, double *u_dev, double rtol, int max_cycles, int *cycles_done,
               double *final_rel_res);

/* Many solves at once (uneven sizes and geometries welcome).
 *   handles[n], u_devs[n]  distinct handles and their u arrays (as for
 *                          bcmg_solve); rtol, max_cycles shared by all
 *   cycles_done[n], final_rel_res[n], statuses[n]   per-solve results
 *                          (host arrays, each may be NULL)
 * Batched kernels: when n >= 2 and every handle has the same dimension,
 * working precision, device, nu1 and nu2, red-black ordering and V-cycles,
 * the solves run together, one launch per stage of the V-cycle for all
 * hierarchies (levels aligned by depth), in a CUDA graph whose loop runs
 * while any solve is unfinished; a finished hierarchy's work is skipped.
 * The launch shape (block size, items per thread) is measured once per
 * batch shape class on the first call of that class (an autotuner; it runs
 * batched cycles on the hierarchies' working copies only); a class is the
 * device, dimension and precision with the number of hierarchies and their
 * total rows each rounded up to a power of two.  Per node the arithmetic is that
 * of bcmg_solve; the coarse levels and the norm reduction sum in another
 * order, so results agree with bcmg_solve alone to rounding (and a cycle
 * count within a few cycles of it), not bit for bit.  The work is ordered
 * after each handle's stream (the stream given at its creation) and is
 * complete when the call returns.
 * Otherwise (mixed batches) every handle's solve is enqueued on its own
 * stream before any is waited for, so the GPU runs them concurrently, and
 * results are identical to bcmg_solve on each handle alone; a handle created
 * with profile = 1 or use_graph = 0 runs its host-driven loop in a second
 * pass.  Returns BCMG_OK if every solve converged, else the first failing
 * status (per-solve ones in statuses); EINVAL for null arrays or a handle
 * that appears twice. */
int bcmg_solve_batch(bcmg_handle *handles, double **u_devs, int n, double rtol, int max_cycles,
                     int *cycles_done, double *final_rel_res, int *statuses);

/* ncycles V-cycles (as bcmg_vcycle) on each of n hierarchies at once:
 * handles[n], u_devs[n] as for bcmg_solve_batch.  An eligible batch (see
 * bcmg_solve_batch) runs through the batched kernels, exactly ncycles
 * cycles per hierarchy whatever its residual, complete when the call
 * returns; other batches enqueue each handle's cycles on its own stream
 * before any is waited for (results identical to bcmg_vcycle on each
 * handle).  EINVAL for null arrays, a handle that appears twice or
 * ncycles < 0. */
int bcmg_vcycle_batch(bcmg_handle *handles, double **u_devs, int n, int ncycles);

/* Device memory (bytes) the handle holds: every level's arrays, lists and
 * tables (not the caller's phi, f or u). */
int bcmg_memory_footprint(bcmg_handle h, int64_t *bytes);

/* A-priori estimate of the device memory a hierarchy of this size will hold
 * (no phi needed), for admission control: the dense per-level arrays over
 * the levels the coarsening rule allows, times 2 for the compacted lists,
 * plus 12 MiB for the chunks small arrays are carved from.  It exceeds bcmg_memory_footprint on the shapes the tests
 * cover; geometries with far more boundary than the test domains can
 * exceed it.  opts may be NULL (defaults). */
int bcmg_footprint_estimate(int dim, int64_t N, const bcmg_opts *opts, int64_t *bytes);

/* The same estimate with the grid size given per axis (N[dim]; size_t
 * result): the library's grids are cubic, so every entry must equal N[0]
 * (EINVAL otherwise). */
int bcmg_footprint(int dim, const int64_t *N, const bcmg_opts *opts, size_t *bytes);

/* Residual norms of u_dev on the finest level into out_host[4]:
 * ||r_I||_2, ||r_G||_2, ||r_I||_inf, ||r_G||_inf (unscaled residuals). */
int bcmg_residual_norm(bcmg_handle h, const double *u_dev, double *out_host);

/* Thread-local message of the last failing call ("" if none). */
const char *bcmg_last_error(void);

/* Kernels this process launched through the library so far (each replayed
 * CUDA-graph node counts once per replay). */
int64_t bcmg_kernel_launches(void);

/* With opts.profile = 1: out_host[0] = summed device time (ms) of the
 * finest-level red/black interior sweeps run by bcmg_solve on this handle,
 * out_host[1] = their number (CUDA events recorded on the launching stream,
 * read after each cycle). */
int bcmg_profile_read(bcmg_handle h, double *out_host);

/* Residual norms for callers that cannot allocate device memory (code that
 * runs inside a stream capture, plugins whose host owns every allocation,
 * processes that forbid cudaMalloc after start-up).  The paper has no
 * counterpart: this is a service of the library, not a step of the method.
 *   r_dev    count FP64 residual values (device), e.g. from bcmg_residual
 *   cls_dev  count node classes (device, BCMG_CLASS_*), e.g. from
 *            bcmg_get_class; only INTERIOR and GHOST entries are summed
 *   count    number of entries, 1 <= count <= 33554432 (the capacity of the
 *            library's fixed scratch); larger counts return BCMG_EINVAL
 *   out_dev  4 FP64 (device): ||r_I||_2, ||r_G||_2, ||r_I||_inf, ||r_G||_inf
 *   stream   cudaStream_t the two kernels are launched on (NULL = legacy)
 * Allocates nothing: the per-block partial sums live in a fixed 128 KiB
 * __device__ array that every device loading the library keeps until the
 * process exits.  The first call on each device resolves that array's device
 * address (cudaGetSymbolAddress) and should come before any stream capture.
 * All calls share the array, so calls that overlap on the GPU race; order
 * them (same stream or events).  Asynchronous: returns after the launches. */
int bcmg_residual_norms_static(const double *r_dev, const uint8_t *cls_dev, int64_t count, double *out_dev,
                               void *stream);

/* Self-test of the division the restriction uses for family means (no
 * counterpart in the paper; the restriction of Sec. 3.3.2 divides by the
 * family's FW weight sum): out_host[i] = a_host[i] / w with w = 1 + i % 64,
 * computed on the device the way the restriction computes it (a table
 * reciprocal and one FMA correction, Markstein's method), in FP64
 * (fp32 = 0) or FP32 (fp32 = 1, result widened).  1 <= n <= 2^24.
 * Synchronous; allocates and frees its own device buffer.  Errors: EINVAL,
 * ENOMEM, ECUDA. */
int bcmg_selftest_div_wsum(int fp32, const double *a_host, int64_t n, double *out_host);

/* Timing of the finest-level interior sweep (eq. GSLEX_2D in red-black
 * order, the dominant kernel of a cycle): nsweeps alternating red and black
 * sweeps of the finest level, in the handle's working precision, launched
 * back to back on the handle's stream between two CUDA events, as they run
 * inside a cycle; *ms_host receives their summed device time (ms).  The
 * sweeps act on the handle's internal working copy only (the next vcycle or
 * solve copies the caller's u in again).  Red-black ordering only.
 * Synchronous.  Errors: EINVAL, ECUDA. */
int bcmg_time_sweeps(bcmg_handle h, int nsweeps, double *ms_host);

/* The same sweeps with u and the scaled right-hand side stored as bfloat16
 * (8-bit significand; sums and updates in FP32, results rounded to nearest)
 * on temporary copies of the working arrays, which are freed again; the
 * handle is left unchanged.  A measurement of what 16-bit storage would
 * gain on the dominant kernel (the paper computes in double precision
 * throughout; no counterpart there).  The finest level must be split by
 * parity (even N).  Synchronous.  Errors: EINVAL, ENOMEM, ECUDA. */
int bcmg_time_sweeps_bf16(bcmg_handle h, int nsweeps, double *ms_host);

/* ---- introspection (host copies, synchronous) ----------------------- */

int bcmg_num_levels(bcmg_handle h, int *levels);

/* out_host[10]: N, n, n^dim, interior, ghost, band, boxdir, clamped (eta
 * forced to 1), stencil fall-backs, active unknowns of the coarsest system
 * (0 on other levels). */
int bcmg_level_info(bcmg_handle h, int level, int64_t *out_host);

/* out_host[3]: the level's interior rows by their part in the cycle's
 * residual: red rows ((i + j [+ k]) even), black rows with a neighbour that
 * is not interior (a ghost or a box-edge node), and the black rows whose 2d
 * neighbours are all interior.  After a red-black smoothing step (red
 * sweep, black sweep, ghost relaxation, Sec. 2.1 with eq. rel for the
 * ghosts) the residual of a row of the third part is zero up to rounding,
 * so the cycle's residual computes the first two parts only and stores zero
 * in the third (no counterpart in the paper).  Errors: EINVAL. */
int bcmg_level_lists(bcmg_handle h, int level, int64_t *out_host);

/* n^dim node classes (BCMG_CLASS_*) of a level. */
int bcmg_get_class(bcmg_handle h, int level, uint8_t *cls_host);

/* Ghost list of a level (ng entries; the vector fields hold 3 per ghost,
 * unused axes 0): node index, eta, outward normal n, local coordinates xi of
 * Q in the stencil, stencil direction s (+1: stencil towards -x_a), degree q
 * per axis, Delta tau, and Q.  Any output pointer may be NULL. */
int bcmg_get_ghosts(bcmg_handle h, int level, int64_t *idx, double *eta, double *n3, double *xi3,
                    int32_t *s3, int32_t *q3, double *dtau, double *Q3);

/* Band node indices of a level (increasing). */
int bcmg_get_band(bcmg_handle h, int level, int64_t *idx_host);

/* ---- stage operators on caller arrays of one level (device, n_l^dim) --
 * These run the same kernels as the V-cycle; they exist so that every step
 * of the cycle can be called and checked on its own. */

/* nsteps smoothing steps: red then black Gauss-Seidel on interior nodes
 * (eq. GSLEX_2D in red-black order), then the simultaneous fictitious-time
 * relaxation of every ghost (eq. rel with Delta tau of eq. DtauOptTheta). */
int bcmg_smooth(bcmg_handle h, int level, double *u_dev, const double *F_dev, int nsteps);

/* r = F - A u on interior (eq. Laph) and ghost (eq. BCh) rows; other nodes
 * of r are left untouched. */
int bcmg_residual(bcmg_handle h, int level, const double *u_dev, const double *F_dev,
                  double *r_dev);

/* Extend ghost values of a into the band along the normal (Sec. 3.3.2). */
int bcmg_extend(bcmg_handle h, int level, double *a_dev);

/* Class-aware restriction (Sec. 3.3.2) of r on level `level` to F on
 * level + 1 (interior and ghost coarse nodes written, others untouched). */
int bcmg_restrict(bcmg_handle h, int level, const double *r_fine_dev, double *F_coarse_dev);

/* u_fine += multilinear interpolation of e_coarse (level + 1) on the fine
 * interior and ghost nodes (Sec. 3.3.2). */
int bcmg_prolong(bcmg_handle h, int level, const double *e_coarse_dev, double *u_fine_dev);

/* Exact correction on the coarsest level: u += A^-1 (F - A u). */
int bcmg_coarsest_solve(bcmg_handle h, double *u_dev, const double *F_dev);

#ifdef __cplusplus
}
#endif

#endif /* BCMG_H */
