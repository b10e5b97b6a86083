/*
 * ellsolve -- GB300 (sm_103a) solver for the elliptic model equation of
 * Mueller & Scheichl, "Massively parallel solvers for elliptic PDEs in
 * Numerical Weather- and Climate Prediction" (arXiv:1307.2036):
 *
 *     -omega^2 (Laplace_2d u + lambda^2 r^-2 d/dr (r^2 du/dr)) + u = f     (Eq. ModelEquation)
 *
 * on the shell 1 <= r <= 1 + H over a doubly periodic box or the cubed sphere
 * (Eqs. x1x2_1, x1x2_2), homogeneous Neumann at the bottom and top (Sec. 3),
 * discretised with cell-centred finite volumes and a 7-point stencil
 * (Sec. 3.1).  Solvers: the tensor-product geometric multigrid V-cycle
 * (Algorithm 1; horizontal-only coarsening, vertical line relaxation,
 * Sec. 4.3.1 and 5.2.1) and CG preconditioned by vertical line relaxation
 * (Algorithm PCG, Sec. 6.2.2).
 *
 * Conventions for every call below:
 *  - Vectors are device buffers of doubles in the layout [nz][P][n][n]:
 *    element (k, p, j, i) at ((k * P + p) * n + j) * n + i, P = 1 (box) or 6
 *    (sphere).  Panel p of the sphere is the cube face with outward normal
 *    N_p, its index i runs along A_p and j along B_p, where
 *      p  N_p        A_p        B_p
 *      0  (+1,0,0)   (0,+1,0)   (0,0,+1)
 *      1  (0,+1,0)   (-1,0,0)   (0,0,+1)
 *      2  (-1,0,0)   (0,-1,0)   (0,0,+1)
 *      3  (0,-1,0)   (+1,0,0)   (0,0,+1)
 *      4  (0,0,+1)   (0,+1,0)   (-1,0,0)
 *      5  (0,0,-1)   (0,+1,0)   (+1,0,0)
 *    and a point of the panel is N_p + xi A_p + eta B_p projected to the sphere.
 *  - Right-hand sides are the pointwise f of Eq. ModelEquation; the library
 *    forms the volume-integrated b = A_P V_k f.  ellsolve_apply returns the
 *    matrix-vector product y = A x of the finite-volume matrix (volume
 *    integrated).  Relative residuals are ||b - A u||_2 / ||b||_2.
 *  - Buffers are owned by the caller; the library never frees them and only
 *    reads/writes them on the handle's CUDA stream, in stream order.
 *  - Calls return a status; none aborts.  On an error the thread-local
 *    message of ellsolve_last_error() says what failed.
 *  - A handle is not thread-safe: one host thread at a time per handle.
 */
#ifndef ELLSOLVE_H
#define ELLSOLVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ellsolve_s *ellsolve_t;
typedef struct ellsolve_server_s *ellsolve_server_t;

typedef enum {
    ELLSOLVE_OK = 0,
    ELLSOLVE_NOT_CONVERGED = 1, /* maxit reached, or the residual stagnated above rtol */
    ELLSOLVE_PENDING = 2,       /* ellsolve_poll: not finished within the timeout */
    ELLSOLVE_ERR_ARG = -1,      /* invalid argument (null pointer, bad size, bad option) */
    ELLSOLVE_ERR_CUDA = -2,     /* a CUDA runtime call failed */
    ELLSOLVE_ERR_NOMEM = -3,    /* device memory allocation failed */
    ELLSOLVE_ERR_NONFINITE = -4,/* a residual norm became NaN or Inf */
    ELLSOLVE_ERR_CAPACITY = -5  /* request larger than the server's HBM budget or slots */
} ellsolve_status;

typedef struct {
    int kind;        /* 0: doubly periodic box (P = 1), 1: cubed sphere (P = 6) */
    int n;           /* cells per panel side (>= 1) */
    int nz;          /* vertical levels (>= 1) */
    double box_side; /* box only: side length (2 pi in the configs) */
    int mapping;     /* sphere only: 0 equiangular, 1 equidistant gnomonic (Eq. x1x2_2) */
} ellsolve_grid;

typedef struct {
    int precision;    /* 0: FP64 throughout; 1: FP32 V-cycles inside FP64 iterative refinement */
    int solver;       /* 0: multigrid V-cycles (Algorithm 1); 1: PCG (Algorithm PCG) */
    int nu_pre;       /* pre-smoothing line-Jacobi sweeps (2) */
    int nu_post;      /* post-smoothing sweeps (2) */
    int nu_coarse;    /* sweeps on the coarsest level (2) */
    double damping;   /* line-Jacobi damping rho (0.8); the coarsest level is undamped */
    int coarsest_min; /* coarsen while n is even and n/2 >= coarsest_min (4) */
    int max_levels;   /* cap on the number of levels, <= 0: no cap */
    int prolong;      /* 0: bilinear (cell-centred), 1: piecewise constant */
    int inner_cycles; /* precision 1: FP32 V-cycles per FP64 refinement step (3) */
    int use_graph;    /* 1: replay the per-iteration work as a CUDA graph */
    int smoother;     /* 0: damped block (line) Jacobi; 1: block red-black SOR (Eq.
                       * BlockRBSOR) with rho = damping, a sweep being a red then a
                       * black half-sweep; a column is red when i + j is even.  On
                       * the cubed sphere, which has no two-colouring, a half-sweep
                       * updates its columns from the iterate before it (0) */
    int precond;      /* PCG: 0 block Jacobi Dtilde^{-1}; 1 block red-black SSOR
                       * (half-sweeps red, black, black, red from 0, rho = 1); 2 one
                       * FP64 V-cycle from 0 with the options above (smoother,
                       * sweeps, damping, prolongation), CG then taking the flexible
                       * beta <r, z - z_old> / <r_old, z_old> (0) */
    int fmg;          /* 1: every V-cycle that starts from a zero iterate (the first
                       * cycle of precision-0 multigrid, the first inner cycle of each
                       * refinement step, the precond-2 preconditioner) is one full
                       * multigrid cycle (Sec. 4.3): the right-hand side restricted to
                       * every level, nu_coarse sweeps from zero on the coarsest, then
                       * per finer level the interpolated coarse solution as the start
                       * of one V-cycle from that level (0) */
    int refine;       /* precision 1, the FP64 residual b - A x of each refinement
                       * step: 0 tracked -- the step updates the stored residual by
                       * -A e in double-float (pairs of binary32) together with x,
                       * with a running bound on its rounding; when the bound is not
                       * below 0.1% of the residual, the residual is recomputed in
                       * FP64 and later steps recompute it; 1 recomputed in FP64 at
                       * every step (0) */
    int line_part;    /* precision 1, the line solves of the small levels (at most
                       * 9,728 columns, n_z % 16 == 0, n_z <= 256), which wait on the
                       * elimination chain of a column: 0 one thread eliminates the
                       * whole column (twisted Thomas, as on the large levels); 1 eight
                       * warps eliminate eight segments of it at once, joined by a
                       * tridiagonal system on the seven levels between them (1) */
} ellsolve_opts;

typedef struct {
    int iterations;      /* V-cycles (MG) or CG iterations done */
    double rel_residual; /* final ||b - A u|| / ||b|| (FP64) */
    double seconds;      /* wall time of the solve on the stream */
    /* Estimate of the relative error ||x* - x|| / ||x*|| against the exact
     * solution x* of the discrete problem, which the FP64 solvers approach.
     * Mixed precision (precision 1): from the refinement updates of x, as
     * q / (1 - q) ||dx_last|| / ||dx_first|| (the error left by a linearly
     * contracting iteration; x starts at 0, so the first update is x* to
     * within the first step's contraction), with q the last step's residual
     * reduction scaled by how much more the error than the residual
     * contracted in the step before (||dx_last|| / ||dx_prev|| against that
     * step's residual reduction).  -1 for the FP64 multigrid and PCG solvers,
     * which report the exact residual only. */
    double rel_error_est;
} ellsolve_result;

/* Fill *o with the defaults listed above. */
void ellsolve_default_opts(ellsolve_opts *o);

/* Build the grid hierarchy and device workspace for one problem.
 *  grid     : box or cubed sphere (copied).
 *  omega2   : omega^2 of Eq. ModelEquation (> 0).
 *  lambda2  : lambda^2 (> 0).
 *  r_levels : host array of nz+1 radii, strictly increasing (copied); Eq.
 *             VerticalGrading gives r_k = 1 + H (k/nz)^2.
 *  opts     : solver options (copied; NULL = defaults).
 *  stream   : cudaStream_t for every later call on the handle (NULL = legacy default).
 *  out      : receives the handle.
 * Errors: ELLSOLVE_ERR_ARG, ELLSOLVE_ERR_NOMEM, ELLSOLVE_ERR_CUDA. */
ellsolve_status ellsolve_create(const ellsolve_grid *grid, double omega2, double lambda2,
                                const double *r_levels, const ellsolve_opts *opts,
                                void *stream, ellsolve_t *out);
/* As ellsolve_create, with vertical background profiles (Sec. 2, the operator
 * D^(z) of Eq. FullSISLEquation): the equation multiplied by the weight p(r)
 * r^2, p = (pi*)^gamma c_p theta*, with q = 1 / (1 + (alpha dt)^2 (N*)^2) in
 * the vertical flux.  The tensor-product structure is unchanged; only the
 * per-level vectors change:
 *   p_cell : nz host values, (int p r^2 dr) / (int r^2 dr) over layer k, > 0;
 *            multiplies V_k in the mass and horizontal terms and in b.
 *   q_face : nz+1 host values, p(r_k) q(r_k) at interface k, > 0 for k =
 *            1..nz-1 (entries 0 and nz are not read: the Neumann faces).
 * Either may be NULL (all ones); both NULL is ellsolve_create.  Copied.
 * Errors as ellsolve_create, and ERR_ARG for a non-positive or non-finite
 * profile value.  Servers take no profiles. */
ellsolve_status ellsolve_create_profiles(const ellsolve_grid *grid, double omega2, double lambda2,
                                         const double *r_levels, const double *p_cell,
                                         const double *q_face, const ellsolve_opts *opts,
                                         void *stream, ellsolve_t *out);
void ellsolve_destroy(ellsolve_t h);

/* Sizes: unknowns on the finest level, and the hierarchy depth. */
size_t ellsolve_size(ellsolve_t h);
int ellsolve_num_levels(ellsolve_t h);

/* y = A x on the finest level (Sec. 3.1 stencil), FP64 device buffers. */
ellsolve_status ellsolve_apply(ellsolve_t h, const void *x_dev, void *y_dev);

/* One multigrid V-cycle (Algorithm 1) in place on u_dev for the pointwise
 * right-hand side f_dev.  precision 1: one refinement step (FP64 residual, FP32
 * V-cycle on it, FP64 update). */
ellsolve_status ellsolve_vcycle(ellsolve_t h, const void *f_dev, void *u_dev);

/* Solve A x = b (b = volume-integrated f) from x = 0 until the relative
 * residual is <= rtol, maxit iterations pass, or the residual stops falling
 * (the attainable FP64 residual is about eps ||A|| ||x|| / ||b||).
 * Returns OK, NOT_CONVERGED (result and x still filled), or an error. */
ellsolve_status ellsolve_solve(ellsolve_t h, const void *rhs_dev, void *x_dev, double rtol,
                               int maxit, ellsolve_result *res);

/* Solve several independent problems in one pass: every multigrid kernel is
 * launched once per level over all members (count handles, all created with
 * precision 1 and solver 0, on the same stream as handles[0]).  rhs/x: arrays
 * of count device pointers.  res: count results.  Returns the worst status. */
ellsolve_status ellsolve_solve_batch(ellsolve_t *handles, int count, const void *const *rhs_dev,
                                     void *const *x_dev, double rtol, int maxit,
                                     ellsolve_result *res);

/* ---- per-level operations on the handle's hierarchy (kernel-level access) ----
 * Vectors here are volume-integrated right-hand sides b and iterates u of level
 * `level` (0 finest) in the same [nz][P][n][n] layout; fp32 selects float
 * buffers and the FP32 kernels, otherwise double. */
ellsolve_status ellsolve_level_shape(ellsolve_t h, int level, int *n, size_t *ncol);
/* y = A_level x */
ellsolve_status ellsolve_level_apply(ellsolve_t h, int level, int fp32, const void *x, void *y);
/* r = b - A_level u */
ellsolve_status ellsolve_level_residual(ellsolve_t h, int level, int fp32, const void *b,
                                        const void *u, void *r);
/* nsweeps damped block-Jacobi vertical line relaxation sweeps (Sec. 4.2,
 * Algorithm Thomas per column), u <- u + rho Dtilde^{-1}(b - A u), in place. */
ellsolve_status ellsolve_level_smooth(ellsolve_t h, int level, int fp32, const void *b, void *u,
                                      int nsweeps, double rho);
/* b_c = R (b - A u) on level+1: residual summed over the 2 x 2 children (Sec. 6.2.1). */
ellsolve_status ellsolve_level_restrict_residual(ellsolve_t h, int level, int fp32,
                                                 const void *b, const void *u, void *b_c);
/* u += P u_c from level+1 (bilinear or constant per opts.prolong). */
ellsolve_status ellsolve_level_prolong_add(ellsolve_t h, int level, int fp32, const void *u_c,
                                           void *u);

/* ellsolve_level_smooth for callers that cannot allocate device memory (the
 * paper has no counterpart: this is a deployment variant).  Such callers are,
 * for example, host programs that give the library a fixed device-memory
 * budget owned by their own allocator or memory pool (a cudaMalloc outside
 * that pool would overrun the budget, or fail once the pool holds the memory),
 * and latency-critical loops where a cudaMalloc / cudaFree pair could
 * synchronise the device.  It runs the same kernels as ellsolve_level_smooth
 * with the same work items and gives the same result bit for bit, but takes
 * its scratch (the partner iterate, the Thomas coefficients, the level
 * descriptor and the work items) from one 64 MiB array that the library holds
 * in static device memory on every GPU where it is loaded, until the process
 * exits.  It calls no cudaMalloc, cudaFree or other allocating routine.
 *  - Limit: the level must need at most 64 MiB of scratch, about
 *    2 * unknowns * sizeof(element) + 4 KB; larger levels return
 *    ELLSOLVE_ERR_CAPACITY with a message.  Nothing in the array needs to
 *    start at zero: every scratch value is written before it is read.
 *  - The device current at the call must be the one current when the handle
 *    was created (ELLSOLVE_ERR_ARG otherwise): the array is per device.
 *  - The first call on a device looks up the array's device address with
 *    cudaGetSymbolAddress (once per device, with that device current); make
 *    that first call before any stream capture on the device.
 *  - All calls on a device share the one array and it keeps the last call's
 *    contents, so calls whose work overlaps on the GPU (from several host
 *    threads or streams) race and must be serialised by the caller.
 *  - The descriptor and work items are copied from host memory, and the call
 *    waits for the handle's stream before returning. */
ellsolve_status ellsolve_level_smooth_noalloc(ellsolve_t h, int level, int fp32, const void *b,
                                              void *u, int nsweeps, double rho);

/* ---- profiling: CUDA-event time of the finest-level smoother launches ----
 * enable != 0 starts recording an event pair around every finest-level
 * line-smoother launch on the handle's stream (and resets the totals).
 * profile_read returns the summed event time, the number of launches timed
 * and their summed algorithmic bytes: per unknown, a sweep reads u and b and
 * writes u (3 words), or reads b and writes u when the iterate is zero (2). */
ellsolve_status ellsolve_profile_enable(ellsolve_t h, int enable);
ellsolve_status ellsolve_profile_read(ellsolve_t h, double *smoother_ms_total, int *launches,
                                      double *bytes_total);
/* number of kernel launches the library issued on this handle so far */
uint64_t ellsolve_launch_count(ellsolve_t h);

/* ---- autotuning ----
 * Times, on every level of the handle's hierarchy, the launch shapes of its
 * kernels and keeps the fastest for later solves on this handle and for
 * batches led by it: for the FP32 line smoother, the resident CTAs per SM (the
 * occupancy cap bounds the L2 working set of the back substitution), the depth
 * of its shared-memory staging ring (prefetch distance against shared memory
 * per CTA) and whether the eliminated right-hand side is parked in tensor
 * memory or in the output buffer; for the residual + restriction and the
 * prolongation of small levels, how far a launch is split along the vertical.
 * The choice changes no result (same arithmetic, different scheduling).  Uses
 * the handle's own FP32 buffers as scratch: call it between solves.
 * precision 1 only.  out_ctas / out_ms (nullable) receive the finest level's
 * CTA cap and its time per sweep.  The paper has no counterpart (its kernels
 * are tuned by hand). */
ellsolve_status ellsolve_autotune(ellsolve_t h, int *out_ctas, double *out_ms);
/* Set the smoother's CTA cap and ring depth on every level, or read the
 * finest level's: ctas_per_sm 0..16 (0 = as many as fit), ring 4 or 8 steps;
 * ERR_ARG outside those.  No result depends on them. */
ellsolve_status ellsolve_set_tuning(ellsolve_t h, int ctas_per_sm, int ring);
ellsolve_status ellsolve_get_tuning(ellsolve_t h, int *ctas_per_sm, int *ring);
/* Set or read one level's launch shape: the streaming smoother's ctas_per_sm
 * (0..16) and ring (4 or 8), tmem (where it parks its eliminated right-hand
 * side: 0 tensor memory on launches of at least 152 CTAs, 1 always while
 * n_z <= 256, 2 never), staged (the fully staged smoother, which copies every
 * level into shared memory first: 0 on launches of fewer than 152 blocks of
 * 128 columns, 1 always, 2 never; where n_z % 16 == 0 and n_z <= 256), and the
 * block counts (>= 1) up to which the restriction from this level and the
 * prolongation onto it are split along the vertical.  ERR_ARG outside those
 * or for a level the handle lacks.  No result depends on them. */
ellsolve_status ellsolve_set_level_tuning(ellsolve_t h, int level, int ctas_per_sm, int ring,
                                          int tmem, int staged, int restrict_chunk,
                                          int prolong_chunk);
ellsolve_status ellsolve_get_level_tuning(ellsolve_t h, int level, int *ctas_per_sm, int *ring,
                                          int *tmem, int *staged, int *restrict_chunk,
                                          int *prolong_chunk);

/* ---- serving: continuous batching of independent solves ----
 * A server owns one CUDA stream's worth of work; submitted requests are admitted
 * while their device footprint fits hbm_budget_bytes and a slot is free, and
 * all admitted requests advance together (one batched launch per level). */
ellsolve_status ellsolve_server_create(size_t hbm_budget_bytes, int max_slots, void *stream,
                                       ellsolve_server_t *out);
/* Copies grid, parameters and r_levels; borrows rhs_dev and x_dev until the
 * request's poll returns OK, NOT_CONVERGED or an error. */
ellsolve_status ellsolve_submit(ellsolve_server_t s, const ellsolve_grid *grid, double omega2,
                                double lambda2, const double *r_levels, const void *rhs_dev,
                                void *x_dev, double rtol, int maxit, uint64_t *ticket);
/* Wait up to timeout_us (0: do not wait, < 0: forever) for the request. */
ellsolve_status ellsolve_poll(ellsolve_server_t s, uint64_t ticket, int timeout_us,
                              ellsolve_result *res);
void ellsolve_server_destroy(ellsolve_server_t s);

/* ---- self-test ----
 * Runs the library's device self-checks on the current device: the exact
 * binary32 <-> binary64 conversions the FP64 refinement kernels do with integer
 * arithmetic are compared bit for bit with the hardware conversions over
 * `samples` pseudo-random bit patterns (a quarter of them on rounding ties).
 * *mismatches (nullable) receives the count.  Returns OK when it is zero,
 * ERR_CUDA with a message otherwise.  Allocates 8 bytes of device memory.
 * The paper has no counterpart. */
ellsolve_status ellsolve_selftest(uint64_t samples, uint64_t *mismatches);

const char *ellsolve_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
