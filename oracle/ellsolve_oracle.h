/*
 * ellsolve oracle -- plain, slow, FP64 CPU reference of the discretised model
 * equation of Mueller & Scheichl, "Massively parallel solvers for elliptic PDEs
 * in Numerical Weather- and Climate Prediction" (arXiv:1307.2036), and of the
 * two solvers studied there: the tensor-product geometric multigrid V-cycle
 * (Algorithm 1, Sec. 4.3.1 and 5.2.1) and CG preconditioned by vertical line
 * relaxation (Algorithm PCG, Sec. 4.1 and 5.2.2).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline of the benchmark may load this code.  It shares no code, header,
 * table generator or helper with the CUDA library, and it never reads anything
 * the CUDA library produced.
 *
 * Vector layout: v[k * ncol + c], c = (p * n + j) * n + i, i.e. the vertical
 * index k slowest, then panel p, then the horizontal indices j, i.
 */
#ifndef ELLSOLVE_ORACLE_H
#define ELLSOLVE_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct og_grid og_grid;

/* kind: 0 doubly periodic box of side `side`, 1 cubed sphere (6 panels).
 * mapping (sphere only): 0 equiangular, 1 equidistant gnomonic (Eq. x1x2_2).
 * r: nz+1 radii r_0 < ... < r_nz (copied).  omega2 = omega^2, lambda2 = lambda^2
 * of Eq. ModelEquation.  The hierarchy halves n while n is even and n/2 >=
 * coarsest_min, with at most max_levels levels (max_levels <= 0: no cap). */
og_grid *og_create(int kind, int n, int nz, int mapping, double side,
                   const double *r, double omega2, double lambda2,
                   int coarsest_min, int max_levels);
void og_destroy(og_grid *g);

int og_nlevels(const og_grid *g);
int og_npanel(const og_grid *g);
int og_level_n(const og_grid *g, int lev);
long og_level_ncol(const og_grid *g, int lev);

/* Geometry copies: area[ncol], trans[ncol*4] = face length / centre distance,
 * nbr[ncol*4] (faces ordered -i, +i, -j, +j), centres xyz[ncol*3]. */
void og_get_geometry(const og_grid *g, int lev, double *area, double *trans, long *nbr);
void og_get_centres(const og_grid *g, int lev, double *xyz);
void og_get_face_lengths(const og_grid *g, int lev, double *ell, double *dist);
void og_get_radial(const og_grid *g, double *V, double *G);
void og_volumes(const og_grid *g, int lev, double *vol);

/* Operator (Sec. 3.1, 7-point cell-centred finite volumes). */
void og_apply(const og_grid *g, int lev, const double *u, double *y);
void og_residual(const og_grid *g, int lev, const double *b, const double *u, double *r);
void og_assemble_dense(const og_grid *g, int lev, double *M);

/* Tridiagonal solvers (Algorithm Thomas).  og_thomas_paper takes the matrix in
 * the paper's notation (a diagonal, b super-, c sub-diagonal); og_thomas_excess
 * takes the diagonal as delta_i + up_i + lo_i with b_i = -up_i, c_i = -lo_i. */
void og_thomas_paper(int n, const double *a, const double *b, const double *c,
                     const double *f, double *u);
void og_thomas_excess(int n, const double *delta, const double *up, const double *lo,
                      const double *f, double *u);

/* Damped block-Jacobi vertical line relaxation, nsweeps sweeps, in place. */
void og_smooth(const og_grid *g, int lev, const double *b, double *u, int nsweeps, double rho);
/* z = Dtilde^{-1} r (the block-Jacobi preconditioner). */
void og_line_precond(const og_grid *g, int lev, const double *r, double *z);

/* Block red-black SOR (Eq. BlockRBSOR): red columns (i + j even), then black,
 * each column of the colour updated from the current iterate; in place. */
void og_smooth_rb(const og_grid *g, int lev, const double *b, double *u, int nsweeps, double rho);
/* z = M^{-1} r for block red-black SSOR: half-sweeps red, black, black, red of
 * A z = r from z = 0. */
void og_rb_ssor(const og_grid *g, int lev, const double *r, double *z, double rho);
/* Smoother of og_smooth / og_vcycle / og_mg_solve: 0 block Jacobi (default),
 * 1 block red-black SOR.  Preconditioner of og_pcg_solve: 0 block Jacobi
 * (default), 1 block red-black SSOR with parameter rho, 2 one V-cycle. */
void og_set_smoother(og_grid *g, int kind);
/* Vertical background profiles: V_k *= p_cell[k] (k < nz), G_k *= q_face[k]
 * (0 < k < nz).  Call once, before any other use of the grid. */
void og_set_profiles(og_grid *g, const double *p_cell, const double *q_face);
void og_set_precond(og_grid *g, int kind, double rho);
/* Kind 2 of og_set_precond: one V-cycle from zero (the grid's smoother) with
 * these sweeps, damping and prolongation; PCG then takes the flexible beta. */
void og_set_mg_precond(og_grid *g, int nu_pre, int nu_post, int nu_coarse, double rho,
                       int prolong_mode);

/* Intergrid transfers between level lev_f and lev_f + 1. */
void og_restrict(const og_grid *g, int lev_f, const double *r_f, double *b_c);
void og_prolong_add(const og_grid *g, int lev_f, const double *u_c, double *u_f, int mode);

/* One V-cycle on the finest level, in place on u.  b is volume integrated. */
void og_vcycle(const og_grid *g, const double *b, double *u, int nu_pre, int nu_post,
               int nu_coarse, double rho, double rho_coarse, int prolong_mode);

/* With on != 0 the first cycle of og_mg_solve and the V-cycle preconditioner
 * (og_set_precond kind 2) are full multigrid cycles (og_fmg). */
void og_set_fmg(og_grid *g, int on);

/* Full multigrid: b restricted to every level, the coarsest level smoothed
 * from zero, then on each finer level the prolongated coarse solution as the
 * start of one V-cycle.  u (finest level) is overwritten. */
void og_fmg(const og_grid *g, const double *b, double *u, int nu_pre, int nu_post, int nu_coarse,
            double rho, double rho_coarse, int prolong_mode);

/* Solvers starting from u = 0.  hist[0..maxit] receives ||r_K||/||r_0||.
 * Return the number of iterations done. */
int og_mg_solve(const og_grid *g, const double *b, double *u, double rtol, int maxit,
                int nu_pre, int nu_post, int nu_coarse, double rho, double rho_coarse,
                int prolong_mode, double *hist);
int og_pcg_solve(const og_grid *g, const double *b, double *u, double rtol, int maxit,
                 double *hist);

#ifdef __cplusplus
}
#endif
#endif
