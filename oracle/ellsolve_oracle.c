/*
 * ellsolve oracle -- plain, slow, FP64 CPU reference (TEST INFRASTRUCTURE ONLY).
 *
 * Follows Mueller & Scheichl, arXiv:1307.2036:
 *   model equation            Eq. ModelEquation (Sec. 3), Neumann top/bottom
 *   cubed-sphere grid         Eqs. x1x2_1, x1x2_2 (Sec. 3.1)
 *   vertical grading          Eq. VerticalGrading (Sec. 3.1)
 *   cell-centred FV, 7 points Sec. 3.1 (two-point face fluxes)
 *   tensor-product structure  Sec. 4.3.1
 *   block (line) relaxation   Sec. 4.2, Eq. BlockRBSOR with the Jacobi ordering
 *   Thomas algorithm          Algorithm Thomas (appendix)
 *   V-cycle                   Algorithm 1 (Sec. 4.3), components of Sec. 6.2.1
 *   full multigrid            Sec. 4.3 (first guess built from the coarsest
 *                             level upwards, one V-cycle per level)
 *   PCG                       Algorithm PCG (appendix), sign of the residual
 *                             update read as r_K = r_{K-1} - alpha q_{K-1}
 *
 * Only the tests, the smoke check and the CPU baseline of the benchmark may
 * load this file's library.  Nothing here is shared with the CUDA library.
 */
#include "ellsolve_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define MAXLEV 32
#define OG_PI 3.14159265358979323846

typedef struct {
    int n;         /* cells per panel side */
    long ncol;     /* P * n * n */
    double *area;  /* [ncol] cell area on the unit sphere (or the flat box) */
    double *ell;   /* [ncol*4] face lengths */
    double *dist;  /* [ncol*4] distances between the two cell centres */
    long *nbr;     /* [ncol*4] neighbouring column across each face */
    double *xyz;   /* [ncol*3] cell centres (unit sphere; box: x, y, 0) */
} og_level;

struct og_grid {
    int kind, P, nz, mapping, nlev;
    int smoother;        /* 0 block Jacobi, 1 block red-black SOR */
    int precond;         /* PCG: 0 block Jacobi, 1 block red-black SSOR, 2 one V-cycle */
    double precond_rho;  /* relaxation parameter of the SSOR preconditioner */
    int mg_nu_pre, mg_nu_post, mg_nu_coarse, mg_prolong;  /* V-cycle preconditioner */
    int fmg;             /* cycles from a zero iterate are full multigrid cycles */
    double mg_rho;
    double side, omega2, lambda2;
    double *r, *V, *G;  /* r[nz+1], V[nz], G[nz+1] */
    og_level lev[MAXLEV];
};

/* ------------------------------------------------------------------------ */
/* Cube panels.  Panel p is the cube face with outward normal N[p]; the      */
/* horizontal indices i, j run along A[p], B[p] (A x B = N).  A point on the */
/* panel is N + xi A + eta B with xi, eta in [-1, 1] (Eq. x1x2_1 up to the   */
/* labelling of the axes).                                                   */
/* ------------------------------------------------------------------------ */
static const int PN[6][3] = {{1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
static const int PA[6][3] = {{0, 1, 0}, {-1, 0, 0}, {0, -1, 0}, {1, 0, 0}, {0, 1, 0}, {0, 1, 0}};
static const int PB[6][3] = {{0, 0, 1}, {0, 0, 1}, {0, 0, 1}, {0, 0, 1}, {-1, 0, 0}, {1, 0, 0}};

/* Mapping coordinate of grid line t (may be half-integer) out of n.  The
 * equidistant gnomonic grid of Eq. x1x2_2 is uniform in xi = tan(phi); the
 * equiangular grid is uniform in the angle. */
static double og_mapcoord(int mapping, double t, int n)
{
    if (mapping == 1) return -1.0 + 2.0 * t / (double)n;
    return tan(-OG_PI / 4.0 + t * (OG_PI / 2.0) / (double)n);
}

static void og_sphere_point(int p, double xi, double eta, double out[3])
{
    double X[3], len = 0.0;
    for (int d = 0; d < 3; ++d) {
        X[d] = PN[p][d] + xi * PA[p][d] + eta * PB[p][d];
        len += X[d] * X[d];
    }
    len = sqrt(len);
    for (int d = 0; d < 3; ++d) out[d] = X[d] / len;
}

/* great-circle arc between unit vectors, via the chord length */
static double og_arc(const double a[3], const double b[3])
{
    double s = 0.0;
    for (int d = 0; d < 3; ++d) s += (a[d] - b[d]) * (a[d] - b[d]);
    return 2.0 * asin(0.5 * sqrt(s));
}

/* solid angle of the spherical triangle a, b, c (Van Oosterom & Strackee) */
static double og_tri_area(const double a[3], const double b[3], const double c[3])
{
    double bxc[3] = {b[1] * c[2] - b[2] * c[1], b[2] * c[0] - b[0] * c[2], b[0] * c[1] - b[1] * c[0]};
    double trip = a[0] * bxc[0] + a[1] * bxc[1] + a[2] * bxc[2];
    double ab = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
    double bc = b[0] * c[0] + b[1] * c[1] + b[2] * c[2];
    double ca = c[0] * a[0] + c[1] * a[1] + c[2] * a[2];
    return 2.0 * atan2(fabs(trip), 1.0 + ab + bc + ca);
}

/* Neighbour of cell (p, i, j) across face q (0: -i, 1: +i, 2: -j, 3: +j),
 * found by stepping on the surface of the cube [-n, n]^3 in integer units:
 * the centre of cell (p, i, j) is n N + (2i+1-n) A + (2j+1-n) B; a step of
 * one cell crosses into the neighbouring face when it leaves [-n, n]. */
static long og_sphere_neighbour(int n, int p, int i, int j, int q)
{
    long X[3], D[3];
    int sgn = (q == 0 || q == 2) ? -1 : 1;
    const int *axis = (q < 2) ? PA[p] : PB[p];
    for (int d = 0; d < 3; ++d) {
        X[d] = (long)n * PN[p][d] + (long)(2 * i + 1 - n) * PA[p][d] + (long)(2 * j + 1 - n) * PB[p][d];
        D[d] = sgn * axis[d];
    }
    long along = X[0] * D[0] + X[1] * D[1] + X[2] * D[2];
    if (along + 2 <= n - 1) {
        for (int d = 0; d < 3; ++d) X[d] += 2 * D[d];
    } else {
        /* to the cube edge, then one unit down the neighbouring face */
        for (int d = 0; d < 3; ++d) X[d] += D[d] - PN[p][d];
    }
    /* locate the face: the coordinate with |X| == n */
    int pp = -1;
    for (int f = 0; f < 6; ++f) {
        long dot = X[0] * PN[f][0] + X[1] * PN[f][1] + X[2] * PN[f][2];
        if (dot == n) { pp = f; break; }
    }
    long xa = X[0] * PA[pp][0] + X[1] * PA[pp][1] + X[2] * PA[pp][2];
    long xb = X[0] * PB[pp][0] + X[1] * PB[pp][1] + X[2] * PB[pp][2];
    long ii = (xa + n - 1) / 2, jj = (xb + n - 1) / 2;
    return ((long)pp * n + jj) * n + ii;
}

static void og_build_level(og_grid *g, og_level *L, int n)
{
    int P = g->P;
    L->n = n;
    L->ncol = (long)P * n * n;
    L->area = (double *)calloc(L->ncol, sizeof(double));
    L->ell = (double *)calloc(L->ncol * 4, sizeof(double));
    L->dist = (double *)calloc(L->ncol * 4, sizeof(double));
    L->nbr = (long *)calloc(L->ncol * 4, sizeof(long));
    L->xyz = (double *)calloc(L->ncol * 3, sizeof(double));

    if (g->kind == 0) {
        double h = g->side / n;
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                long c = (long)j * n + i;
                L->area[c] = h * h;
                L->nbr[4 * c + 0] = (long)j * n + (i + n - 1) % n;
                L->nbr[4 * c + 1] = (long)j * n + (i + 1) % n;
                L->nbr[4 * c + 2] = (long)((j + n - 1) % n) * n + i;
                L->nbr[4 * c + 3] = (long)((j + 1) % n) * n + i;
                for (int q = 0; q < 4; ++q) {
                    L->ell[4 * c + q] = h;
                    L->dist[4 * c + q] = h;
                }
                L->xyz[3 * c + 0] = (i + 0.5) * h;
                L->xyz[3 * c + 1] = (j + 0.5) * h;
                L->xyz[3 * c + 2] = 0.0;
            }
        return;
    }

    /* cubed sphere */
    for (int p = 0; p < 6; ++p)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                long c = ((long)p * n + j) * n + i;
                double x0 = og_mapcoord(g->mapping, i, n), x1 = og_mapcoord(g->mapping, i + 1, n);
                double y0 = og_mapcoord(g->mapping, j, n), y1 = og_mapcoord(g->mapping, j + 1, n);
                double c00[3], c10[3], c01[3], c11[3], ctr[3];
                og_sphere_point(p, x0, y0, c00);
                og_sphere_point(p, x1, y0, c10);
                og_sphere_point(p, x0, y1, c01);
                og_sphere_point(p, x1, y1, c11);
                og_sphere_point(p, og_mapcoord(g->mapping, i + 0.5, n), og_mapcoord(g->mapping, j + 0.5, n), ctr);
                L->area[c] = og_tri_area(c00, c10, c11) + og_tri_area(c00, c11, c01);
                L->ell[4 * c + 0] = og_arc(c00, c01);
                L->ell[4 * c + 1] = og_arc(c10, c11);
                L->ell[4 * c + 2] = og_arc(c00, c10);
                L->ell[4 * c + 3] = og_arc(c01, c11);
                for (int d = 0; d < 3; ++d) L->xyz[3 * c + d] = ctr[d];
                for (int q = 0; q < 4; ++q) L->nbr[4 * c + q] = og_sphere_neighbour(n, p, i, j, q);
            }
    for (long c = 0; c < L->ncol; ++c)
        for (int q = 0; q < 4; ++q) L->dist[4 * c + q] = og_arc(&L->xyz[3 * c], &L->xyz[3 * L->nbr[4 * c + q]]);
}

og_grid *og_create(int kind, int n, int nz, int mapping, double side, const double *r,
                   double omega2, double lambda2, int coarsest_min, int max_levels)
{
    og_grid *g = (og_grid *)calloc(1, sizeof(og_grid));
    g->smoother = 0;
    g->precond = 0;
    g->precond_rho = 1.0;
    g->mg_nu_pre = g->mg_nu_post = g->mg_nu_coarse = 2;
    g->mg_rho = 0.8;
    g->mg_prolong = 0;
    g->kind = kind;
    g->P = kind == 0 ? 1 : 6;
    g->nz = nz;
    g->mapping = mapping;
    g->side = side;
    g->omega2 = omega2;
    g->lambda2 = lambda2;
    g->r = (double *)malloc((nz + 1) * sizeof(double));
    g->V = (double *)malloc(nz * sizeof(double));
    g->G = (double *)calloc(nz + 1, sizeof(double));
    memcpy(g->r, r, (nz + 1) * sizeof(double));
    /* V_k = int_{r_k}^{r_{k+1}} r^2 dr, written as the factored difference of
     * cubes so that thin cells keep full relative accuracy. */
    for (int k = 0; k < nz; ++k) {
        double a = r[k], b = r[k + 1];
        g->V[k] = (b - a) * (b * b + a * b + a * a) / 3.0;
    }
    /* G_k = r_k^2 / (rho_k - rho_{k-1}) with cell centres rho_k = (r_k + r_{k+1})/2;
     * zero flux through r_0 and r_nz (homogeneous Neumann). */
    for (int k = 1; k < nz; ++k) g->G[k] = 2.0 * r[k] * r[k] / (r[k + 1] - r[k - 1]);
    g->G[0] = 0.0;
    g->G[nz] = 0.0;

    int nl = 0, m = n;
    for (;;) {
        og_build_level(g, &g->lev[nl], m);
        ++nl;
        if (m % 2 != 0 || m / 2 < coarsest_min || nl >= MAXLEV) break;
        if (max_levels > 0 && nl >= max_levels) break;
        m /= 2;
    }
    g->nlev = nl;
    return g;
}

void og_destroy(og_grid *g)
{
    if (!g) return;
    for (int l = 0; l < g->nlev; ++l) {
        free(g->lev[l].area);
        free(g->lev[l].ell);
        free(g->lev[l].dist);
        free(g->lev[l].nbr);
        free(g->lev[l].xyz);
    }
    free(g->r);
    free(g->V);
    free(g->G);
    free(g);
}

int og_nlevels(const og_grid *g) { return g->nlev; }
int og_npanel(const og_grid *g) { return g->P; }
int og_level_n(const og_grid *g, int lev) { return g->lev[lev].n; }
long og_level_ncol(const og_grid *g, int lev) { return g->lev[lev].ncol; }

void og_get_geometry(const og_grid *g, int lev, double *area, double *trans, long *nbr)
{
    const og_level *L = &g->lev[lev];
    for (long c = 0; c < L->ncol; ++c) {
        area[c] = L->area[c];
        for (int q = 0; q < 4; ++q) {
            trans[4 * c + q] = L->ell[4 * c + q] / L->dist[4 * c + q];
            nbr[4 * c + q] = L->nbr[4 * c + q];
        }
    }
}

void og_get_centres(const og_grid *g, int lev, double *xyz)
{
    memcpy(xyz, g->lev[lev].xyz, g->lev[lev].ncol * 3 * sizeof(double));
}

void og_get_face_lengths(const og_grid *g, int lev, double *ell, double *dist)
{
    memcpy(ell, g->lev[lev].ell, g->lev[lev].ncol * 4 * sizeof(double));
    memcpy(dist, g->lev[lev].dist, g->lev[lev].ncol * 4 * sizeof(double));
}

void og_get_radial(const og_grid *g, double *V, double *G)
{
    memcpy(V, g->V, g->nz * sizeof(double));
    memcpy(G, g->G, (g->nz + 1) * sizeof(double));
}

void og_volumes(const og_grid *g, int lev, double *vol)
{
    const og_level *L = &g->lev[lev];
    for (int k = 0; k < g->nz; ++k)
        for (long c = 0; c < L->ncol; ++c) vol[k * L->ncol + c] = L->area[c] * g->V[k];
}

/* ------------------------------------------------------------------------ */
/* Operator.  Integrating Eq. ModelEquation over the cell P x [r_k, r_{k+1}]  */
/* with two-point face fluxes gives                                          */
/*   (Au)_{P,k} = A_P V_k u_{P,k}                                            */
/*              + omega^2 V_k sum_Q (l_PQ / d_PQ) (u_{P,k} - u_{Q,k})         */
/*              + omega^2 lambda^2 A_P [G_{k+1} (u_{P,k} - u_{P,k+1})         */
/*                                      + G_k (u_{P,k} - u_{P,k-1})]          */
/* ------------------------------------------------------------------------ */
static double og_row(const og_grid *g, const og_level *L, const double *u, long c, int k)
{
    long nc = L->ncol;
    double up = u[k * nc + c];
    double horiz = 0.0;
    for (int q = 0; q < 4; ++q) {
        double T = L->ell[4 * c + q] / L->dist[4 * c + q];
        horiz += T * (up - u[k * nc + L->nbr[4 * c + q]]);
    }
    double vert = 0.0;
    if (k + 1 < g->nz) vert += g->G[k + 1] * (up - u[(k + 1) * nc + c]);
    if (k > 0) vert += g->G[k] * (up - u[(k - 1) * nc + c]);
    return L->area[c] * g->V[k] * up + g->omega2 * g->V[k] * horiz +
           g->omega2 * g->lambda2 * L->area[c] * vert;
}

void og_apply(const og_grid *g, int lev, const double *u, double *y)
{
    const og_level *L = &g->lev[lev];
    for (int k = 0; k < g->nz; ++k)
        for (long c = 0; c < L->ncol; ++c) y[k * L->ncol + c] = og_row(g, L, u, c, k);
}

void og_residual(const og_grid *g, int lev, const double *b, const double *u, double *r)
{
    const og_level *L = &g->lev[lev];
    for (int k = 0; k < g->nz; ++k)
        for (long c = 0; c < L->ncol; ++c) {
            long m = k * L->ncol + c;
            r[m] = b[m] - og_row(g, L, u, c, k);
        }
}

/* Dense matrix (row-major, N = nz * ncol) assembled entry by entry from the
 * stencil coefficients; independent of og_apply. */
void og_assemble_dense(const og_grid *g, int lev, double *M)
{
    const og_level *L = &g->lev[lev];
    long nc = L->ncol, N = nc * g->nz;
    memset(M, 0, (size_t)(N * N) * sizeof(double));
    double w2 = g->omega2, wl2 = g->omega2 * g->lambda2;
    for (int k = 0; k < g->nz; ++k)
        for (long c = 0; c < nc; ++c) {
            long row = k * nc + c;
            M[row * N + row] += L->area[c] * g->V[k];
            for (int q = 0; q < 4; ++q) {
                double t = w2 * g->V[k] * L->ell[4 * c + q] / L->dist[4 * c + q];
                long col = k * nc + L->nbr[4 * c + q];
                M[row * N + row] += t;
                M[row * N + col] -= t;
            }
            if (k + 1 < g->nz) {
                double t = wl2 * L->area[c] * g->G[k + 1];
                M[row * N + row] += t;
                M[row * N + (k + 1) * nc + c] -= t;
            }
            if (k > 0) {
                double t = wl2 * L->area[c] * g->G[k];
                M[row * N + row] += t;
                M[row * N + (k - 1) * nc + c] -= t;
            }
        }
}

/* ------------------------------------------------------------------------ */
/* Algorithm Thomas, literally: a diagonal, b super-diagonal, c sub-diagonal. */
/* ------------------------------------------------------------------------ */
void og_thomas_paper(int n, const double *a, const double *b, const double *c,
                     const double *f, double *u)
{
    double *bp = (double *)malloc(n * sizeof(double));
    double *fp = (double *)malloc(n * sizeof(double));
    bp[0] = (n > 1) ? b[0] / a[0] : 0.0;
    fp[0] = f[0] / a[0];
    for (int i = 1; i < n - 1; ++i) {
        double den = a[i] - bp[i - 1] * c[i];
        bp[i] = b[i] / den;
        fp[i] = (f[i] - fp[i - 1] * c[i]) / den;
    }
    if (n > 1) fp[n - 1] = (f[n - 1] - fp[n - 2] * c[n - 1]) / (a[n - 1] - bp[n - 2] * c[n - 1]);
    u[n - 1] = fp[n - 1];
    for (int i = n - 2; i >= 0; --i) u[i] = fp[i] - bp[i] * u[i + 1];
    free(bp);
    free(fp);
}

/* The same algorithm for a diagonally dominant M-matrix given as
 * a_i = delta_i + up_i + lo_i, b_i = -up_i, c_i = -lo_i (delta, up, lo >= 0).
 * The denominator a_i - b'_{i-1} c_i is formed as eps_i + up_i where
 * eps_i = delta_i + lo_i * eps_{i-1} / m_{i-1} is the part of the pivot in
 * excess of the coupling to the next row; algebraically identical, but free
 * of the cancellation that the plain form suffers when delta << up + lo. */
void og_thomas_excess(int n, const double *delta, const double *up, const double *lo,
                      const double *f, double *u)
{
    double *m = (double *)malloc(n * sizeof(double));
    double *fp = (double *)malloc(n * sizeof(double));
    double eps_prev = 0.0, m_prev = 1.0, fp_prev = 0.0;
    for (int i = 0; i < n; ++i) {
        double lo_i = (i > 0) ? lo[i] : 0.0;
        double up_i = (i < n - 1) ? up[i] : 0.0;
        double eps = delta[i] + lo_i * (eps_prev / m_prev);
        m[i] = eps + up_i;
        fp[i] = (f[i] + lo_i * fp_prev) / m[i];
        eps_prev = eps;
        m_prev = m[i];
        fp_prev = fp[i];
    }
    u[n - 1] = fp[n - 1];
    for (int i = n - 2; i >= 0; --i) u[i] = fp[i] + (up[i] / m[i]) * u[i + 1];
    free(m);
    free(fp);
}

/* ------------------------------------------------------------------------ */
/* Block (vertical line) relaxation, Sec. 4.2: Dtilde_P is the tridiagonal    */
/* block of A coupling the cells of column P (the full diagonal and the       */
/* vertical off-diagonals).  One damped block-Jacobi sweep is                 */
/*   u <- u + rho Dtilde^{-1} (b - A u).                                      */
/* ------------------------------------------------------------------------ */
static void og_column_solve(const og_grid *g, const og_level *L, long c, const double *rhs, double *x)
{
    int nz = g->nz;
    double *delta = (double *)malloc(nz * sizeof(double));
    double *up = (double *)malloc(nz * sizeof(double));
    double *lo = (double *)malloc(nz * sizeof(double));
    double sumT = 0.0;
    for (int q = 0; q < 4; ++q) sumT += L->ell[4 * c + q] / L->dist[4 * c + q];
    double wl2 = g->omega2 * g->lambda2;
    for (int k = 0; k < nz; ++k) {
        delta[k] = L->area[c] * g->V[k] + g->omega2 * g->V[k] * sumT;
        up[k] = wl2 * L->area[c] * g->G[k + 1];
        lo[k] = wl2 * L->area[c] * g->G[k];
    }
    og_thomas_excess(nz, delta, up, lo, rhs, x);
    free(delta);
    free(up);
    free(lo);
}

/* ------------------------------------------------------------------------ */
/* Block red-black SOR (Sec. 4.2, Eq. BlockRBSOR): a column is red when the   */
/* sum i + j of its horizontal indices is even and black otherwise (Sec.      */
/* 6.2.1).  One sweep updates the red columns, then the black ones:           */
/*   u_c <- u_c + rho Dtilde_c^{-1} (b - A u)_c   for every column c of the   */
/* colour, the residual taken with the current iterate.  On the periodic box  */
/* (n even) no two columns of one colour are neighbours.  On the cubed sphere */
/* that cannot hold everywhere (three cells meet pairwise at a cube corner):  */
/* columns of one colour are updated together, so a same-colour neighbour     */
/* enters with its value from before the half-sweep.                          */
/* ------------------------------------------------------------------------ */
static int og_colour(const og_level *L, long c)
{
    long n = L->n;
    return (int)(((c % n) + (c / n) % n) & 1);
}

static void og_half_sweep(const og_grid *g, int lev, const double *b, double *u, int colour,
                          double rho)
{
    const og_level *L = &g->lev[lev];
    long nc = L->ncol, N = nc * g->nz;
    int nz = g->nz;
    double *r = (double *)malloc(N * sizeof(double));
    double *col_r = (double *)malloc(nz * sizeof(double));
    double *col_e = (double *)malloc(nz * sizeof(double));
    og_residual(g, lev, b, u, r);
    for (long c = 0; c < nc; ++c) {
        if (og_colour(L, c) != colour) continue;
        for (int k = 0; k < nz; ++k) col_r[k] = r[k * nc + c];
        og_column_solve(g, L, c, col_r, col_e);
        for (int k = 0; k < nz; ++k) u[k * nc + c] += rho * col_e[k];
    }
    free(r);
    free(col_r);
    free(col_e);
}

void og_set_smoother(og_grid *g, int kind) { g->smoother = kind; }

/* Vertical background profiles (Sec. 2, Eq. FullSISLEquation and the vertical
 * operator D^(z) of the Appendix).  Multiplying the equation by the weight
 * p(r) r^2, p = (pi*)^gamma c_p theta*, keeps it symmetric: the mass and
 * horizontal terms of layer k take V_k = int p r^2 dr instead of int r^2 dr,
 * and the vertical flux through r_k takes p q r^2 / (rho_k - rho_{k-1}) with
 * q = 1 / (1 + (alpha dt)^2 (N*)^2).  The caller gives p_cell[k] = (int p r^2
 * dr) / (int r^2 dr) over layer k and q_face[k] = p(r_k) q(r_k) at the
 * interior interfaces k = 1..nz-1; both 1 give the model equation. */
void og_set_profiles(og_grid *g, const double *p_cell, const double *q_face)
{
    for (int k = 0; k < g->nz; ++k) g->V[k] *= p_cell[k];
    for (int k = 1; k < g->nz; ++k) g->G[k] *= q_face[k];
}

void og_set_precond(og_grid *g, int kind, double rho)
{
    g->precond = kind;
    g->precond_rho = rho;
}

void og_set_mg_precond(og_grid *g, int nu_pre, int nu_post, int nu_coarse, double rho,
                       int prolong_mode)
{
    g->mg_nu_pre = nu_pre;
    g->mg_nu_post = nu_post;
    g->mg_nu_coarse = nu_coarse;
    g->mg_rho = rho;
    g->mg_prolong = prolong_mode;
}

void og_set_fmg(og_grid *g, int on) { g->fmg = on ? 1 : 0; }

void og_smooth_rb(const og_grid *g, int lev, const double *b, double *u, int nsweeps, double rho)
{
    for (int s = 0; s < nsweeps; ++s) {
        og_half_sweep(g, lev, b, u, 0, rho);
        og_half_sweep(g, lev, b, u, 1, rho);
    }
}

/* Block red-black SSOR as the CG preconditioner (Sec. 7.2): z = M^{-1} r is
 * the result of a forward sweep (red, black) and a backward sweep (black,
 * red) of Au = r from u = 0.  Each half-sweep is symmetric in the A inner
 * product, so the sequence red, black, black, red gives a symmetric M. */
void og_rb_ssor(const og_grid *g, int lev, const double *r, double *z, double rho)
{
    long N = g->lev[lev].ncol * g->nz;
    memset(z, 0, N * sizeof(double));
    og_half_sweep(g, lev, r, z, 0, rho);
    og_half_sweep(g, lev, r, z, 1, rho);
    og_half_sweep(g, lev, r, z, 1, rho);
    og_half_sweep(g, lev, r, z, 0, rho);
}

void og_line_precond(const og_grid *g, int lev, const double *r, double *z);
/* z = M^{-1} r.  Kind 2 (Sec. 4.3: multigrid as a preconditioner for a
 * Krylov method) is one V-cycle of A z = r from z = 0 (Algorithm 1). */
void og_vcycle(const og_grid *g, const double *b, double *u, int nu_pre, int nu_post,
               int nu_coarse, double rho, double rho_coarse, int prolong_mode);
static void og_precond(const og_grid *g, const double *r, double *z)
{
    if (g->precond == 1) {
        og_rb_ssor(g, 0, r, z, g->precond_rho);
    } else if (g->precond == 2) {
        memset(z, 0, g->lev[0].ncol * g->nz * sizeof(double));
        if (g->fmg)
            og_fmg(g, r, z, g->mg_nu_pre, g->mg_nu_post, g->mg_nu_coarse, g->mg_rho, 1.0,
                   g->mg_prolong);
        else
            og_vcycle(g, r, z, g->mg_nu_pre, g->mg_nu_post, g->mg_nu_coarse, g->mg_rho, 1.0,
                      g->mg_prolong);
    } else {
        og_line_precond(g, 0, r, z);
    }
}

void og_smooth(const og_grid *g, int lev, const double *b, double *u, int nsweeps, double rho)
{
    if (g->smoother == 1) {
        og_smooth_rb(g, lev, b, u, nsweeps, rho);
        return;
    }
    const og_level *L = &g->lev[lev];
    long nc = L->ncol, N = nc * g->nz;
    int nz = g->nz;
    double *r = (double *)malloc(N * sizeof(double));
    double *col_r = (double *)malloc(nz * sizeof(double));
    double *col_e = (double *)malloc(nz * sizeof(double));
    for (int s = 0; s < nsweeps; ++s) {
        og_residual(g, lev, b, u, r); /* all columns use the old iterate */
        for (long c = 0; c < nc; ++c) {
            for (int k = 0; k < nz; ++k) col_r[k] = r[k * nc + c];
            og_column_solve(g, L, c, col_r, col_e);
            for (int k = 0; k < nz; ++k) u[k * nc + c] += rho * col_e[k];
        }
    }
    free(r);
    free(col_r);
    free(col_e);
}

void og_line_precond(const og_grid *g, int lev, const double *r, double *z)
{
    const og_level *L = &g->lev[lev];
    long nc = L->ncol;
    int nz = g->nz;
    double *col_r = (double *)malloc(nz * sizeof(double));
    double *col_e = (double *)malloc(nz * sizeof(double));
    for (long c = 0; c < nc; ++c) {
        for (int k = 0; k < nz; ++k) col_r[k] = r[k * nc + c];
        og_column_solve(g, L, c, col_r, col_e);
        for (int k = 0; k < nz; ++k) z[k * nc + c] = col_e[k];
    }
    free(col_r);
    free(col_e);
}

/* ------------------------------------------------------------------------ */
/* Intergrid transfers (Sec. 6.2.1): horizontal cell average for the          */
/* restriction -- in the volume-integrated form the coarse right-hand side    */
/* is the sum of the four children -- and linear interpolation for the        */
/* prolongation, with the vertical index unchanged.                           */
/* ------------------------------------------------------------------------ */
void og_restrict(const og_grid *g, int lev_f, const double *r_f, double *b_c)
{
    const og_level *F = &g->lev[lev_f], *C = &g->lev[lev_f + 1];
    int nf = F->n, nc = C->n;
    for (int k = 0; k < g->nz; ++k)
        for (int p = 0; p < g->P; ++p)
            for (int J = 0; J < nc; ++J)
                for (int I = 0; I < nc; ++I) {
                    double s = 0.0;
                    for (int b = 0; b < 2; ++b)
                        for (int a = 0; a < 2; ++a)
                            s += r_f[k * F->ncol + ((long)p * nf + 2 * J + b) * nf + 2 * I + a];
                    b_c[k * C->ncol + ((long)p * nc + J) * nc + I] = s;
                }
}

/* mode 0: cell-centred bilinear interpolation in index space, weights
 * 9/16, 3/16, 3/16, 1/16 from the parent, its two neighbours towards the
 * child and the cell diagonally across the shared corner.  Where that corner
 * is a corner of the cube only three cells meet; the missing diagonal value
 * is replaced by the linear extrapolation u_x + u_y - u_parent, which gives
 * weights 1/2, 1/4, 1/4.  mode 1: piecewise constant. */
void og_prolong_add(const og_grid *g, int lev_f, const double *u_c, double *u_f, int mode)
{
    const og_level *F = &g->lev[lev_f], *C = &g->lev[lev_f + 1];
    int nf = F->n, ncn = C->n;
    for (int p = 0; p < g->P; ++p)
        for (int j = 0; j < nf; ++j)
            for (int i = 0; i < nf; ++i) {
                long fc = ((long)p * nf + j) * nf + i;
                long pc = ((long)p * ncn + j / 2) * ncn + i / 2;
                int qx = (i % 2) ? 1 : 0, qy = (j % 2) ? 3 : 2;
                long X = C->nbr[4 * pc + qx], Y = C->nbr[4 * pc + qy], D = -1;
                long panel_sz = (long)ncn * ncn;
                if (X / panel_sz == p) D = C->nbr[4 * X + qy];
                else if (Y / panel_sz == p) D = C->nbr[4 * Y + qx];
                for (int k = 0; k < g->nz; ++k) {
                    const double *uc = u_c + k * C->ncol;
                    double e;
                    if (mode == 1) e = uc[pc];
                    else if (D >= 0) e = (9.0 * uc[pc] + 3.0 * uc[X] + 3.0 * uc[Y] + uc[D]) / 16.0;
                    else e = (2.0 * uc[pc] + uc[X] + uc[Y]) / 4.0;
                    u_f[k * F->ncol + fc] += e;
                }
            }
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 (multigrid V-cycle).  Level 0 is the finest grid here (the   */
/* paper numbers the finest level L and the coarsest 1).  On the coarsest    */
/* level the exact solve is replaced by nu_coarse relaxation sweeps.         */
/* ------------------------------------------------------------------------ */
static void og_vcycle_level(const og_grid *g, int lev, const double *b, double *u, int nu_pre,
                            int nu_post, int nu_coarse, double rho, double rho_coarse, int mode)
{
    if (lev == g->nlev - 1) {
        og_smooth(g, lev, b, u, nu_coarse, rho_coarse);
        return;
    }
    long N = g->lev[lev].ncol * g->nz, Nc = g->lev[lev + 1].ncol * g->nz;
    double *r = (double *)malloc(N * sizeof(double));
    double *bc = (double *)malloc(Nc * sizeof(double));
    double *uc = (double *)calloc(Nc, sizeof(double));
    og_smooth(g, lev, b, u, nu_pre, rho);
    og_residual(g, lev, b, u, r);
    og_restrict(g, lev, r, bc);
    og_vcycle_level(g, lev + 1, bc, uc, nu_pre, nu_post, nu_coarse, rho, rho_coarse, mode);
    og_prolong_add(g, lev, uc, u, mode);
    og_smooth(g, lev, b, u, nu_post, rho);
    free(r);
    free(bc);
    free(uc);
}

void og_vcycle(const og_grid *g, const double *b, double *u, int nu_pre, int nu_post,
               int nu_coarse, double rho, double rho_coarse, int prolong_mode)
{
    og_vcycle_level(g, 0, b, u, nu_pre, nu_post, nu_coarse, rho, rho_coarse, prolong_mode);
}

/* Full multigrid (Sec. 4.3): the right-hand side restricted to every level
 * (cell averages in volume-integrated form: sums of the children), nu_coarse
 * sweeps on the coarsest level from zero, then on each finer level the
 * coarse solution prolongated as the start of one V-cycle of that level. */
void og_fmg(const og_grid *g, const double *b, double *u, int nu_pre, int nu_post, int nu_coarse,
            double rho, double rho_coarse, int prolong_mode)
{
    int L = g->nlev;
    double *bl[MAXLEV], *ul[MAXLEV];
    for (int l = 0; l < L; ++l) {
        long N = g->lev[l].ncol * g->nz;
        bl[l] = l == 0 ? (double *)b : (double *)malloc(N * sizeof(double));
        ul[l] = l == 0 ? u : (double *)malloc(N * sizeof(double));
        memset(ul[l], 0, N * sizeof(double));
    }
    for (int l = 0; l + 1 < L; ++l) og_restrict(g, l, bl[l], bl[l + 1]);
    og_smooth(g, L - 1, bl[L - 1], ul[L - 1], nu_coarse, rho_coarse);
    for (int l = L - 2; l >= 0; --l) {
        og_prolong_add(g, l, ul[l + 1], ul[l], prolong_mode);  /* onto zero: interpolation */
        og_vcycle_level(g, l, bl[l], ul[l], nu_pre, nu_post, nu_coarse, rho, rho_coarse,
                        prolong_mode);
    }
    for (int l = 1; l < L; ++l) {
        free(bl[l]);
        free(ul[l]);
    }
}

static double og_norm(const double *x, long N)
{
    double s = 0.0;
    for (long m = 0; m < N; ++m) s += x[m] * x[m];
    return sqrt(s);
}

static double og_dot(const double *x, const double *y, long N)
{
    double s = 0.0;
    for (long m = 0; m < N; ++m) s += x[m] * y[m];
    return s;
}

int og_mg_solve(const og_grid *g, const double *b, double *u, double rtol, int maxit,
                int nu_pre, int nu_post, int nu_coarse, double rho, double rho_coarse,
                int prolong_mode, double *hist)
{
    long N = g->lev[0].ncol * g->nz;
    double *r = (double *)malloc(N * sizeof(double));
    memset(u, 0, N * sizeof(double));
    double r0 = og_norm(b, N);
    if (hist) hist[0] = 1.0;
    int it = 0;
    if (r0 == 0.0) { free(r); return 0; }
    while (it < maxit) {
        if (it == 0 && g->fmg)  /* the first cycle starts from zero */
            og_fmg(g, b, u, nu_pre, nu_post, nu_coarse, rho, rho_coarse, prolong_mode);
        else
            og_vcycle(g, b, u, nu_pre, nu_post, nu_coarse, rho, rho_coarse, prolong_mode);
        ++it;
        og_residual(g, 0, b, u, r);
        double rel = og_norm(r, N) / r0;
        if (hist) hist[it] = rel;
        if (rel <= rtol) break;
    }
    free(r);
    return it;
}

/* Algorithm PCG with M = Dtilde (block Jacobi over vertical columns), the
 * block red-black SSOR preconditioner or one V-cycle (og_set_precond). */
int og_pcg_solve(const og_grid *g, const double *b, double *u, double rtol, int maxit, double *hist)
{
    long N = g->lev[0].ncol * g->nz;
    double *r = (double *)malloc(N * sizeof(double));
    double *z = (double *)malloc(N * sizeof(double));
    double *p = (double *)malloc(N * sizeof(double));
    double *q = (double *)malloc(N * sizeof(double));
    memset(u, 0, N * sizeof(double));
    og_residual(g, 0, b, u, r);
    og_precond(g, r, z);
    memcpy(p, z, N * sizeof(double));
    double kappa_old = og_dot(r, z, N);
    double r0 = og_norm(r, N);
    if (hist) hist[0] = 1.0;
    int K = 0;
    if (r0 > 0.0) {
        for (K = 1; K <= maxit; ++K) {
            og_apply(g, 0, p, q);
            double alpha = kappa_old / og_dot(p, q, N);
            for (long m = 0; m < N; ++m) {
                u[m] += alpha * p[m];
                r[m] -= alpha * q[m];
            }
            double rel = og_norm(r, N) / r0;
            if (hist) hist[K] = rel;
            if (rel < rtol) break;
            /* the V-cycle preconditioner is not symmetric (bilinear
             * prolongation against the 2x2 sum), so its beta is the flexible
             * (Polak-Ribiere) one, <r_K, z_K - z_{K-1}> / <r_{K-1}, z_{K-1}>,
             * which equals the standard one for a symmetric M */
            double cross = g->precond == 2 ? og_dot(r, z, N) : 0.0;
            og_precond(g, r, z);
            double kappa = og_dot(r, z, N);
            double beta = (kappa - cross) / kappa_old;
            for (long m = 0; m < N; ++m) p[m] = z[m] + beta * p[m];
            kappa_old = kappa;
        }
        if (K > maxit) K = maxit;
    }
    free(r);
    free(z);
    free(p);
    free(q);
    return K;
}
