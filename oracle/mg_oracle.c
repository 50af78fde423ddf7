/*
 * mg_oracle.c -- plain, slow, FP64 CPU multigrid for the pressure equation
 *   div( (1/rho) grad p ) = S                                   (Eq. 9)
 * of Shin, Chergui & Juric, "A solver for massively parallel direct numerical
 * simulation of three-dimensional multiphase flows" (arXiv 1410.8568), Sec. 2.3.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness oracle of the CUDA
 * library in paper_1410_8568_gb300/.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or helper with the CUDA path.
 *
 * What it computes.  The method's result is the unique zero-mean solution p* of
 * the cell-centred finite-difference system of Eq. 10 (with the face
 * coefficients of Eqs. 11-12 built by the caller or by oracle_faces_from_density),
 * for a right-hand side projected to zero sum.  Multigrid is only the route to
 * p*.  The route here follows the paper's list of features (Sec. 2.3):
 *   (1) cell-centred second-order differences of Eq. 9  -> oracle_apply
 *   (2) harmonic face coefficient (Eqs. 11-12)          -> oracle_faces_from_density
 *   (3) restriction of the residual                      -> oracle_restrict (8-child mean)
 *   (4) prolongation of the coarse error                 -> oracle_prolong_add (trilinear),
 *       or by cell flux conservation (Eqs. 13-14)       -> oracle_prolong_flux_add
 *   (5) red-black relaxation                             -> oracle_smooth_colour
 *   (6) exact solve of the error on the coarsest grid    -> oracle_coarse_solve (dense LU)
 * and the stopping test and average reduction rate of Eq. 15.
 * Around the solve, the projection step of the Navier-Stokes module (Sec. 2.2:
 * Chorin's projection on the staggered MAC grid, S a function of the
 * non-projected velocity) -> oracle_divergence (S = D u* / dt) and
 * oracle_project (u = u* - dt alpha G p).
 *
 * Readings where the paper is silent (each one also listed in the design notes):
 *  - the restriction of the residual (3), for which the paper names a linear
 *    interpolation but gives no formula, is read as the mean of the 8 fine
 *    children of a coarse cell;
 *  - the coarse face coefficient is the mean of the 4 fine face coefficients
 *    that tile the coarse face (flux through a coarse face = sum of fine fluxes);
 *  - prolongation (4) uses trilinear weights 3/4, 1/4 per axis; at a Neumann
 *    wall the missing coarse neighbour is replaced by the edge cell, at a
 *    periodic boundary it wraps;
 *  - SOR relaxation factor omega is a parameter (1 = Gauss-Seidel); red cells
 *    are those with (i+j+k) even and are relaxed first;
 *  - the coarsest-grid solve (GMRES in the paper, (6)) is an exact dense solve
 *    of the bordered system [-A 1; 1^T 0][e; l] = [-r; 0] on coarsest grids of
 *    at most 512 cells; larger coarsest grids (sizes with a large odd factor)
 *    are solved by restarted GMRES (oracle_gmres) to a relative residual of
 *    1e-13, the solution projected to zero mean;
 *  - coarsening of all three axes continues while every axis is even and > 4;
 *  - flux-conserving prolongation (4), Eqs. 13-14: Eq. 13 as printed does not
 *    give a convex weighting; it is read as continuity of the flux alpha de/dx
 *    across the coarse face between cells L and R, which gives the face value
 *    e_f = (alpha_L e_L + alpha_R e_R) / (alpha_L + alpha_R).  The values at
 *    the edges and nodes (the "analogous expressions" the paper mentions for
 *    3D) are the alpha-weighted means of the 4 and 8 coarse cells that meet
 *    there.  A fine cell occupies one octant of its coarse cell; its value is
 *    the mean of the 8 corner values of that octant (coarse centre, 3 face
 *    centres, 3 edge midpoints, the node), i.e. trilinear interpolation at the
 *    octant's centre.  The cell coefficient alpha_c of a coarse cell, which the
 *    paper does not define, is the mean of the coefficients of its faces that
 *    are not walls.  Walls mirror (the partner is the cell itself), periodic
 *    axes wrap.  For a constant alpha this is exactly the trilinear rule.
 *
 * Layout (the library's documented layout, shared as an interface only):
 * cell (i,j,k) of an nx*ny*nz grid is element i + nx*(j + ny*k).  Face array
 * a[d] holds, for each cell, the coefficient alpha = 1/rho of its LOW face along
 * axis d (between cell c - e_d and c).  At a Neumann wall the low face of the
 * first cell is the wall and its entry is ignored (zero flux); the high face of
 * the last cell is the other wall.  On a periodic axis the low face of the first
 * cell is the face shared with the last cell.
 *
 * Operator (Eq. 10 divided by h^2, per axis spacing h_d):
 *   (A p)_c = sum_d sum_{side} alpha_f / h_d^2 * (p_nb - p_c).
 * A is symmetric negative semidefinite with A 1 = 0.
 *
 * Loops over z-planes are split across OpenMP threads only where the updates
 * are independent (every result is the same for any thread count); all sums are
 * taken plane by plane and then over planes in a fixed order.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OG_NEUMANN 0
#define OG_PERIODIC 1

typedef struct {
    int n[3];    /* cells per axis */
    double h[3]; /* cell size per axis */
    int bc[3];   /* OG_NEUMANN or OG_PERIODIC */
} og_grid;

static long cell_count(const og_grid *g) { return (long)g->n[0] * g->n[1] * g->n[2]; }

static long cell_index(const og_grid *g, int i, int j, int k)
{
    return i + (long)g->n[0] * (j + (long)g->n[1] * k);
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the following calls (n >= 1); returns the number in effect. */
int oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* Coefficient of the face of cell (i,j,k) on side `side` (-1 low, +1 high) of
 * axis d, and the index of the cell across that face.  Returns 0 for a wall. */
static double face_coef(const og_grid *g, const double *const a[3], int i, int j, int k,
                        int d, int side, long *nb)
{
    int c[3] = {i, j, k};
    int n = g->n[d];
    int m = c[d] + side;        /* neighbour coordinate along d */
    int f = side < 0 ? c[d] : c[d] + 1; /* face = low face of the cell at coordinate f */
    if (m < 0 || m >= n) {
        if (g->bc[d] == OG_NEUMANN) {
            *nb = -1;
            return 0.0;
        }
        m = (m + n) % n;
    }
    if (f == n) f = 0; /* periodic: high face of the last cell is the low face of the first */
    if (f == 0 && g->bc[d] == OG_NEUMANN) { /* cannot happen for interior faces; kept explicit */
        *nb = -1;
        return 0.0;
    }
    int q[3] = {i, j, k};
    q[d] = f;
    double alpha = a[d][cell_index(g, q[0], q[1], q[2])];
    int r[3] = {i, j, k};
    r[d] = m;
    *nb = cell_index(g, r[0], r[1], r[2]);
    return alpha;
}

/* ------------------------------------------------------------------------ */
/* (2) Harmonic face coefficient, Eqs. 11-12                                 */
/* ------------------------------------------------------------------------ */

/* alpha = 1/rho at cell centres; the face value between cells L and R is
 *   harmonic (mode 0, Eqs. 11-12): 2 alpha_L alpha_R / (alpha_L + alpha_R)
 *   arithmetic (mode 1):            (alpha_L + alpha_R) / 2
 * Neumann wall entries are written as 0. */
int oracle_faces_from_density(const og_grid *g, const double *rho, int mode,
                              double *ax, double *ay, double *az)
{
    double *a[3] = {ax, ay, az};
    for (int k = 0; k < g->n[2]; k++)
        for (int j = 0; j < g->n[1]; j++)
            for (int i = 0; i < g->n[0]; i++) {
                long c = cell_index(g, i, j, k);
                int q[3] = {i, j, k};
                for (int d = 0; d < 3; d++) {
                    if (q[d] == 0 && g->bc[d] == OG_NEUMANN) {
                        a[d][c] = 0.0;
                        continue;
                    }
                    int l[3] = {i, j, k};
                    l[d] = (q[d] - 1 + g->n[d]) % g->n[d];
                    double alpha_l = 1.0 / rho[cell_index(g, l[0], l[1], l[2])];
                    double alpha_r = 1.0 / rho[c];
                    if (mode == 0)
                        a[d][c] = 2.0 * alpha_l * alpha_r / (alpha_l + alpha_r);
                    else
                        a[d][c] = 0.5 * (alpha_l + alpha_r);
                }
            }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* (1) Cell-centred operator of Eq. 10                                       */
/* ------------------------------------------------------------------------ */

static double apply_at(const og_grid *g, const double *const a[3], const double *p,
                       int i, int j, int k)
{
    long c = cell_index(g, i, j, k);
    double s = 0.0;
    for (int d = 0; d < 3; d++)
        for (int side = -1; side <= 1; side += 2) {
            long nb;
            double alpha = face_coef(g, a, i, j, k, d, side, &nb);
            if (nb < 0) continue;
            s += alpha / (g->h[d] * g->h[d]) * (p[nb] - p[c]);
        }
    return s;
}

void oracle_apply(const og_grid *g, const double *ax, const double *ay, const double *az,
                  const double *p, double *out)
{
    const double *a[3] = {ax, ay, az};
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->n[2]; k++)
        for (int j = 0; j < g->n[1]; j++)
            for (int i = 0; i < g->n[0]; i++)
                out[cell_index(g, i, j, k)] = apply_at(g, a, p, i, j, k);
}

/* r = b - A p */
void oracle_residual(const og_grid *g, const double *ax, const double *ay, const double *az,
                     const double *b, const double *p, double *r)
{
    const double *a[3] = {ax, ay, az};
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->n[2]; k++)
        for (int j = 0; j < g->n[1]; j++)
            for (int i = 0; i < g->n[0]; i++) {
                long c = cell_index(g, i, j, k);
                r[c] = b[c] - apply_at(g, a, p, i, j, k);
            }
}

/* Sums over the grid, plane by plane then over planes, in a fixed order. */
static double grid_sum(const og_grid *g, const double *x, int squares)
{
    int nz = g->n[2];
    long plane = (long)g->n[0] * g->n[1];
    double *part = (double *)malloc(sizeof(double) * (size_t)nz);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++) {
        double s = 0.0;
        const double *xp = x + plane * k;
        for (long t = 0; t < plane; t++) s += squares ? xp[t] * xp[t] : xp[t];
        part[k] = s;
    }
    double s = 0.0;
    for (int k = 0; k < nz; k++) s += part[k];
    free(part);
    return s;
}

double oracle_norm2(const og_grid *g, const double *x) { return sqrt(grid_sum(g, x, 1)); }

double oracle_mean(const og_grid *g, const double *x) { return grid_sum(g, x, 0) / (double)cell_count(g); }

static void subtract_constant(const og_grid *g, double *x, double c)
{
    long n = cell_count(g);
    for (long t = 0; t < n; t++) x[t] -= c;
}

/* ------------------------------------------------------------------------ */
/* (5) Red-black SOR relaxation                                              */
/* ------------------------------------------------------------------------ */

/* One half-sweep over the cells of one colour ((i+j+k) % 2 == colour):
 * each such cell is set so that its own equation (A p)_c = b_c holds given its
 * neighbours (all of the other colour), then relaxed by omega. */
void oracle_smooth_colour(const og_grid *g, const double *ax, const double *ay, const double *az,
                          const double *b, double *p, int colour, double omega)
{
    const double *a[3] = {ax, ay, az};
    /* Cells of one colour only touch cells of the other colour unless a
     * periodic axis has an odd length; then the sweep runs in plain order. */
    int independent = 1;
    for (int d = 0; d < 3; d++)
        if (g->bc[d] == OG_PERIODIC && g->n[d] % 2 == 1 && g->n[d] > 1) independent = 0;
#pragma omp parallel for schedule(static) if (independent)
    for (int k = 0; k < g->n[2]; k++)
        for (int j = 0; j < g->n[1]; j++)
            for (int i = 0; i < g->n[0]; i++) {
                if (((i + j + k) & 1) != colour) continue;
                long c = cell_index(g, i, j, k);
                double diag = 0.0, off = 0.0;
                for (int d = 0; d < 3; d++)
                    for (int side = -1; side <= 1; side += 2) {
                        long nb;
                        double alpha = face_coef(g, a, i, j, k, d, side, &nb);
                        if (nb < 0 || nb == c) continue;
                        double w = alpha / (g->h[d] * g->h[d]);
                        diag += w;
                        off += w * p[nb];
                    }
                if (diag <= 0.0) continue;
                double gs = (off - b[c]) / diag;
                p[c] = (1.0 - omega) * p[c] + omega * gs;
            }
}

/* ------------------------------------------------------------------------ */
/* Coarse grid, coarse coefficients, (3) restriction, (4) prolongation        */
/* ------------------------------------------------------------------------ */

int oracle_can_coarsen(const og_grid *g)
{
    for (int d = 0; d < 3; d++)
        if (g->n[d] % 2 != 0 || g->n[d] <= 4) return 0;
    return 1;
}

void oracle_coarse_grid(const og_grid *g, og_grid *gc)
{
    for (int d = 0; d < 3; d++) {
        gc->n[d] = g->n[d] / 2;
        gc->h[d] = 2.0 * g->h[d];
        gc->bc[d] = g->bc[d];
    }
}

/* Coarse face = mean of the 4 fine faces that tile it.  The low face of coarse
 * cell (I,J,K) along x is tiled by the low faces of fine cells
 * (2I, 2J+b, 2K+c), b, c in {0,1}; likewise for y and z. */
void oracle_coarsen_faces(const og_grid *g, const double *ax, const double *ay, const double *az,
                          double *cx, double *cy, double *cz)
{
    og_grid gc;
    oracle_coarse_grid(g, &gc);
    const double *a[3] = {ax, ay, az};
    double *ca[3] = {cx, cy, cz};
    for (int K = 0; K < gc.n[2]; K++)
        for (int J = 0; J < gc.n[1]; J++)
            for (int I = 0; I < gc.n[0]; I++) {
                long C = cell_index(&gc, I, J, K);
                for (int d = 0; d < 3; d++) {
                    double s = 0.0;
                    for (int u = 0; u < 2; u++)
                        for (int v = 0; v < 2; v++) {
                            int f[3];
                            int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
                            int base[3] = {2 * I, 2 * J, 2 * K};
                            f[d] = base[d];
                            f[e1] = base[e1] + u;
                            f[e2] = base[e2] + v;
                            s += a[d][cell_index(g, f[0], f[1], f[2])];
                        }
                    ca[d][C] = 0.25 * s;
                }
            }
}

/* b_c(I,J,K) = (1/8) sum of r over the 8 fine children */
void oracle_restrict(const og_grid *g, const double *r, double *bc)
{
    og_grid gc;
    oracle_coarse_grid(g, &gc);
#pragma omp parallel for schedule(static)
    for (int K = 0; K < gc.n[2]; K++)
        for (int J = 0; J < gc.n[1]; J++)
            for (int I = 0; I < gc.n[0]; I++) {
                double s = 0.0;
                for (int c = 0; c < 2; c++)
                    for (int b = 0; b < 2; b++)
                        for (int a = 0; a < 2; a++)
                            s += r[cell_index(g, 2 * I + a, 2 * J + b, 2 * K + c)];
                bc[cell_index(&gc, I, J, K)] = s / 8.0;
            }
}

/* Neighbouring coarse coordinate used by fine coordinate i (the second of the
 * two coarse cells whose centres bracket the fine centre). */
static int prolong_partner(int i, int nc, int bc)
{
    int I = i / 2;
    int J = (i % 2 == 0) ? I - 1 : I + 1;
    if (J < 0 || J >= nc) {
        if (bc == OG_NEUMANN) return I; /* mirror: ghost takes the edge value */
        J = (J + nc) % nc;
    }
    return J;
}

/* x_fine += trilinear interpolation of the coarse error e (weights 3/4 on the
 * coarse cell containing the fine centre, 1/4 on the partner, per axis). */
void oracle_prolong_add(const og_grid *g, const double *e, double *x)
{
    og_grid gc;
    oracle_coarse_grid(g, &gc);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->n[2]; k++)
        for (int j = 0; j < g->n[1]; j++)
            for (int i = 0; i < g->n[0]; i++) {
                int I[2] = {i / 2, prolong_partner(i, gc.n[0], g->bc[0])};
                int J[2] = {j / 2, prolong_partner(j, gc.n[1], g->bc[1])};
                int K[2] = {k / 2, prolong_partner(k, gc.n[2], g->bc[2])};
                const double w[2] = {0.75, 0.25};
                double s = 0.0;
                for (int c = 0; c < 2; c++)
                    for (int b = 0; b < 2; b++)
                        for (int a = 0; a < 2; a++)
                            s += w[a] * w[b] * w[c] * e[cell_index(&gc, I[a], J[b], K[c])];
                x[cell_index(g, i, j, k)] += s;
            }
}

/* Cell coefficient used by the flux-conserving prolongation: the mean of the
 * alpha of the cell's faces that are not walls (1 for a cell with none). */
void oracle_cell_alpha(const og_grid *g, const double *ax, const double *ay, const double *az,
                       double *out)
{
    const double *a[3] = {ax, ay, az};
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->n[2]; k++)
        for (int j = 0; j < g->n[1]; j++)
            for (int i = 0; i < g->n[0]; i++) {
                double s = 0.0;
                int m = 0;
                for (int d = 0; d < 3; d++)
                    for (int side = -1; side <= 1; side += 2) {
                        long nb;
                        double alpha = face_coef(g, a, i, j, k, d, side, &nb);
                        if (nb < 0) continue; /* wall */
                        s += alpha;
                        m++;
                    }
                out[cell_index(g, i, j, k)] = m ? s / m : 1.0;
            }
}

/* x_fine += flux-conserving interpolation of the coarse error e (Eqs. 13-14,
 * read as above).  ac = cell coefficients of the coarse grid.  For a fine cell,
 * the 8 coarse cells of its octant's corners are C (the coarse cell holding
 * it) shifted by its partner along any subset S of the axes; the corner value
 * of S is the alpha-weighted mean of the 2^|S| cells obtained from C by
 * shifting along any subset of S. */
void oracle_prolong_flux_add(const og_grid *g, const double *ac, const double *e, double *x)
{
    og_grid gc;
    oracle_coarse_grid(g, &gc);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->n[2]; k++)
        for (int j = 0; j < g->n[1]; j++)
            for (int i = 0; i < g->n[0]; i++) {
                int I[2] = {i / 2, prolong_partner(i, gc.n[0], g->bc[0])};
                int J[2] = {j / 2, prolong_partner(j, gc.n[1], g->bc[1])};
                int K[2] = {k / 2, prolong_partner(k, gc.n[2], g->bc[2])};
                double sum = 0.0;
                for (int S = 0; S < 8; S++) { /* corner: bit 0 x, bit 1 y, bit 2 z */
                    double num = 0.0, den = 0.0;
                    for (int T = 0; T < 8; T++) {
                        if ((T & S) != T) continue; /* shifts only along the axes of S */
                        long c = cell_index(&gc, I[T & 1], J[(T >> 1) & 1], K[(T >> 2) & 1]);
                        num += ac[c] * e[c];
                        den += ac[c];
                    }
                    sum += num / den;
                }
                x[cell_index(g, i, j, k)] += sum / 8.0;
            }
}

/* ------------------------------------------------------------------------ */
/* Projection step around the solve (Sec. 2.2, MAC grid)                     */
/* ------------------------------------------------------------------------ */

/* Face velocities use the face layout: u[d][c] is the normal velocity on the
 * LOW face of cell c along d; on a Neumann axis the low face of the first cell
 * is a wall (its entry is ignored: zero normal velocity) and the high wall of
 * the last cell carries none.  Divergence at the cell centre (second-order
 * centred differences, Sec. 2.2), divided by dt:
 *   S_c = sum_d (u_d(high face) - u_d(low face)) / h_d / dt. */
void oracle_divergence(const og_grid *g, const double *ux, const double *uy, const double *uz,
                       double dt, double *S)
{
    const double *u[3] = {ux, uy, uz};
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->n[2]; k++)
        for (int j = 0; j < g->n[1]; j++)
            for (int i = 0; i < g->n[0]; i++) {
                int q[3] = {i, j, k};
                double div = 0.0;
                for (int d = 0; d < 3; d++) {
                    int n = g->n[d];
                    double lo = (q[d] == 0 && g->bc[d] == OG_NEUMANN) ? 0.0 : u[d][cell_index(g, i, j, k)];
                    double hi;
                    if (q[d] + 1 < n) {
                        int r[3] = {i, j, k};
                        r[d] = q[d] + 1;
                        hi = u[d][cell_index(g, r[0], r[1], r[2])];
                    } else if (g->bc[d] == OG_PERIODIC) {
                        int r[3] = {i, j, k};
                        r[d] = 0;
                        hi = u[d][cell_index(g, r[0], r[1], r[2])];
                    } else {
                        hi = 0.0; /* wall */
                    }
                    div += (hi - lo) / g->h[d];
                }
                S[cell_index(g, i, j, k)] = div / dt;
            }
}

/* u_f -= dt alpha_f (p_c - p_{c-1}) / h_d on every face that is not a wall
 * (the face between the cell and its low neighbour along d; periodic: the low
 * face of the first cell joins it to the last).  With the operator of Eq. 10,
 * D(alpha G p) = A p, so the projected field satisfies D u = dt (S - A p). */
void oracle_project(const og_grid *g, const double *ax, const double *ay, const double *az,
                    const double *p, double dt, double *ux, double *uy, double *uz)
{
    const double *a[3] = {ax, ay, az};
    double *u[3] = {ux, uy, uz};
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->n[2]; k++)
        for (int j = 0; j < g->n[1]; j++)
            for (int i = 0; i < g->n[0]; i++) {
                int q[3] = {i, j, k};
                long c = cell_index(g, i, j, k);
                for (int d = 0; d < 3; d++) {
                    int r[3] = {i, j, k};
                    if (q[d] > 0) r[d] = q[d] - 1;
                    else if (g->bc[d] == OG_PERIODIC) r[d] = g->n[d] - 1;
                    else continue; /* wall face */
                    long m = cell_index(g, r[0], r[1], r[2]);
                    u[d][c] -= dt * a[d][c] * (p[c] - p[m]) / g->h[d];
                }
            }
}

/* ------------------------------------------------------------------------ */
/* (6) Exact solve on the coarsest grid                                      */
/* ------------------------------------------------------------------------ */

/* Solve A e = r with sum(e) = 0 through the bordered system
 *   [-A 1; 1^T 0] [e; l] = [-r; 0]
 * by Gaussian elimination with partial pivoting.  Returns 0, or -1 if the
 * system is singular (a grid split by zero coefficients). */
int oracle_coarse_solve(const og_grid *g, const double *ax, const double *ay, const double *az,
                        const double *r, double *e)
{
    const double *a[3] = {ax, ay, az};
    long n = cell_count(g);
    long m = n + 1;
    double *M = (double *)calloc((size_t)(m * m), sizeof(double));
    double *y = (double *)calloc((size_t)m, sizeof(double));
    if (!M || !y) { free(M); free(y); return -2; }
    for (int k = 0; k < g->n[2]; k++)
        for (int j = 0; j < g->n[1]; j++)
            for (int i = 0; i < g->n[0]; i++) {
                long c = cell_index(g, i, j, k);
                for (int d = 0; d < 3; d++)
                    for (int side = -1; side <= 1; side += 2) {
                        long nb;
                        double alpha = face_coef(g, a, i, j, k, d, side, &nb);
                        if (nb < 0) continue;
                        double w = alpha / (g->h[d] * g->h[d]);
                        M[c * m + c] += w;   /* row c of -A */
                        M[c * m + nb] -= w;
                    }
                M[c * m + n] = 1.0;
                M[n * m + c] = 1.0;
                y[c] = -r[c];
            }
    y[n] = 0.0;
    int status = 0;
    for (long col = 0; col < m; col++) {
        long piv = col;
        double best = fabs(M[col * m + col]);
        for (long row = col + 1; row < m; row++)
            if (fabs(M[row * m + col]) > best) { best = fabs(M[row * m + col]); piv = row; }
        if (best == 0.0) { status = -1; break; }
        if (piv != col) {
            for (long t = 0; t < m; t++) {
                double tmp = M[col * m + t];
                M[col * m + t] = M[piv * m + t];
                M[piv * m + t] = tmp;
            }
            double tmp = y[col]; y[col] = y[piv]; y[piv] = tmp;
        }
        for (long row = col + 1; row < m; row++) {
            double f = M[row * m + col] / M[col * m + col];
            if (f == 0.0) continue;
            for (long t = col; t < m; t++) M[row * m + t] -= f * M[col * m + t];
            y[row] -= f * y[col];
        }
    }
    if (status == 0) {
        for (long row = m - 1; row >= 0; row--) {
            double s = y[row];
            for (long t = row + 1; t < m; t++) s -= M[row * m + t] * y[t];
            y[row] = s / M[row * m + row];
        }
        memcpy(e, y, sizeof(double) * (size_t)n);
    }
    free(M);
    free(y);
    return status;
}

/* Restarted GMRES(m) (Saad & Schultz 1986) for A e = r - mean(r) on a grid
 * with walls or periodic axes (A singular, the system consistent): Arnoldi
 * with modified Gram-Schmidt, Givens rotations on the Hessenberg matrix, the
 * least-squares update at the end of each cycle or on convergence; e starts
 * at 0 and is returned with zero mean.  Stops when ||r - A e|| <= tol ||r||
 * (the recurrence's residual estimate) or after max_it Arnoldi steps.
 * Returns 0 converged, 1 not converged; *iters = Arnoldi steps. */
int oracle_gmres(const og_grid *g, const double *ax, const double *ay, const double *az,
                 const double *r_in, double *e, double tol, int max_it, int m, int *iters)
{
    long n = cell_count(g);
    size_t bytes = sizeof(double) * (size_t)n;
    double *b = (double *)malloc(bytes), *w = (double *)malloc(bytes), *res = (double *)malloc(bytes);
    double *V = (double *)malloc(bytes * (size_t)(m + 1));
    double *H = (double *)calloc((size_t)(m + 1) * m, sizeof(double)); /* H[i*m + j] */
    double *cs = (double *)malloc(sizeof(double) * m), *sn = (double *)malloc(sizeof(double) * m);
    double *gv = (double *)malloc(sizeof(double) * (m + 1)), *y = (double *)malloc(sizeof(double) * m);
    memcpy(b, r_in, bytes);
    subtract_constant(g, b, oracle_mean(g, b));
    memset(e, 0, bytes);
    double bnorm = oracle_norm2(g, b);
    int status = 1, it = 0;
    if (bnorm == 0.0) status = 0;
    while (status == 1 && it < max_it) {
        /* res = b - A e */
        oracle_residual(g, ax, ay, az, b, e, res);
        double beta = oracle_norm2(g, res);
        if (beta <= tol * bnorm) { status = 0; break; }
        for (long c = 0; c < n; c++) V[c] = res[c] / beta;
        for (int i = 0; i <= m; i++) gv[i] = 0.0;
        gv[0] = beta;
        int j = 0;
        for (; j < m && it < max_it; j++) {
            double *vj = V + (size_t)j * n, *vn = V + (size_t)(j + 1) * n;
            oracle_apply(g, ax, ay, az, vj, w);
            for (int i = 0; i <= j; i++) {
                const double *vi = V + (size_t)i * n;
                double h = 0.0;
                for (long c = 0; c < n; c++) h += w[c] * vi[c];
                H[i * m + j] = h;
                for (long c = 0; c < n; c++) w[c] -= h * vi[c];
            }
            double hn = oracle_norm2(g, w);
            H[(j + 1) * m + j] = hn;
            for (long c = 0; c < n; c++) vn[c] = hn > 0.0 ? w[c] / hn : 0.0;
            /* previous rotations, then a new one that zeroes H[j+1][j] */
            for (int i = 0; i < j; i++) {
                double a = H[i * m + j], bb = H[(i + 1) * m + j];
                H[i * m + j] = cs[i] * a + sn[i] * bb;
                H[(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
            }
            double a = H[j * m + j], bb = H[(j + 1) * m + j];
            double den = sqrt(a * a + bb * bb);
            cs[j] = den > 0.0 ? a / den : 1.0;
            sn[j] = den > 0.0 ? bb / den : 0.0;
            H[j * m + j] = den;
            H[(j + 1) * m + j] = 0.0;
            gv[j + 1] = -sn[j] * gv[j];
            gv[j] = cs[j] * gv[j];
            it++;
            if (fabs(gv[j + 1]) <= tol * bnorm || hn == 0.0) { j++; break; }
        }
        /* y = H(0:j, 0:j)^-1 g(0:j), e += V y */
        for (int i = j - 1; i >= 0; i--) {
            double s2 = gv[i];
            for (int k = i + 1; k < j; k++) s2 -= H[i * m + k] * y[k];
            y[i] = H[i * m + i] != 0.0 ? s2 / H[i * m + i] : 0.0;
        }
        for (int i = 0; i < j; i++) {
            const double *vi = V + (size_t)i * n;
            for (long c = 0; c < n; c++) e[c] += y[i] * vi[c];
        }
    }
    if (status == 1) {
        oracle_residual(g, ax, ay, az, b, e, res);
        if (oracle_norm2(g, res) <= tol * bnorm) status = 0;
    }
    subtract_constant(g, e, oracle_mean(g, e));
    *iters = it;
    free(b);
    free(w);
    free(res);
    free(V);
    free(H);
    free(cs);
    free(sn);
    free(gv);
    free(y);
    return status;
}

/* ------------------------------------------------------------------------ */
/* V-cycle and the outer iteration with the stopping test / Eq. 15            */
/* ------------------------------------------------------------------------ */

typedef struct {
    og_grid g;
    double *a[3];
    double *x, *b, *r;
    double *ac; /* cell coefficients (flux-conserving prolongation, coarse levels) */
} og_level;

typedef struct {
    int nlev;
    og_level lev[32];
    int nu1, nu2;
    double omega;
    int prolong; /* 0 trilinear, 1 flux-conserving */
} og_hier;

static void free_hier(og_hier *H)
{
    for (int l = 0; l < H->nlev; l++) {
        og_level *L = &H->lev[l];
        if (l > 0) {
            for (int d = 0; d < 3; d++) free(L->a[d]);
            free(L->x);
            free(L->b);
        }
        free(L->r);
        free(L->ac);
    }
}

static int build_hier(og_hier *H, const og_grid *g, const double *ax, const double *ay, const double *az)
{
    H->nlev = 1;
    og_level *L0 = &H->lev[0];
    L0->g = *g;
    L0->a[0] = (double *)ax;
    L0->a[1] = (double *)ay;
    L0->a[2] = (double *)az;
    L0->r = (double *)malloc(sizeof(double) * (size_t)cell_count(g));
    while (oracle_can_coarsen(&H->lev[H->nlev - 1].g) && H->nlev < 32) {
        og_level *F = &H->lev[H->nlev - 1];
        og_level *C = &H->lev[H->nlev];
        oracle_coarse_grid(&F->g, &C->g);
        long nc = cell_count(&C->g);
        for (int d = 0; d < 3; d++) C->a[d] = (double *)malloc(sizeof(double) * (size_t)nc);
        C->x = (double *)malloc(sizeof(double) * (size_t)nc);
        C->b = (double *)malloc(sizeof(double) * (size_t)nc);
        C->r = (double *)malloc(sizeof(double) * (size_t)nc);
        oracle_coarsen_faces(&F->g, F->a[0], F->a[1], F->a[2], C->a[0], C->a[1], C->a[2]);
        if (H->prolong == 1) {
            C->ac = (double *)malloc(sizeof(double) * (size_t)nc);
            oracle_cell_alpha(&C->g, C->a[0], C->a[1], C->a[2], C->ac);
        }
        H->nlev++;
    }
    return 0;
}

static void smooth(const og_hier *H, const og_level *L, int sweeps)
{
    for (int s = 0; s < sweeps; s++) {
        oracle_smooth_colour(&L->g, L->a[0], L->a[1], L->a[2], L->b, L->x, 0, H->omega);
        oracle_smooth_colour(&L->g, L->a[0], L->a[1], L->a[2], L->b, L->x, 1, H->omega);
    }
}

static int vcycle(og_hier *H, int l)
{
    og_level *L = &H->lev[l];
    if (l == H->nlev - 1) {
        if (cell_count(&L->g) <= 512)
            return oracle_coarse_solve(&L->g, L->a[0], L->a[1], L->a[2], L->b, L->x);
        int its;
        oracle_gmres(&L->g, L->a[0], L->a[1], L->a[2], L->b, L->x, 1e-13, 2000, 50, &its);
        return 0;
    }
    smooth(H, L, H->nu1);
    og_level *C = &H->lev[l + 1];
    oracle_residual(&L->g, L->a[0], L->a[1], L->a[2], L->b, L->x, L->r);
    oracle_restrict(&L->g, L->r, C->b);
    memset(C->x, 0, sizeof(double) * (size_t)cell_count(&C->g));
    int st = vcycle(H, l + 1);
    if (st) return st;
    if (H->prolong == 1) oracle_prolong_flux_add(&L->g, C->ac, C->x, L->x);
    else oracle_prolong_add(&L->g, C->x, L->x);
    smooth(H, L, H->nu2);
    return 0;
}

/* Solve A x = b to ||b - A x||_2 <= tol ||b||_2 with V(nu1, nu2) cycles.
 * b is first projected to zero mean; x is the warm start on entry and the
 * zero-mean iterate on exit.  hist[0..*ncycles] receives the residual norms
 * R_0 .. R_nc (Eq. 15 uses R_nc and R_0).  If `stagnate` is non-zero the
 * iteration also stops once three cycles in a row have not lowered the best
 * residual by 10% (used to reach p* to rounding).
 * prolong selects the prolongation (4): 0 trilinear, 1 flux-conserving.
 * Returns 0 converged, 1 not converged in max_cycles, 2 stopped on
 * stagnation, <0 error. */
int oracle_solve(const og_grid *g, const double *ax, const double *ay, const double *az,
                 const double *b_in, double *x, double tol, int max_cycles, int nu1, int nu2,
                 double omega, int stagnate, int prolong, double *hist, int *ncycles)
{
    og_hier H;
    memset(&H, 0, sizeof(H));
    H.nu1 = nu1;
    H.nu2 = nu2;
    H.omega = omega;
    H.prolong = prolong;
    build_hier(&H, g, ax, ay, az);
    og_level *L0 = &H.lev[0];
    long n = cell_count(g);
    double *b = (double *)malloc(sizeof(double) * (size_t)n);
    memcpy(b, b_in, sizeof(double) * (size_t)n);
    subtract_constant(g, b, oracle_mean(g, b));
    L0->b = b;
    L0->x = x;
    double bnorm = oracle_norm2(g, b);
    int status = 1, cyc = 0, rises = 0;
    if (bnorm == 0.0) {
        memset(x, 0, sizeof(double) * (size_t)n);
        hist[0] = 0.0;
        status = 0;
    } else {
        oracle_residual(g, ax, ay, az, b, x, L0->r);
        double best = oracle_norm2(g, L0->r);
        hist[0] = best;
        if (best <= tol * bnorm) status = 0;
        while (status == 1 && cyc < max_cycles) {
            int st = vcycle(&H, 0);
            if (st) { status = st; break; }
            subtract_constant(g, x, oracle_mean(g, x));
            cyc++;
            oracle_residual(g, ax, ay, az, b, x, L0->r);
            double rn = oracle_norm2(g, L0->r);
            hist[cyc] = rn;
            if (rn <= tol * bnorm) { status = 0; break; }
            if (!(rn == rn)) { status = -3; break; } /* NaN */
            /* progress = a new minimum at least 10% below the previous one */
            if (rn < 0.9 * best) {
                best = rn;
                rises = 0;
            } else {
                rises++;
            }
            if (stagnate && rises >= 3) { status = 2; break; }
        }
    }
    subtract_constant(g, x, oracle_mean(g, x));
    *ncycles = cyc;
    free(b);
    L0->x = NULL;
    L0->b = NULL;
    free_hier(&H);
    return status;
}

/* Preconditioner of oracle_pcg_solve: z = M r.  precond = 1: one V(nu1, nu2)
 * cycle of the hierarchy H on A z = r from z = 0, then z - mean(z);
 * precond = 0: z = r.  Returns 0, or the cycle's (negative) error status. */
static int pcg_precondition(og_hier *H, const og_grid *g, int precond, double *r, double *z, size_t bytes)
{
    if (!precond) {
        memcpy(z, r, bytes);
        return 0;
    }
    og_level *L0 = &H->lev[0];
    L0->b = r;
    L0->x = z;
    memset(z, 0, bytes);
    int st = vcycle(H, 0);
    if (st) return st;
    subtract_constant(g, z, oracle_mean(g, z));
    return 0;
}

/* Conjugate gradients on the SPD operator -A (zero-mean subspace), with the
 * residual kept in the sign of the multigrid (r = b - A x, q = A d):
 *   alpha = (r.z) / (d.q),  x += alpha d,  r -= alpha q,
 *   beta = -alpha (z_new.q) / (r.z)_old   (Polak-Ribiere form, which equals the
 *   Fletcher-Reeves one for a fixed symmetric preconditioner),
 *   d = z_new + beta d.
 * precond = 1: z = one V(nu1, nu2) cycle on A z = r from z = 0 (the multigrid
 * of this file as the preconditioner), then z - mean(z); precond = 0: z = r
 * (plain CG).  Stopping test and history as oracle_solve (hist[k] = ||r_k||,
 * r the recursive residual).  Returns 0 converged, 1 not converged, -3 NaN,
 * -4 breakdown (d.q >= 0). */
int oracle_pcg_solve(const og_grid *g, const double *ax, const double *ay, const double *az,
                     const double *b_in, double *x, double tol, int max_it, int nu1, int nu2,
                     double omega, int precond, double *hist, int *nit)
{
    og_hier H;
    memset(&H, 0, sizeof(H));
    H.nu1 = nu1;
    H.nu2 = nu2;
    H.omega = omega;
    H.prolong = 0;
    build_hier(&H, g, ax, ay, az);
    og_level *L0 = &H.lev[0];
    long n = cell_count(g);
    size_t bytes = sizeof(double) * (size_t)n;
    double *b = (double *)malloc(bytes), *r = (double *)malloc(bytes), *z = (double *)malloc(bytes);
    double *d = (double *)malloc(bytes), *q = (double *)malloc(bytes);
    memcpy(b, b_in, bytes);
    subtract_constant(g, b, oracle_mean(g, b));
    double bnorm = oracle_norm2(g, b);
    int status = 1, it = 0;
    oracle_residual(g, ax, ay, az, b, x, r);
    double rn = oracle_norm2(g, r);
    hist[0] = rn;
    double rz = 0.0;
    if (bnorm == 0.0 || rn <= tol * bnorm) status = 0;
    if (status == 1) {
        int st = pcg_precondition(&H, g, precond, r, z, bytes);
        if (st) {
            status = st;
        } else {
            memcpy(d, z, bytes);
            rz = 0.0;
            for (long c = 0; c < n; c++) rz += r[c] * z[c];
        }
    }
    while (status == 1 && it < max_it) {
        oracle_apply(g, ax, ay, az, d, q);
        double dq = 0.0;
        for (long c = 0; c < n; c++) dq += d[c] * q[c];
        if (!(dq < 0.0)) { status = -4; break; }
        double alpha = rz / dq;
        for (long c = 0; c < n; c++) {
            x[c] += alpha * d[c];
            r[c] -= alpha * q[c];
        }
        it++;
        rn = oracle_norm2(g, r);
        hist[it] = rn;
        if (!(rn == rn)) { status = -3; break; }
        if (rn <= tol * bnorm) { status = 0; break; }
        int st = pcg_precondition(&H, g, precond, r, z, bytes);
        if (st) {
            status = st;
            break;
        }
        double zq = 0.0, rz_new = 0.0;
        for (long c = 0; c < n; c++) {
            zq += z[c] * q[c];
            rz_new += r[c] * z[c];
        }
        double beta = -alpha * zq / rz;
        rz = rz_new;
        for (long c = 0; c < n; c++) d[c] = z[c] + beta * d[c];
    }
    subtract_constant(g, x, oracle_mean(g, x));
    *nit = it;
    L0->x = NULL;
    L0->b = NULL;
    free(b);
    free(r);
    free(z);
    free(d);
    free(q);
    free_hier(&H);
    return status;
}

/* Eq. 15: gamma = (R_nc / R_0)^(1/nc) */
double oracle_gamma(const double *hist, int ncycles)
{
    if (ncycles <= 0 || hist[0] == 0.0) return 0.0;
    return pow(hist[ncycles] / hist[0], 1.0 / (double)ncycles);
}
