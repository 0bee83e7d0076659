/*
 * psolve_oracle.c -- plain, serial FP64 CPU oracle for the preconditioned
 * Bi-CGSTAB Poisson solver of arxiv 2503.08935.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product (CUDA) path includes,
 * links or calls this file; only the tests, the smoke check and the timed
 * CPU-baseline leg of the benchmark load it.  It shares no code, header,
 * table or constant with the CUDA library.
 *
 * Every routine is the textbook definition written out with plain loops in
 * the order the paper states it:
 *   - 7-point operator          : Eq. 3 (second-order difference) and Eq. 6
 *                                 (Kronecker sum of 1-D matrices: Dirichlet D,
 *                                 Eq. 4, where neighbours outside the grid are
 *                                 0, or, on a face with a zero-flux Neumann
 *                                 condition, N of Eq. 5, where the boundary
 *                                 unknown's outside neighbour equals its
 *                                 inside one).
 *   - Block restriction         : Eq. 12-14 (R_s A R_s^T, non-overlapping
 *                                 equal blocks; cross-block neighbours are 0).
 *   - Eigenvalue bounds         : Eq. 8-11 with the Dirichlet spectrum Eq. 9;
 *                                 for N (Eq. 5) the closed form of its
 *                                 spectrum (see mu_range_1d).
 *   - Chebyshev iteration       : Eq. 15 (theta, delta, sigma) and Algorithm 2.
 *   - Preconditioned Bi-CGSTAB  : Algorithm 1 (right-preconditioned form with
 *                                 the half-step exit), stopping on the
 *                                 relative residual ||r||_2/||b||_2.
 *   - Dot products              : Ogita-Rump-Oishi "Dot2" (SIAM J. Sci.
 *                                 Comput. 26(6), 2005), summed in index order,
 *                                 so the oracle's dots are close to correctly
 *                                 rounded and independent of any GPU
 *                                 reduction tree.
 *
 * Layout: a grid vector is n[0]*n[1]*n[2] doubles, x fastest:
 *   idx(i,j,k) = i + n[0]*(j + n[1]*k).
 *
 * Build with -O2 -ffp-contract=off and without -ffast-math: Dot2's
 * error-free transformations need IEEE rounding of every operation.
 *
 * The same source compiles a second time with -fopenmp (liboracle_omp.so),
 * for the timed CPU baseline and for long stored reference runs.  That build
 * only spreads the loops over threads with a static schedule: every grid
 * point is computed by the same expression, and the dot product is the same
 * Dot2 recurrence run on ORACLE_DOT_CHUNKS fixed index ranges and joined in
 * range order (see oracle_dot), so its results do not depend on the thread
 * count.  The serial build is the one the parity tests use.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#define ORACLE_PAR_FOR _Pragma("omp parallel for schedule(static)")
#else
#define ORACLE_PAR_FOR
#endif

#include "psolve_oracle.h"

int oracle_threads(int32_t n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Dot2 (Ogita, Rump, Oishi 2005): error-free TwoProduct via fma, Knuth's     */
/* TwoSum, and a running compensation term.                                   */
/* ------------------------------------------------------------------------ */
static void two_sum(double a, double b, double *s, double *e)
{
    double x = a + b;
    double z = x - a;
    *e = (a - (x - z)) + (b - z);
    *s = x;
}

static void two_prod(double a, double b, double *p, double *e)
{
    double x = a * b;
    *e = fma(a, b, -x);
    *p = x;
}

/* The Dot2 recurrence over a[i0..i1) b[i0..i1) (i1 > i0): running sum p and
 * accumulated error s, result p + s. */
static void dot2_range(int64_t i0, int64_t i1, const double *a, const double *b, double *p_out, double *s_out)
{
    double p, s, h, r, q;
    two_prod(a[i0], b[i0], &p, &s);
    for (int64_t i = i0 + 1; i < i1; ++i) {
        two_prod(a[i], b[i], &h, &r);
        two_sum(p, h, &p, &q);
        s = s + (q + r);
    }
    *p_out = p;
    *s_out = s;
}

#ifdef _OPENMP
#define ORACLE_DOT_CHUNKS 64
/* OpenMP build: the index range is cut into ORACLE_DOT_CHUNKS fixed ranges
 * (independent of the thread count), each summed by the recurrence above,
 * and the range results are joined in range order by the same step (TwoSum
 * of the running sums, errors added to s), which keeps Dot2's error bound. */
double oracle_dot(int64_t N, const double *a, const double *b)
{
    if (N <= 0) return 0.0;
    double pc[ORACLE_DOT_CHUNKS], sc[ORACLE_DOT_CHUNKS];
    ORACLE_PAR_FOR
    for (int c = 0; c < ORACLE_DOT_CHUNKS; ++c) {
        const int64_t i0 = N * c / ORACLE_DOT_CHUNKS, i1 = N * (c + 1) / ORACLE_DOT_CHUNKS;
        pc[c] = 0.0;
        sc[c] = 0.0;
        if (i1 > i0) dot2_range(i0, i1, a, b, &pc[c], &sc[c]);
    }
    double p = pc[0], s = sc[0], q;
    for (int c = 1; c < ORACLE_DOT_CHUNKS; ++c) {
        two_sum(p, pc[c], &p, &q);
        s = s + (q + sc[c]);
    }
    return p + s;
}
#else
double oracle_dot(int64_t N, const double *a, const double *b)
{
    if (N <= 0) return 0.0;
    double p, s;
    dot2_range(0, N, a, b, &p, &s);
    return p + s;
}
#endif

/* ------------------------------------------------------------------------ */
/* 7-point operator, Eq. 3 / Eq. 6.                                           */
/* ------------------------------------------------------------------------ */

/* Value of u at integer coordinates c_in (one of which may be out of range).
 * Outside the grid it is 0 (zero Dirichlet ghost, Eq. 4), except across a
 * face with a zero-flux Neumann condition (bc[face] == 1, faces ordered x-,
 * x+, y-, y+, z-, z+), where the outside neighbour of the boundary unknown
 * equals its inside neighbour (matrix N, Eq. 5: its row reads
 * 2 u_0 - 2 u_1).  When bs != NULL it is also 0 outside the block of size bs
 * that contains `home` (Eq. 14). */
static double nb_value(const int64_t n[3], const int64_t *bs, const int32_t *bc, const double *u,
                       const int64_t home[3], const int64_t c_in[3])
{
    int64_t c[3] = {c_in[0], c_in[1], c_in[2]};
    for (int d = 0; d < 3; ++d) {
        if (c[d] < 0 && bc && bc[2 * d] == 1) c[d] = home[d] + 1;
        if (c[d] >= n[d] && bc && bc[2 * d + 1] == 1) c[d] = home[d] - 1;
        if (c[d] < 0 || c[d] >= n[d]) return 0.0;
        if (bs && (c[d] / bs[d]) != (home[d] / bs[d])) return 0.0;
    }
    return u[c[0] + n[0] * (c[1] + n[1] * c[2])];
}

/* Boundary conditions: NULL (all Dirichlet) or six codes 0 (Dirichlet) / 1
 * (Neumann); a Neumann face needs at least 2 points (and 2 per block) on its
 * axis. */
static int check_bc(const int64_t n[3], const int64_t *bs, const int32_t *bc)
{
    if (!bc) return ORACLE_OK;
    for (int f = 0; f < 6; ++f) {
        if (bc[f] != 0 && bc[f] != 1) return ORACLE_E_ARG;
        const int d = f / 2;
        if (bc[f] == 1 && (n[d] < 2 || (bs && bs[d] < 2))) return ORACLE_E_ARG;
    }
    return ORACLE_OK;
}

int oracle_apply_A(const int64_t n[3], const double h[3], const int32_t blocks[3],
                   const double *u, double *out)
{
    return oracle_apply_A_bc(n, h, NULL, blocks, u, out);
}

int oracle_apply_A_bc(const int64_t n[3], const double h[3], const int32_t bc[6], const int32_t blocks[3],
                      const double *u, double *out)
{
    int64_t bs_store[3];
    const int64_t *bs = NULL;
    for (int d = 0; d < 3; ++d)
        if (n[d] < 1 || !(h[d] > 0.0)) return ORACLE_E_ARG;
    if (blocks) {
        for (int d = 0; d < 3; ++d) {
            if (blocks[d] < 1 || n[d] % blocks[d] != 0) return ORACLE_E_ARG;
            bs_store[d] = n[d] / blocks[d];
        }
        bs = bs_store;
    }
    if (check_bc(n, bs, bc)) return ORACLE_E_ARG;
    ORACLE_PAR_FOR
    for (int64_t k = 0; k < n[2]; ++k)
        for (int64_t j = 0; j < n[1]; ++j)
            for (int64_t i = 0; i < n[0]; ++i) {
                const int64_t home[3] = {i, j, k};
                const double uc = u[i + n[0] * (j + n[1] * k)];
                double acc = 0.0;
                for (int d = 0; d < 3; ++d) {
                    int64_t lo[3] = {i, j, k}, hi[3] = {i, j, k};
                    lo[d] -= 1;
                    hi[d] += 1;
                    const double ul = nb_value(n, bs, bc, u, home, lo);
                    const double uh = nb_value(n, bs, bc, u, home, hi);
                    /* (-u_{d-1} + 2 u_d - u_{d+1}) / h_d^2 , Eq. 3 */
                    acc += (-ul + 2.0 * uc - uh) / (h[d] * h[d]);
                }
                out[i + n[0] * (j + n[1] * k)] = acc;
            }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Eigenvalue bounds, Eq. 8-11 with Eq. 9.                                    */
/* ------------------------------------------------------------------------ */
static double mu_dirichlet(int64_t i, int64_t n)
{
    const double pi = 3.14159265358979323846;
    const double s = sin((double)i * pi / (2.0 * (double)(n + 1)));
    return 4.0 * s * s; /* Eq. 9 */
}

int oracle_eig_bounds(const int64_t n[3], const double h[3], double *lmin, double *lmax)
{
    double lo = 0.0, hi = 0.0;
    for (int d = 0; d < 3; ++d) {
        if (n[d] < 1 || !(h[d] > 0.0)) return ORACLE_E_ARG;
        /* Eq. 10 / 11: sum over axes of the extreme 1-D eigenvalues. */
        lo += mu_dirichlet(1, n[d]) / (h[d] * h[d]);
        hi += mu_dirichlet(n[d], n[d]) / (h[d] * h[d]);
    }
    *lmin = lo;
    *lmax = hi;
    return ORACLE_OK;
}

/* Extreme eigenvalues of the 1-D operator of size m with face conditions fm
 * (minus side) and fp (plus side), 0 = Dirichlet (D, Eq. 4), 1 = Neumann (N,
 * Eq. 5).  D: Eq. 9.  One Neumann face: N is similar to a symmetric matrix
 * with the eigenvectors cos((2i-1) pi j / (2m)), j counted from the Neumann
 * end, so mu_i = 4 sin^2((2i-1) pi / (4m)), i = 1..m.  Neumann on both faces:
 * eigenvectors cos(i pi j / (m-1)), mu_i = 4 sin^2(i pi / (2(m-1))),
 * i = 0..m-1, so the range is [0, 4]. */
static void mu_range_1d(int64_t m, int fm, int fp, double *mn, double *mx)
{
    const double pi = 3.14159265358979323846;
    if (!fm && !fp) {
        *mn = mu_dirichlet(1, m);
        *mx = mu_dirichlet(m, m);
    } else if (fm != fp) {
        const double s1 = sin(pi / (4.0 * (double)m));
        const double s2 = sin((2.0 * (double)m - 1.0) * pi / (4.0 * (double)m));
        *mn = 4.0 * s1 * s1;
        *mx = 4.0 * s2 * s2;
    } else {
        const double s2 = sin((double)(m - 1) * pi / (2.0 * (double)(m - 1)));
        *mn = 0.0;
        *mx = 4.0 * s2 * s2;
    }
}

int oracle_eig_bounds_bc(const int64_t n[3], const double h[3], const int32_t bc[6], double *lmin,
                         double *lmax)
{
    if (!bc) return oracle_eig_bounds(n, h, lmin, lmax);
    if (check_bc(n, NULL, bc)) return ORACLE_E_ARG;
    double lo = 0.0, hi = 0.0;
    for (int d = 0; d < 3; ++d) {
        if (n[d] < 1 || !(h[d] > 0.0)) return ORACLE_E_ARG;
        double mn, mx;
        mu_range_1d(n[d], bc[2 * d], bc[2 * d + 1], &mn, &mx);
        lo += mn / (h[d] * h[d]); /* Eq. 10 */
        hi += mx / (h[d] * h[d]); /* Eq. 11 */
    }
    *lmin = lo;
    *lmax = hi;
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Chebyshev iteration, Eq. 15 and Algorithm 2.                               */
/* The operator is the full grid operator (blocks == NULL) or its block-      */
/* diagonal restriction (Eq. 14).  [a, b] is the eigenvalue interval.         */
/* ------------------------------------------------------------------------ */
int oracle_cheb(const int64_t n[3], const double h[3], const int32_t blocks[3],
                double a, double b, int32_t degree, const double *rhs, double *x)
{
    return oracle_cheb_bc(n, h, NULL, blocks, a, b, degree, rhs, x);
}

int oracle_cheb_bc(const int64_t n[3], const double h[3], const int32_t bc[6], const int32_t blocks[3],
                   double a, double b, int32_t degree, const double *rhs, double *x)
{
    if (degree < 0 || !(b > a) || !(a > 0.0)) return ORACLE_E_ARG;
    const int64_t N = n[0] * n[1] * n[2];
    const double theta = 0.5 * (b + a);
    const double delta = 0.5 * (b - a);
    const double sigma = theta / delta;
    double rho_old = 1.0 / sigma;
    double rho_cur = 1.0 / (2.0 * sigma - rho_old);

    double *z = (double *)malloc(sizeof(double) * (size_t)N);
    double *y = (double *)malloc(sizeof(double) * (size_t)N);
    double *w = (double *)malloc(sizeof(double) * (size_t)N);
    double *Av = (double *)malloc(sizeof(double) * (size_t)N);
    if (!z || !y || !w || !Av) {
        free(z); free(y); free(w); free(Av);
        return ORACLE_E_OOM;
    }
    int st = ORACLE_OK;
    ORACLE_PAR_FOR
    for (int64_t q = 0; q < N; ++q) z[q] = rhs[q] / theta;
    if (degree == 0) {
        memcpy(x, z, sizeof(double) * (size_t)N);
        goto done;
    }
    st = oracle_apply_A_bc(n, h, bc, blocks, rhs, Av);
    if (st) goto done;
    ORACLE_PAR_FOR
    for (int64_t q = 0; q < N; ++q)
        y[q] = 2.0 * rho_cur / delta * (2.0 * rhs[q] - Av[q] / theta);
    for (int32_t it = 2; it <= degree; ++it) {
        rho_old = rho_cur;
        rho_cur = 1.0 / (2.0 * sigma - rho_old);
        st = oracle_apply_A_bc(n, h, bc, blocks, y, Av);
        if (st) goto done;
        ORACLE_PAR_FOR
        for (int64_t q = 0; q < N; ++q)
            w[q] = rho_cur * (2.0 * sigma * y[q] + 2.0 / delta * (rhs[q] - Av[q]) - rho_old * z[q]);
        double *tmp = z; /* z <- y, y <- w */
        z = y;
        y = w;
        w = tmp;
    }
    memcpy(x, y, sizeof(double) * (size_t)N);
done:
    free(z); free(y); free(w); free(Av);
    return st;
}

/* Interval [a, b] handed to the Chebyshev iteration for a preconditioner.
 * G(CI): closed-form bounds of the whole grid.  BJ(CI): bounds of one block
 * (all blocks are equal, so they share them).  GNoComm(CI): bounds of the
 * whole grid with the block-restricted operator.  Each bound is multiplied by
 * its scale (the eigenvalue rescaling of the experimental set-up). */
int oracle_cheb_interval(const int64_t n[3], const double h[3], int32_t precond,
                         const int32_t blocks[3], double lmin_scale, double lmax_scale,
                         double *a, double *b)
{
    return oracle_cheb_interval_bc(n, h, NULL, precond, blocks, lmin_scale, lmax_scale, a, b);
}

/* With face conditions: G(CI) and GNoComm(CI) take the whole grid's bounds.
 * BJ(CI) blocks differ in their outer faces (a block on a Neumann face has
 * that face, the others have Dirichlet ghosts), so the interval covers every
 * kind of block: per axis the smallest minimum and the largest maximum over
 * the first, the interior and the last block. */
int oracle_cheb_interval_bc(const int64_t n[3], const double h[3], const int32_t bc[6], int32_t precond,
                            const int32_t blocks[3], double lmin_scale, double lmax_scale, double *a,
                            double *b)
{
    if (bc && !(bc[0] == 0 && bc[1] == 0 && bc[2] == 0 && bc[3] == 0 && bc[4] == 0 && bc[5] == 0)) {
        double lo = 0.0, hi = 0.0;
        if (check_bc(n, NULL, bc)) return ORACLE_E_ARG;
        for (int d = 0; d < 3; ++d) {
            if (n[d] < 1 || !(h[d] > 0.0)) return ORACLE_E_ARG;
            double mn, mx;
            const int fm = bc[2 * d], fp = bc[2 * d + 1];
            if (precond == ORACLE_PC_BJ_CHEB && blocks && blocks[d] > 1) {
                if (n[d] % blocks[d]) return ORACLE_E_ARG;
                const int64_t m = n[d] / blocks[d];
                double mn2, mx2;
                mu_range_1d(m, fm, 0, &mn, &mx);   /* first block */
                mu_range_1d(m, 0, fp, &mn2, &mx2); /* last block */
                if (mn2 < mn) mn = mn2;
                if (mx2 > mx) mx = mx2;
                if (blocks[d] > 2) {
                    mu_range_1d(m, 0, 0, &mn2, &mx2); /* interior blocks */
                    if (mn2 < mn) mn = mn2;
                    if (mx2 > mx) mx = mx2;
                }
            } else {
                if (precond == ORACLE_PC_BJ_CHEB && (!blocks || blocks[d] < 1)) return ORACLE_E_ARG;
                mu_range_1d(n[d], fm, fp, &mn, &mx);
            }
            lo += mn / (h[d] * h[d]);
            hi += mx / (h[d] * h[d]);
        }
        *a = lmin_scale * lo;
        *b = lmax_scale * hi;
        if (!(*b > *a) || !(*a > 0.0)) return ORACLE_E_ARG;
        return ORACLE_OK;
    }
    int64_t m[3] = {n[0], n[1], n[2]};
    if (precond == ORACLE_PC_BJ_CHEB) {
        for (int d = 0; d < 3; ++d) {
            if (!blocks || blocks[d] < 1 || n[d] % blocks[d]) return ORACLE_E_ARG;
            m[d] = n[d] / blocks[d];
        }
    }
    double lo, hi;
    int st = oracle_eig_bounds(m, h, &lo, &hi);
    if (st) return st;
    *a = lmin_scale * lo;
    *b = lmax_scale * hi;
    if (!(*b > *a) || !(*a > 0.0)) return ORACLE_E_ARG;
    return ORACLE_OK;
}

/* Inner Bi-CGSTAB of the flexible preconditioners (Sec. on G(BiCGS) and
 * BJ(BiCGS)): out = approximate solution of A out = in from out = 0, stopped at
 * inner_rtol relative to ||in|| or after inner_maxit iterations (the last
 * iterate is used either way). */
static int inner_solve(const int64_t n[3], const double h[3], const int32_t bc[6], const oracle_pc *pc,
                       const double *in, double *out)
{
    oracle_pc none;
    memset(&none, 0, sizeof none);
    none.type = ORACLE_PC_NONE;
    for (int f = 0; f < 6; ++f) none.bc[f] = bc ? bc[f] : 0;
    oracle_result r;
    const int st = oracle_bicgstab_rr(n, h, in, out, 0, pc->inner_rtol, pc->inner_maxit, &none, 1, 0, &r, NULL,
                                      NULL);
    return (st == ORACLE_OK || st == ORACLE_NOT_CONVERGED) ? ORACLE_OK : st;
}

/* BJ(BiCGS): the block-diagonal system (Eq. 13-14) solved block by block; a
 * block keeps the domain's condition on the faces it shares with the domain
 * and has zero Dirichlet ghosts towards its neighbours. */
static int block_inner_solves(const int64_t n[3], const double h[3], const oracle_pc *pc, const double *in,
                              double *out)
{
    int64_t m[3];
    for (int d = 0; d < 3; ++d) {
        if (pc->blocks[d] < 1 || n[d] % pc->blocks[d]) return ORACLE_E_ARG;
        m[d] = n[d] / pc->blocks[d];
    }
    const int64_t M = m[0] * m[1] * m[2];
    double *bi = (double *)malloc(sizeof(double) * (size_t)M);
    double *xi = (double *)malloc(sizeof(double) * (size_t)M);
    if (!bi || !xi) {
        free(bi); free(xi);
        return ORACLE_E_OOM;
    }
    int st = ORACLE_OK;
    for (int64_t Bz = 0; Bz < pc->blocks[2] && !st; ++Bz)
        for (int64_t By = 0; By < pc->blocks[1] && !st; ++By)
            for (int64_t Bx = 0; Bx < pc->blocks[0] && !st; ++Bx) {
                const int64_t B[3] = {Bx, By, Bz};
                int32_t bbc[6];
                for (int d = 0; d < 3; ++d) {
                    bbc[2 * d] = (B[d] == 0) ? pc->bc[2 * d] : 0;
                    bbc[2 * d + 1] = (B[d] == pc->blocks[d] - 1) ? pc->bc[2 * d + 1] : 0;
                }
                for (int64_t k = 0; k < m[2]; ++k)
                    for (int64_t j = 0; j < m[1]; ++j)
                        for (int64_t i = 0; i < m[0]; ++i)
                            bi[i + m[0] * (j + m[1] * k)] =
                                in[(Bx * m[0] + i) + n[0] * ((By * m[1] + j) + n[1] * (Bz * m[2] + k))];
                st = inner_solve(m, h, bbc, pc, bi, xi);
                for (int64_t k = 0; k < m[2] && !st; ++k)
                    for (int64_t j = 0; j < m[1]; ++j)
                        for (int64_t i = 0; i < m[0]; ++i)
                            out[(Bx * m[0] + i) + n[0] * ((By * m[1] + j) + n[1] * (Bz * m[2] + k))] =
                                xi[i + m[0] * (j + m[1] * k)];
            }
    free(bi);
    free(xi);
    return st;
}

int oracle_precond_apply(const int64_t n[3], const double h[3], const oracle_pc *pc,
                         const double *in, double *out)
{
    const int64_t N = n[0] * n[1] * n[2];
    if (pc->type == ORACLE_PC_NONE) {
        memcpy(out, in, sizeof(double) * (size_t)N);
        return ORACLE_OK;
    }
    if (pc->type == ORACLE_PC_G_BICGS) return inner_solve(n, h, pc->bc, pc, in, out);
    if (pc->type == ORACLE_PC_BJ_BICGS) return block_inner_solves(n, h, pc, in, out);
    double a, b;
    int st = oracle_cheb_interval_bc(n, h, pc->bc, pc->type, pc->blocks, pc->lmin_scale, pc->lmax_scale, &a,
                                     &b);
    if (st) return st;
    const int32_t *blk = (pc->type == ORACLE_PC_CHEB) ? NULL : pc->blocks;
    return oracle_cheb_bc(n, h, pc->bc, blk, a, b, pc->degree, in, out);
}

/* ------------------------------------------------------------------------ */
/* Preconditioned Bi-CGSTAB, Algorithm 1.                                     */
/* ------------------------------------------------------------------------ */
static int finite(double v) { return isfinite(v); }

int oracle_bicgstab(const int64_t n[3], const double h[3], const double *bvec,
                    double *x, int32_t use_x0, double rtol, int32_t maxit,
                    const oracle_pc *pc, int32_t half_step_check,
                    oracle_result *res, double *hist_s, double *hist_r)
{
    return oracle_bicgstab_rr(n, h, bvec, x, use_x0, rtol, maxit, pc, half_step_check, 0,
                              res, hist_s, hist_r);
}

/* rr_every > 0 adds residual replacement, which is not part of the paper's
 * method: after the update of iteration i (a multiple of rr_every, i < maxit,
 * not converged), r is recomputed as b - A x, its norm takes the stop test,
 * and beta (proportional to rho_i) and rho_i are rescaled to rho = r~ . r of
 * the new r.  rr_every = 0 is Algorithm 1 exactly. */
int oracle_bicgstab_rr(const int64_t n[3], const double h[3], const double *bvec,
                       double *x, int32_t use_x0, double rtol, int32_t maxit,
                       const oracle_pc *pc, int32_t half_step_check, int32_t rr_every,
                       oracle_result *res, double *hist_s, double *hist_r)
{
    return oracle_bicgstab_snap(n, h, bvec, x, use_x0, rtol, maxit, pc, half_step_check, rr_every, res, hist_s,
                                hist_r, 0, NULL, NULL);
}

/* Copy of x after outer iteration i into the snapshot slots that ask for it. */
static void snapshot(int64_t N, const double *x, int32_t i, int32_t nsnap, const int32_t *snap_at,
                     double *snap_x)
{
    for (int32_t j = 0; j < nsnap; ++j)
        if (snap_at[j] == i) memcpy(snap_x + (size_t)j * (size_t)N, x, sizeof(double) * (size_t)N);
}

/* oracle_bicgstab_rr that also copies x after the outer iterations listed in
 * snap_at[0..nsnap) into snap_x (nsnap vectors of N doubles): the iterate a
 * run with maxit = snap_at[j] would return.  Slots of iterations the solve
 * does not reach are left untouched.  Records only; no arithmetic changes. */
int oracle_bicgstab_snap(const int64_t n[3], const double h[3], const double *bvec,
                         double *x, int32_t use_x0, double rtol, int32_t maxit,
                         const oracle_pc *pc, int32_t half_step_check, int32_t rr_every,
                         oracle_result *res, double *hist_s, double *hist_r,
                         int32_t nsnap, const int32_t *snap_at, double *snap_x)
{
    memset(res, 0, sizeof(*res));
    if (nsnap < 0 || (nsnap > 0 && (!snap_at || !snap_x))) return res->status = ORACLE_E_ARG;
    if (rr_every < 0) return res->status = ORACLE_E_ARG;
    for (int d = 0; d < 3; ++d)
        if (n[d] < 1 || !(h[d] > 0.0)) return res->status = ORACLE_E_ARG;
    if (maxit < 0 || !(rtol >= 0.0) || !pc || pc->degree < 0) return res->status = ORACLE_E_ARG;
    const int64_t N = n[0] * n[1] * n[2];
    const size_t bytes = sizeof(double) * (size_t)N;

    double *r = malloc(bytes), *rt = malloc(bytes), *p = malloc(bytes);
    double *ph = malloc(bytes), *w = malloc(bytes), *s = malloc(bytes);
    double *rh = malloc(bytes), *t = malloc(bytes);
    int st = ORACLE_OK;
    if (!r || !rt || !p || !ph || !w || !s || !rh || !t) { st = ORACLE_E_OOM; goto out; }

    const double nb = sqrt(oracle_dot(N, bvec, bvec));
    if (!finite(nb)) { st = ORACLE_NONFINITE; goto out; }
    if (nb == 0.0) { /* b = 0: the solution is x = 0 */
        memset(x, 0, bytes);
        st = ORACLE_OK;
        goto out;
    }
    /* r0 = b - A x0 */
    if (use_x0) {
        st = oracle_apply_A_bc(n, h, pc->bc, NULL, x, t);
        if (st) goto out;
        ORACLE_PAR_FOR
        for (int64_t q = 0; q < N; ++q) r[q] = bvec[q] - t[q];
    } else {
        memset(x, 0, bytes);
        memcpy(r, bvec, bytes);
    }
    memcpy(rt, r, bytes); /* r~ = r0 */
    memcpy(p, r, bytes);  /* p0 = r0 */
    double rho = oracle_dot(N, rt, r);
    double rnorm = sqrt(oracle_dot(N, r, r));
    res->rel_res_recursive = rnorm / nb;
    if (rnorm / nb <= rtol) { st = ORACLE_OK; goto out; }

    st = ORACLE_NOT_CONVERGED;
    for (int32_t i = 1; i <= maxit; ++i) {
        res->iterations = i;
        int e = oracle_precond_apply(n, h, pc, p, ph); /* M p^ = p */
        if (e) { st = e; break; }
        e = oracle_apply_A_bc(n, h, pc->bc, NULL, ph, w); /* w = A p^ */
        if (e) { st = e; break; }
        const double sig1 = oracle_dot(N, rt, w);
        if (!finite(sig1)) { st = ORACLE_NONFINITE; break; }
        if (sig1 == 0.0) { st = ORACLE_BREAKDOWN; break; }
        const double alpha = rho / sig1;
        ORACLE_PAR_FOR
        for (int64_t q = 0; q < N; ++q) s[q] = r[q] - alpha * w[q];
        const double snorm = sqrt(oracle_dot(N, s, s));
        if (hist_s) hist_s[i - 1] = snorm / nb;
        if (!finite(snorm)) { st = ORACLE_NONFINITE; break; }
        if (half_step_check && snorm / nb <= rtol) {
            ORACLE_PAR_FOR
            for (int64_t q = 0; q < N; ++q) x[q] = x[q] + alpha * ph[q];
            snapshot(N, x, i, nsnap, snap_at, snap_x);
            res->half_step_exit = 1;
            res->rel_res_recursive = snorm / nb;
            st = ORACLE_OK;
            break;
        }
        e = oracle_precond_apply(n, h, pc, s, rh); /* M r^ = s */
        if (e) { st = e; break; }
        e = oracle_apply_A_bc(n, h, pc->bc, NULL, rh, t); /* t = A r^ */
        if (e) { st = e; break; }
        const double tt = oracle_dot(N, t, t);
        const double ts = oracle_dot(N, t, s);
        if (!finite(tt) || !finite(ts)) { st = ORACLE_NONFINITE; break; }
        if (tt == 0.0) { st = ORACLE_BREAKDOWN; break; }
        const double omega = ts / tt;
        if (omega == 0.0) { st = ORACLE_BREAKDOWN; break; }
        ORACLE_PAR_FOR
        for (int64_t q = 0; q < N; ++q) {
            x[q] = x[q] + alpha * ph[q] + omega * rh[q];
            r[q] = s[q] - omega * t[q];
        }
        snapshot(N, x, i, nsnap, snap_at, snap_x);
        rnorm = sqrt(oracle_dot(N, r, r));
        res->rel_res_recursive = rnorm / nb;
        if (hist_r) hist_r[i - 1] = rnorm / nb;
        if (!finite(rnorm)) { st = ORACLE_NONFINITE; break; }
        if (rnorm / nb <= rtol) { st = ORACLE_OK; break; }
        double rho_new = oracle_dot(N, rt, r);
        if (rho_new == 0.0) { st = ORACLE_BREAKDOWN; break; }
        double beta = (rho_new / rho) * (alpha / omega);
        if (rr_every > 0 && i % rr_every == 0 && i < maxit) {
            /* residual replacement (see above) */
            e = oracle_apply_A_bc(n, h, pc->bc, NULL, x, t);
            if (e) { st = e; break; }
            ORACLE_PAR_FOR
            for (int64_t q = 0; q < N; ++q) r[q] = bvec[q] - t[q];
            rnorm = sqrt(oracle_dot(N, r, r));
            const double rho_true = oracle_dot(N, rt, r);
            res->rel_res_recursive = rnorm / nb;
            if (hist_r) hist_r[i - 1] = rnorm / nb;
            if (!finite(rnorm) || !finite(rho_true)) { st = ORACLE_NONFINITE; break; }
            if (rnorm / nb <= rtol) { st = ORACLE_OK; break; }
            if (rho_true == 0.0) { st = ORACLE_BREAKDOWN; break; }
            beta = beta * (rho_true / rho_new);
            rho_new = rho_true;
        }
        rho = rho_new;
        ORACLE_PAR_FOR
        for (int64_t q = 0; q < N; ++q) p[q] = r[q] + beta * (p[q] - omega * w[q]);
    }

out:
    if (st != ORACLE_E_ARG && st != ORACLE_E_OOM && N > 0 && r && t) {
        /* true residual ||b - A x|| / ||b|| of the returned x */
        if (oracle_apply_A_bc(n, h, pc->bc, NULL, x, t) == ORACLE_OK) {
            ORACLE_PAR_FOR
            for (int64_t q = 0; q < N; ++q) r[q] = bvec[q] - t[q];
            const double nbb = sqrt(oracle_dot(N, bvec, bvec));
            res->rel_res_true = nbb > 0.0 ? sqrt(oracle_dot(N, r, r)) / nbb : 0.0;
        }
    }
    res->status = st;
    free(r); free(rt); free(p); free(ph); free(w); free(s); free(rh); free(t);
    return st;
}
