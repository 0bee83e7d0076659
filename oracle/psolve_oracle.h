/*
 * psolve_oracle.h -- interface of the FP64 CPU oracle (psolve_oracle.c).
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU
 * baseline leg of the benchmark.  The CUDA library neither includes nor links
 * this header; the two sides agree only on the numeric meaning of the status
 * and preconditioner codes, which both take from their own definitions.
 *
 * Vectors are n[0]*n[1]*n[2] doubles, x fastest (i + n0*(j + n1*k)).
 */
#ifndef PSOLVE_ORACLE_H
#define PSOLVE_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    ORACLE_OK = 0,
    ORACLE_E_ARG = 1,
    ORACLE_E_OOM = 2,
    ORACLE_NOT_CONVERGED = 4,
    ORACLE_BREAKDOWN = 5,
    ORACLE_NONFINITE = 6
};

enum {
    ORACLE_PC_NONE = 0,        /* M = I                                       */
    ORACLE_PC_CHEB = 1,        /* G(CI): Chebyshev on the whole grid          */
    ORACLE_PC_BJ_CHEB = 2,     /* BJ(CI): Chebyshev per block, block bounds   */
    ORACLE_PC_GNOCOMM_CHEB = 3, /* GNoComm(CI): per block, whole-grid bounds  */
    ORACLE_PC_G_BICGS = 4,      /* G(BiCGS): inner Bi-CGSTAB on the whole grid */
    ORACLE_PC_BJ_BICGS = 5      /* BJ(BiCGS): inner Bi-CGSTAB on each block     */
};

typedef struct {
    int32_t type;       /* ORACLE_PC_*                                        */
    int32_t degree;     /* Chebyshev iterMax of Algorithm 2 (A-applications)  */
    int32_t blocks[3];  /* number of equal blocks along x, y, z (BJ/GNoComm)  */
    double lmin_scale;  /* lower bound handed to CI = lmin_scale * lambda_min */
    double lmax_scale;  /* upper bound handed to CI = lmax_scale * lambda_max */
    int32_t bc[6];      /* face conditions of the operator (A and M), x-, x+,
                           y-, y+, z-, z+: 0 zero Dirichlet (D, Eq. 4), 1 zero-
                           flux Neumann (N, Eq. 5)                           */
    double inner_rtol;  /* G(BiCGS) / BJ(BiCGS): inner relative tolerance  */
    int32_t inner_maxit;/* and iteration limit of the inner Bi-CGSTAB      */
    int32_t pad_;
} oracle_pc;

typedef struct {
    int32_t status;            /* ORACLE_*                                    */
    int32_t iterations;        /* outer index i at exit (0 if r0 passes)      */
    int32_t half_step_exit;    /* 1 if the exit was the ||s|| test            */
    int32_t pad_;
    double rel_res_recursive;  /* ||r||/||b|| of the recursive residual       */
    double rel_res_true;       /* ||b - A x||/||b|| recomputed at exit        */
} oracle_result;

double oracle_dot(int64_t N, const double *a, const double *b);
/* Threads the OpenMP build uses from now on (n > 0 sets it); returns the
 * count in force (always 1 for the serial build). */
int oracle_threads(int32_t n);
int oracle_apply_A(const int64_t n[3], const double h[3], const int32_t blocks[3],
                   const double *u, double *out);
int oracle_eig_bounds(const int64_t n[3], const double h[3], double *lmin, double *lmax);
/* The same with face conditions (NULL: all Dirichlet; see oracle_pc.bc). */
int oracle_apply_A_bc(const int64_t n[3], const double h[3], const int32_t bc[6], const int32_t blocks[3],
                      const double *u, double *out);
int oracle_eig_bounds_bc(const int64_t n[3], const double h[3], const int32_t bc[6], double *lmin,
                         double *lmax);
int oracle_cheb_bc(const int64_t n[3], const double h[3], const int32_t bc[6], const int32_t blocks[3],
                   double a, double b, int32_t degree, const double *rhs, double *x);
int oracle_cheb_interval_bc(const int64_t n[3], const double h[3], const int32_t bc[6], int32_t precond,
                            const int32_t blocks[3], double lmin_scale, double lmax_scale, double *a,
                            double *b);
int oracle_cheb(const int64_t n[3], const double h[3], const int32_t blocks[3],
                double a, double b, int32_t degree, const double *rhs, double *x);
int oracle_cheb_interval(const int64_t n[3], const double h[3], int32_t precond,
                         const int32_t blocks[3], double lmin_scale, double lmax_scale,
                         double *a, double *b);
int oracle_precond_apply(const int64_t n[3], const double h[3], const oracle_pc *pc,
                         const double *in, double *out);
int oracle_bicgstab(const int64_t n[3], const double h[3], const double *b,
                    double *x, int32_t use_x0, double rtol, int32_t maxit,
                    const oracle_pc *pc, int32_t half_step_check,
                    oracle_result *res, double *hist_s, double *hist_r);
/* oracle_bicgstab with residual replacement every rr_every iterations
 * (0 = none; an addition to the paper's method, see psolve_oracle.c). */
int oracle_bicgstab_rr(const int64_t n[3], const double h[3], const double *b,
                       double *x, int32_t use_x0, double rtol, int32_t maxit,
                       const oracle_pc *pc, int32_t half_step_check, int32_t rr_every,
                       oracle_result *res, double *hist_s, double *hist_r);
/* oracle_bicgstab_rr that also copies x after the outer iterations snap_at[j]
 * (j < nsnap) into snap_x + j*N (record only; see psolve_oracle.c). */
int oracle_bicgstab_snap(const int64_t n[3], const double h[3], const double *b,
                         double *x, int32_t use_x0, double rtol, int32_t maxit,
                         const oracle_pc *pc, int32_t half_step_check, int32_t rr_every,
                         oracle_result *res, double *hist_s, double *hist_r,
                         int32_t nsnap, const int32_t *snap_at, double *snap_x);

#ifdef __cplusplus
}
#endif
#endif
