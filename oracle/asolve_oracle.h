/*
 * asolve_oracle.h -- plain, slow, FP64 CPU oracle for the adaptive solver of
 * Sanderson & Curtin, "An Adaptive Solver for Systems of Linear Equations"
 * (arXiv 2007.11208).
 *
 * TEST INFRASTRUCTURE ONLY.  This header and asolve_oracle.c are the checker
 * the GPU library is compared against.  Only the test suite, the smoke check
 * and the CPU-baseline leg of the benchmark may load this code; the product
 * library never does, and shares no code, header or constant with it.
 *
 * Storage: every matrix is dense, column-major, leading dimension n (paper
 * Sec. 1 and Sec. 2.1: "column-major dense matrix"); element (i,j), 0-based,
 * is A[i + j*n].  Band storage follows the LAPACK band layout the paper
 * names in Sec. 2.1 (xGBTRF): element (i,j) of the band matrix sits at
 * AB[(kl+ku+i-j) + j*ldab] with ldab >= 2*kl+ku+1, the top kl rows being
 * fill-in room for the U factor.
 */
#ifndef ASOLVE_ORACLE_H
#define ASOLVE_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Detected class (Sec. 2: banded, then triangular, then sympd, else general). */
enum { OR_CLS_NONE = 0, OR_CLS_BANDED = 1, OR_CLS_LOWER = 2, OR_CLS_UPPER = 3,
       OR_CLS_SYMPD = 4, OR_CLS_GENERAL = 5 };
/* Primary (factorisation) route actually taken. */
enum { OR_ROUTE_NONE = 0, OR_ROUTE_BAND_LU = 1, OR_ROUTE_TRI_LOWER = 2,
       OR_ROUTE_TRI_UPPER = 3, OR_ROUTE_CHOL = 4, OR_ROUTE_CHOL_FAIL_LU = 5,
       OR_ROUTE_LU = 6, OR_ROUTE_SVD = 7, OR_ROUTE_TRIDIAG = 8, OR_ROUTE_LDLT = 9,
       OR_ROUTE_CHOL_FAIL_LDLT = 10 };
/* Status codes: negative = error (X not a solution), positive = warning. */
enum { OR_OK = 0, OR_W_APPROX = 1, OR_W_ILLCOND = 2, OR_E_INVALID = -1,
       OR_E_NONFINITE = -2, OR_E_SINGULAR = -3 };
/* Flags. */
enum { OR_NO_APPROX = 1, OR_FORCE_LU = 2, OR_FORCE_SVD = 4, OR_NO_RCOND = 8,
       /* the closing remarks' tridiagonal specialisation: banded systems with
        * kl = ku = 1 take the tridiagonal route (opt-in; off, they take the
        * band LU of Sec. 2.1) */
       OR_TRIDIAG = 256,
       /* the closing remarks' plain-symmetric specialisation: a system of
        * order n <= OR_LDLT_NMAX that is symmetric within the Fig. 4
        * tolerance but not likely_sympd, or whose Cholesky factorisation
        * fails, takes the Bunch-Kaufman LDL^T route (opt-in) */
       OR_SYM_INDEF = 512 };
enum { OR_LDLT_NMAX = 1024 };
/* A system given in band storage reaches the SVD fallback (Sec. 2.5) only up
 * to this order: the SVD runs on a dense copy. */
enum { OR_SVD_DENSIFY_NMAX = 8192 };

typedef struct {
  int64_t kl, ku;          /* sub/super-diagonal counts (Sec. 2.1)            */
  int32_t lower, upper;    /* triangular structure (Sec. 2.2)                 */
  int32_t sympd;           /* likely_sympd (Fig. 4)                           */
  int32_t banded;          /* band rule: band positions <= 25% of n^2        */
  int32_t nonfinite;       /* any Inf/NaN in A                                */
  int32_t cls;             /* OR_CLS_*                                        */
  double  norm1;           /* max column abs sum                              */
  double  norminf;         /* max row abs sum                                 */
} or_scan_t;

typedef struct {
  int32_t cls, route, status, svd_used;
  int64_t kl, ku;
  double  rcond;           /* estimate from the primary route, NaN if none    */
  int64_t svd_rank;        /* retained singular values, -1 if SVD not run     */
} or_info_t;

typedef struct {
  double rcond_threshold;  /* Sec. 2.5: 0.5*eps                               */
  double sympd_tol;        /* Fig. 4: 100*eps                                 */
  double band_frac;        /* Sec. 2.1: 0.25                                  */
  double svd_trunc_rel;    /* SVD truncation tau = svd_trunc_rel * sigma_max;
                              <= 0 selects n*eps                              */
} or_config_t;

void    or_default_config(or_config_t* cfg);

/* Sec. 2.1 / 2.2 / Fig. 4 scan of a dense n x n matrix. */
void    or_scan(const double* A, int64_t n, const or_config_t* cfg, or_scan_t* out);
void    or_scan_many(const double* A, int64_t n, int64_t count,
                     const or_config_t* cfg, or_scan_t* out);
int64_t or_band_count(int64_t n, int64_t kl, int64_t ku);
int     or_likely_sympd(const double* A, int64_t n, double tol);

/* Factorisations (return 0 on success, k+1 on failure at step k). */
int     or_lu_factor(double* A, int64_t n, int64_t* ipiv);
void    or_lu_solve(const double* LU, const int64_t* ipiv, int64_t n, double* B,
                    int64_t nrhs, int trans);
int     or_chol_factor(double* A, int64_t n);
void    or_chol_solve(const double* L, int64_t n, double* B, int64_t nrhs);
int     or_tri_solve(const double* T, int64_t n, int lower, double* B, int64_t nrhs,
                     int trans);
void    or_band_pack(const double* A, int64_t n, int64_t kl, int64_t ku,
                     double* AB, int64_t ldab);
int     or_band_lu_factor(double* AB, int64_t ldab, int64_t n, int64_t kl,
                          int64_t ku, int64_t* ipiv);
void    or_band_lu_solve(const double* AB, int64_t ldab, int64_t n, int64_t kl,
                         int64_t ku, const int64_t* ipiv, double* B, int64_t nrhs,
                         int trans);

/* Tridiagonal LU with partial pivoting on the three diagonals (xGTTRF
 * semantics): dl[0..n-2] sub-, d[0..n-1] main, du[0..n-2] super-diagonal,
 * du2[0..n-3] the second super-diagonal the interchanges fill in, ipiv[i] = i
 * or i+1.  Returns 0, or i+1 at the first exact zero pivot d[i]. */
int     or_gt_factor(double* dl, double* d, double* du, double* du2, int64_t* ipiv, int64_t n);
void    or_gt_solve(const double* dl, const double* d, const double* du, const double* du2,
                    const int64_t* ipiv, int64_t n, double* B, int64_t nrhs, int trans);

/* The symmetry test of Fig. 4 alone: every pair within tol, absolute or
 * relative. */
int     or_is_symmetric(const double* A, int64_t n, double tol);
/* Symmetric-indefinite LDL^T with Bunch-Kaufman pivoting (xSYTRF semantics,
 * lower triangle read and overwritten): P A P^T = L D L^T, D with 1 x 1 and
 * 2 x 2 blocks.  ipiv[k] = kp >= 0: 1 x 1 pivot, rows/columns k and kp
 * interchanged; ipiv[k] = ipiv[k+1] = -(kp+1): a 2 x 2 pivot at (k, k+1)
 * with k+1 and kp interchanged.  Returns 0, or k+1 at the first zero 1 x 1
 * pivot (an exactly zero column). */
int     or_ldlt_factor(double* A, int64_t n, int64_t* ipiv);
void    or_ldlt_solve(const double* F, const int64_t* ipiv, int64_t n, double* B, int64_t nrhs);

/* Reciprocal condition estimate (1-norm). */
double  or_norm1(const double* A, int64_t n);
double  or_norminf(const double* A, int64_t n);
double  or_est_inv_norm1_lu(const double* LU, const int64_t* ipiv, int64_t n);
double  or_est_inv_norm1_chol(const double* L, int64_t n);
double  or_est_inv_norm1_tri(const double* T, int64_t n, int lower);
double  or_est_inv_norm1_band(const double* AB, int64_t ldab, int64_t n, int64_t kl,
                              int64_t ku, const int64_t* ipiv);
double  or_est_inv_norm1_gt(const double* dl, const double* d, const double* du,
                            const double* du2, const int64_t* ipiv, int64_t n);
double  or_est_inv_norm1_ldlt(const double* F, const int64_t* ipiv, int64_t n);
double  or_rcond_from(double anorm, double ainvnm);

/* One-sided Jacobi SVD: on return G = A V (columns u_i*sigma_i), V orthogonal,
 * sigma[i] = ||G(:,i)||_2.  Returns the number of sweeps used. */
int     or_jacobi_svd(double* G, double* V, double* sigma, int64_t n, int max_sweeps);
/* Minimum-norm solve through the SVD (Sec. 2.5).  Returns the rank kept. */
int64_t or_svd_solve(const double* A, int64_t n, const double* B, int64_t nrhs,
                     double trunc_rel, double* X);

/* Residual R = B - A X with compensated (Dot2) accumulation and the per
 * column normwise backward error berr[c] = ||r||inf / (||A||inf ||x||inf + ||b||inf). */
void    or_residual_dot2(const double* A, int64_t n, const double* X, const double* B,
                         int64_t nrhs, double* R, double* berr);

/* The whole adaptive solve: scan, route, factor, solve, rcond, SVD fallback. */
int     or_solve(const double* A, const double* B, int64_t n, int64_t nrhs,
                 uint32_t flags, const or_config_t* cfg, double* X, or_info_t* info);
/* Same, for a matrix given only in band storage (declared kl, ku). */
int     or_solve_band(const double* AB, int64_t ldab, int64_t kl, int64_t ku,
                      const double* B, int64_t n, int64_t nrhs, uint32_t flags,
                      const or_config_t* cfg, double* X, or_info_t* info);

#ifdef __cplusplus
}
#endif
#endif
