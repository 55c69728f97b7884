/*
 * asolve_oracle.c -- plain, slow, FP64 CPU oracle of the adaptive solver in
 * Sanderson & Curtin, "An Adaptive Solver for Systems of Linear Equations"
 * (arXiv 2007.11208).
 *
 * TEST INFRASTRUCTURE ONLY: the checker that the GPU library is compared
 * against.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark load it.  It shares no code with the GPU library.
 *
 * Every routine is the unblocked textbook form of the step it stands for,
 * in the paper's order; there is no blocking, fusion or reordering.  It is
 * compiled with -ffp-contract=off so that every expression is evaluated as
 * written in IEEE double precision (fma() is called only where the
 * compensated residual needs an exact product error).
 *
 * Readings of the paper taken here (where it is silent or ambiguous):
 *  - "non-zero" means a != 0.0 (so -0.0 counts as zero, NaN as non-zero);
 *  - kl/ku are always computed over the whole matrix; the early stop of
 *    Sec. 2.1 changes only the speed of the check, not its outcome;
 *  - the 25% rule counts band positions: not banded iff
 *    band_count > band_frac * n^2, band_count = n(kl+ku+1) - kl(kl+1)/2
 *    - ku(ku+1)/2;
 *  - lower is tested before upper (so a diagonal matrix too small to be
 *    banded is solved as lower triangular);
 *  - rcond is LAPACK's 1-norm estimate (Hager 1984, Higham 1988) through
 *    the factors of the route taken, rcond = (1/est)/||A||_1;
 *  - the SVD fallback truncates at tau = svd_trunc_rel * sigma_max
 *    (default n*eps) and keeps sigma_i > tau;
 *  - any Inf/NaN in A or B is an error before routing.
 */
#include "asolve_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define EPS DBL_EPSILON /* 2^-52: Sec. 2.3 footnote (machine epsilon) */
#define AT(A, n, i, j) ((A)[(size_t)(i) + (size_t)(j) * (size_t)(n)])

void or_default_config(or_config_t* cfg) {
  cfg->rcond_threshold = 0.5 * EPS; /* Sec. 2.5: "0.5 epsilon" following LAPACK */
  cfg->sympd_tol = 100.0 * EPS;     /* Fig. 4: tolerance 100*eps */
  cfg->band_frac = 0.25;            /* Sec. 2.1: 25% threshold */
  cfg->svd_trunc_rel = 0.0;         /* 0 -> n*eps */
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.1: number of in-band positions for bandwidths kl, ku.            */
int64_t or_band_count(int64_t n, int64_t kl, int64_t ku) {
  return n * (kl + ku + 1) - kl * (kl + 1) / 2 - ku * (ku + 1) / 2;
}

/* Fig. 4 (likely_sympd), written out in the order the figure gives. */
int or_likely_sympd(const double* A, int64_t n, double tol) {
  double max_diag = 0.0;
  for (int64_t j = 0; j < n; ++j) { /* diagonal pass */
    double d = AT(A, n, j, j);
    if (d <= 0.0) return 0;
    if (d > max_diag) max_diag = d;
  }
  for (int64_t j = 0; j + 1 < n; ++j) { /* lower-triangle pass */
    for (int64_t i = j + 1; i < n; ++i) {
      double a_ij = AT(A, n, i, j), a_ji = AT(A, n, j, i);
      double delta = fabs(a_ij - a_ji);
      double mx = fabs(a_ij) > fabs(a_ji) ? fabs(a_ij) : fabs(a_ji);
      if (delta > tol && delta > tol * mx) return 0;          /* symmetry */
      if (fabs(a_ij) >= max_diag) return 0;                   /* max modulus */
      if ((fabs(a_ij) + fabs(a_ji)) >= (AT(A, n, i, i) + AT(A, n, j, j)))
        return 0;                                             /* dominance */
    }
  }
  return 1;
}

double or_norm1(const double* A, int64_t n) {
  double best = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += fabs(AT(A, n, i, j));
    if (s > best) best = s;
  }
  return best;
}

double or_norminf(const double* A, int64_t n) {
  double best = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j) s += fabs(AT(A, n, i, j));
    if (s > best) best = s;
  }
  return best;
}

/* Sec. 2.1 (bandwidths by column traversal), Sec. 2.2 (triangular check),
 * Fig. 4 (likely_sympd), then the detection order of Sec. 2. */
void or_scan(const double* A, int64_t n, const or_config_t* cfg, or_scan_t* out) {
  memset(out, 0, sizeof(*out));
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i)
      if (!isfinite(AT(A, n, i, j))) out->nonfinite = 1;
  int64_t kl = 0, ku = 0;
  for (int64_t j = 0; j < n; ++j) {
    /* super-diagonals: from the top of column j down to the diagonal, the
       first non-zero element fixes the distance j - i */
    for (int64_t i = 0; i < j; ++i)
      if (AT(A, n, i, j) != 0.0) {
        if (j - i > ku) ku = j - i;
        break;
      }
    /* sub-diagonals: from the bottom of column j up to the diagonal, the
       last non-zero element fixes the distance i - j */
    for (int64_t i = n - 1; i > j; --i)
      if (AT(A, n, i, j) != 0.0) {
        if (i - j > kl) kl = i - j;
        break;
      }
  }
  out->kl = kl;
  out->ku = ku;
  /* triangular structure, checked element by element as Sec. 2.2 states */
  int lower = 1, upper = 1;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) {
      if (i < j && AT(A, n, i, j) != 0.0) lower = 0;
      if (i > j && AT(A, n, i, j) != 0.0) upper = 0;
    }
  out->lower = lower;
  out->upper = upper;
  out->sympd = or_likely_sympd(A, n, cfg->sympd_tol);
  int64_t cnt = or_band_count(n, kl, ku);
  out->banded = ((double)cnt <= cfg->band_frac * (double)n * (double)n);
  out->norm1 = or_norm1(A, n);
  out->norminf = or_norminf(A, n);
  if (n == 0) out->cls = OR_CLS_NONE;
  else if (out->banded) out->cls = OR_CLS_BANDED;
  else if (lower) out->cls = OR_CLS_LOWER;
  else if (upper) out->cls = OR_CLS_UPPER;
  else if (out->sympd) out->cls = OR_CLS_SYMPD;
  else out->cls = OR_CLS_GENERAL;
}

void or_scan_many(const double* A, int64_t n, int64_t count, const or_config_t* cfg,
                  or_scan_t* out) {
  for (int64_t c = 0; c < count; ++c) or_scan(A + (size_t)c * n * n, n, cfg, out + c);
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.4: A = P L U by right-looking Gaussian elimination with partial
 * pivoting (the pivot is the first row holding the largest |a|). */
int or_lu_factor(double* A, int64_t n, int64_t* ipiv) {
  for (int64_t k = 0; k < n; ++k) {
    int64_t p = k;
    double amax = fabs(AT(A, n, k, k));
    for (int64_t i = k + 1; i < n; ++i)
      if (fabs(AT(A, n, i, k)) > amax) { amax = fabs(AT(A, n, i, k)); p = i; }
    ipiv[k] = p;
    if (AT(A, n, p, k) == 0.0) return (int)(k + 1);
    if (p != k)
      for (int64_t j = 0; j < n; ++j) {
        double t = AT(A, n, k, j);
        AT(A, n, k, j) = AT(A, n, p, j);
        AT(A, n, p, j) = t;
      }
    for (int64_t i = k + 1; i < n; ++i) AT(A, n, i, k) = AT(A, n, i, k) / AT(A, n, k, k);
    for (int64_t j = k + 1; j < n; ++j)
      for (int64_t i = k + 1; i < n; ++i)
        AT(A, n, i, j) = AT(A, n, i, j) - AT(A, n, i, k) * AT(A, n, k, j);
  }
  return 0;
}

/* Eq. 4: L (U x) = b, forward then back substitution (trans: A^T x = b). */
void or_lu_solve(const double* LU, const int64_t* ipiv, int64_t n, double* B,
                 int64_t nrhs, int trans) {
  for (int64_t c = 0; c < nrhs; ++c) {
    double* b = B + (size_t)c * n;
    if (!trans) {
      for (int64_t k = 0; k < n; ++k) {
        double t = b[k]; b[k] = b[ipiv[k]]; b[ipiv[k]] = t;
      }
      for (int64_t i = 0; i < n; ++i) { /* L y = Pb, unit diagonal */
        double s = b[i];
        for (int64_t j = 0; j < i; ++j) s = s - AT(LU, n, i, j) * b[j];
        b[i] = s;
      }
      for (int64_t i = n - 1; i >= 0; --i) { /* U x = y */
        double s = b[i];
        for (int64_t j = i + 1; j < n; ++j) s = s - AT(LU, n, i, j) * b[j];
        b[i] = s / AT(LU, n, i, i);
      }
    } else {
      for (int64_t i = 0; i < n; ++i) { /* U^T z = b */
        double s = b[i];
        for (int64_t j = 0; j < i; ++j) s = s - AT(LU, n, j, i) * b[j];
        b[i] = s / AT(LU, n, i, i);
      }
      for (int64_t i = n - 1; i >= 0; --i) { /* L^T w = z */
        double s = b[i];
        for (int64_t j = i + 1; j < n; ++j) s = s - AT(LU, n, j, i) * b[j];
        b[i] = s;
      }
      for (int64_t k = n - 1; k >= 0; --k) { /* x = P w */
        double t = b[k]; b[k] = b[ipiv[k]]; b[ipiv[k]] = t;
      }
    }
  }
}

/* Sec. 2.3 (xPOTRF): A = L L^T from the lower triangle, column by column;
 * fails when a pivot is not > 0 (which also catches NaN). */
int or_chol_factor(double* A, int64_t n) {
  for (int64_t j = 0; j < n; ++j) {
    double d = AT(A, n, j, j);
    for (int64_t k = 0; k < j; ++k) d = d - AT(A, n, j, k) * AT(A, n, j, k);
    if (!(d > 0.0)) return (int)(j + 1);
    double ljj = sqrt(d);
    AT(A, n, j, j) = ljj;
    for (int64_t i = j + 1; i < n; ++i) {
      double s = AT(A, n, i, j);
      for (int64_t k = 0; k < j; ++k) s = s - AT(A, n, i, k) * AT(A, n, j, k);
      AT(A, n, i, j) = s / ljj;
    }
  }
  return 0;
}

void or_chol_solve(const double* L, int64_t n, double* B, int64_t nrhs) {
  for (int64_t c = 0; c < nrhs; ++c) {
    double* b = B + (size_t)c * n;
    for (int64_t i = 0; i < n; ++i) { /* L y = b */
      double s = b[i];
      for (int64_t j = 0; j < i; ++j) s = s - AT(L, n, i, j) * b[j];
      b[i] = s / AT(L, n, i, i);
    }
    for (int64_t i = n - 1; i >= 0; --i) { /* L^T x = y */
      double s = b[i];
      for (int64_t j = i + 1; j < n; ++j) s = s - AT(L, n, j, i) * b[j];
      b[i] = s / AT(L, n, i, i);
    }
  }
}

/* Eq. 3 (forward substitution) and its mirror image (back substitution).
 * trans solves T^T x = b.  Returns k+1 if T(k,k) == 0 (singular). */
int or_tri_solve(const double* T, int64_t n, int lower, double* B, int64_t nrhs,
                 int trans) {
  for (int64_t k = 0; k < n; ++k)
    if (AT(T, n, k, k) == 0.0) return (int)(k + 1);
  int fwd = trans ? !lower : lower; /* T^T of a lower matrix is upper */
  for (int64_t c = 0; c < nrhs; ++c) {
    double* b = B + (size_t)c * n;
    if (fwd) {
      for (int64_t i = 0; i < n; ++i) {
        double s = b[i];
        for (int64_t j = 0; j < i; ++j)
          s = s - (trans ? AT(T, n, j, i) : AT(T, n, i, j)) * b[j];
        b[i] = s / AT(T, n, i, i);
      }
    } else {
      for (int64_t i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int64_t j = i + 1; j < n; ++j)
          s = s - (trans ? AT(T, n, j, i) : AT(T, n, i, j)) * b[j];
        b[i] = s / AT(T, n, i, i);
      }
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.1: band storage.  Element (i,j) of A at BAND(i,j) =
 * AB[(kl+ku+i-j) + j*ldab]; the top kl rows are fill room for U. */
#define BAND(AB, ldab, kv, i, j) ((AB)[(size_t)((kv) + (i) - (j)) + (size_t)(j) * (size_t)(ldab)])

void or_band_pack(const double* A, int64_t n, int64_t kl, int64_t ku, double* AB,
                  int64_t ldab) {
  int64_t kv = kl + ku;
  memset(AB, 0, sizeof(double) * (size_t)ldab * (size_t)n);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = (j - ku > 0 ? j - ku : 0); i <= j + kl && i < n; ++i)
      BAND(AB, ldab, kv, i, j) = AT(A, n, i, j);
}

/* Sec. 2.1 (xGBTRF): LU with partial pivoting restricted to the band; the
 * pivot is searched among the kl rows below the diagonal and U grows up
 * to kl+ku super-diagonals. */
int or_band_lu_factor(double* AB, int64_t ldab, int64_t n, int64_t kl, int64_t ku,
                      int64_t* ipiv) {
  int64_t kv = kl + ku, ju = 0;
  for (int64_t j = 0; j < n; ++j) {
    int64_t km = kl < n - 1 - j ? kl : n - 1 - j;
    int64_t jp = 0;
    double amax = fabs(BAND(AB, ldab, kv, j, j));
    for (int64_t t = 1; t <= km; ++t)
      if (fabs(BAND(AB, ldab, kv, j + t, j)) > amax) {
        amax = fabs(BAND(AB, ldab, kv, j + t, j));
        jp = t;
      }
    ipiv[j] = j + jp;
    if (BAND(AB, ldab, kv, j + jp, j) == 0.0) return (int)(j + 1);
    int64_t reach = j + ku + jp < n - 1 ? j + ku + jp : n - 1;
    if (reach > ju) ju = reach;
    if (jp != 0)
      for (int64_t c = j; c <= ju; ++c) {
        double t = BAND(AB, ldab, kv, j, c);
        BAND(AB, ldab, kv, j, c) = BAND(AB, ldab, kv, j + jp, c);
        BAND(AB, ldab, kv, j + jp, c) = t;
      }
    for (int64_t t = 1; t <= km; ++t)
      BAND(AB, ldab, kv, j + t, j) = BAND(AB, ldab, kv, j + t, j) / BAND(AB, ldab, kv, j, j);
    for (int64_t c = j + 1; c <= ju; ++c)
      for (int64_t t = 1; t <= km; ++t)
        BAND(AB, ldab, kv, j + t, c) =
            BAND(AB, ldab, kv, j + t, c) - BAND(AB, ldab, kv, j + t, j) * BAND(AB, ldab, kv, j, c);
  }
  return 0;
}

/* Sec. 2.1 (xGBTRS): solve with the band factors (trans: A^T x = b). */
void or_band_lu_solve(const double* AB, int64_t ldab, int64_t n, int64_t kl, int64_t ku,
                      const int64_t* ipiv, double* B, int64_t nrhs, int trans) {
  int64_t kv = kl + ku;
  for (int64_t c = 0; c < nrhs; ++c) {
    double* b = B + (size_t)c * n;
    if (!trans) {
      for (int64_t j = 0; j < n; ++j) { /* apply P_j then L_j */
        int64_t km = kl < n - 1 - j ? kl : n - 1 - j;
        double t = b[j]; b[j] = b[ipiv[j]]; b[ipiv[j]] = t;
        for (int64_t s = 1; s <= km; ++s) b[j + s] = b[j + s] - BAND(AB, ldab, kv, j + s, j) * b[j];
      }
      for (int64_t i = n - 1; i >= 0; --i) { /* U x = y, bandwidth kv */
        double s = b[i];
        for (int64_t j = i + 1; j <= i + kv && j < n; ++j) s = s - BAND(AB, ldab, kv, i, j) * b[j];
        b[i] = s / BAND(AB, ldab, kv, i, i);
      }
    } else {
      for (int64_t i = 0; i < n; ++i) { /* U^T z = b */
        double s = b[i];
        for (int64_t j = (i - kv > 0 ? i - kv : 0); j < i; ++j) s = s - BAND(AB, ldab, kv, j, i) * b[j];
        b[i] = s / BAND(AB, ldab, kv, i, i);
      }
      for (int64_t j = n - 1; j >= 0; --j) { /* L_j^T then P_j, in reverse */
        int64_t km = kl < n - 1 - j ? kl : n - 1 - j;
        double s = b[j];
        for (int64_t t = 1; t <= km; ++t) s = s - BAND(AB, ldab, kv, j + t, j) * b[j + t];
        b[j] = s;
        double t = b[j]; b[j] = b[ipiv[j]]; b[ipiv[j]] = t;
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Tridiagonal systems, the closing remarks' specialisation of the banded
 * case: Gaussian elimination with partial pivoting on the three diagonals
 * (xGTTRF semantics).  At step i only rows i and i+1 hold entries of column
 * i; they are interchanged when |dl[i]| > |d[i]| (a tie keeps row i, the
 * first maximum).  An interchange brings the second super-diagonal entry
 * du2[i] of the new row i.  The multiplier is the entry divided by the
 * pivot.  Returns 0, or i+1 at the first exact zero pivot d[i]. */
int or_gt_factor(double* dl, double* d, double* du, double* du2, int64_t* ipiv, int64_t n) {
  for (int64_t i = 0; i < n; ++i) ipiv[i] = i;
  for (int64_t i = 0; i + 2 < n; ++i) du2[i] = 0.0;
  for (int64_t i = 0; i + 1 < n; ++i) {
    if (fabs(d[i]) >= fabs(dl[i])) { /* no interchange */
      if (d[i] != 0.0) {
        double l = dl[i] / d[i];
        dl[i] = l;
        d[i + 1] = d[i + 1] - l * du[i];
      }
    } else { /* rows i and i+1 interchanged */
      double l = d[i] / dl[i];
      d[i] = dl[i];
      dl[i] = l;
      double t = du[i];
      du[i] = d[i + 1];
      d[i + 1] = t - l * d[i + 1];
      if (i + 2 < n) {
        du2[i] = du[i + 1];
        du[i + 1] = -(l * du[i + 1]);
      }
      ipiv[i] = i + 1;
    }
  }
  for (int64_t i = 0; i < n; ++i)
    if (d[i] == 0.0) return (int)(i + 1);
  return 0;
}

/* Solve with the tridiagonal factors (xGTTRS semantics; trans: A^T x = b). */
void or_gt_solve(const double* dl, const double* d, const double* du, const double* du2,
                 const int64_t* ipiv, int64_t n, double* B, int64_t nrhs, int trans) {
  for (int64_t c = 0; c < nrhs; ++c) {
    double* b = B + (size_t)c * n;
    if (!trans) {
      for (int64_t i = 0; i + 1 < n; ++i) { /* L y = P b */
        if (ipiv[i] == i) {
          b[i + 1] = b[i + 1] - dl[i] * b[i];
        } else {
          double t = b[i];
          b[i] = b[i + 1];
          b[i + 1] = t - dl[i] * b[i];
        }
      }
      for (int64_t i = n - 1; i >= 0; --i) { /* U x = y: d, du, du2 */
        double s = b[i];
        if (i + 1 < n) s = s - du[i] * b[i + 1];
        if (i + 2 < n) s = s - du2[i] * b[i + 2];
        b[i] = s / d[i];
      }
    } else {
      for (int64_t i = 0; i < n; ++i) { /* U^T z = b */
        double s = b[i];
        if (i >= 1) s = s - du[i - 1] * b[i - 1];
        if (i >= 2) s = s - du2[i - 2] * b[i - 2];
        b[i] = s / d[i];
      }
      for (int64_t i = n - 2; i >= 0; --i) { /* L^T then P^T, in reverse */
        if (ipiv[i] == i) {
          b[i] = b[i] - dl[i] * b[i + 1];
        } else {
          double t = b[i + 1];
          b[i + 1] = b[i] - dl[i] * t;
          b[i] = t;
        }
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Plain symmetric (not positive definite) systems, the closing remarks'
 * other specialisation.  Symmetry is the Fig. 4 test on its own. */
int or_is_symmetric(const double* A, int64_t n, double tol) {
  for (int64_t j = 0; j + 1 < n; ++j)
    for (int64_t i = j + 1; i < n; ++i) {
      double a_ij = AT(A, n, i, j), a_ji = AT(A, n, j, i);
      double delta = fabs(a_ij - a_ji);
      double mx = fabs(a_ij) > fabs(a_ji) ? fabs(a_ij) : fabs(a_ji);
      if (delta > tol && delta > tol * mx) return 0;
    }
  return 1;
}

static void swap_d(double* a, double* b) { double t = *a; *a = *b; *b = t; }

/* Bunch-Kaufman LDL^T of the lower triangle, column by column (Bunch &
 * Kaufman 1977, the partial-pivoting variant LAPACK's xSYTRF uses): with
 * alpha = (1 + sqrt 17)/8, colmax the largest off-diagonal modulus of
 * column k (at row imax) and rowmax the largest off-diagonal modulus of
 * row/column imax of the trailing matrix,
 *   |a_kk| >= alpha colmax                    -> 1 x 1 pivot a_kk;
 *   |a_kk| rowmax >= alpha colmax^2           -> 1 x 1 pivot a_kk;
 *   |a_imax,imax| >= alpha rowmax             -> 1 x 1 pivot a_imax,imax (k <-> imax);
 *   otherwise                                 -> 2 x 2 pivot on (k, imax) (k+1 <-> imax).
 * After the symmetric interchange the trailing matrix is updated with the
 * pivot block E: A22 -= C E^-1 C^T, and the multipliers C E^-1 stored as L. */
int or_ldlt_factor(double* A, int64_t n, int64_t* ipiv) {
#define LT(i, j) A[(size_t)(i) + (size_t)(j) * (size_t)n]
  const double alpha = (1.0 + sqrt(17.0)) / 8.0;
  int info = 0;
  int64_t k = 0;
  while (k < n) {
    int64_t kstep = 1, kp = k, imax = k;
    const double absakk = fabs(LT(k, k));
    double colmax = 0.0;
    for (int64_t i = k + 1; i < n; ++i)
      if (fabs(LT(i, k)) > colmax) { colmax = fabs(LT(i, k)); imax = i; }
    if (absakk == 0.0 && colmax == 0.0) { /* a zero column: D(k) = 0 */
      if (!info) info = (int)(k + 1);
      ipiv[k] = k;
      k += 1;
      continue;
    }
    if (absakk < alpha * colmax) {
      double rowmax = 0.0;
      for (int64_t j = k; j < imax; ++j) rowmax = fmax(rowmax, fabs(LT(imax, j)));
      for (int64_t i = imax + 1; i < n; ++i) rowmax = fmax(rowmax, fabs(LT(i, imax)));
      if (absakk >= alpha * colmax * (colmax / rowmax)) kp = k;
      else if (fabs(LT(imax, imax)) >= alpha * rowmax) kp = imax;
      else { kp = imax; kstep = 2; }
    }
    const int64_t kk = k + kstep - 1; /* the row/column brought to kp's place */
    if (kp != kk) { /* symmetric interchange of kk and kp, lower triangle */
      for (int64_t i = kp + 1; i < n; ++i) swap_d(&LT(i, kk), &LT(i, kp));
      for (int64_t j = kk + 1; j < kp; ++j) swap_d(&LT(j, kk), &LT(kp, j));
      swap_d(&LT(kk, kk), &LT(kp, kp));
      if (kstep == 2) swap_d(&LT(k + 1, k), &LT(kp, k));
    }
    if (kstep == 1) {
      const double d = LT(k, k);
      for (int64_t j = k + 1; j < n; ++j) {
        const double lj = LT(j, k) / d;
        for (int64_t i = j; i < n; ++i) LT(i, j) = LT(i, j) - LT(i, k) * lj;
      }
      for (int64_t i = k + 1; i < n; ++i) LT(i, k) = LT(i, k) / d;
      ipiv[k] = kp;
    } else {
      /* E = [a b; b c], E^-1 = [c -b; -b a] / (a c - b^2) */
      const double a = LT(k, k), b = LT(k + 1, k), c = LT(k + 1, k + 1);
      const double det = a * c - b * b;
      for (int64_t j = k + 2; j < n; ++j) {
        const double w0 = (c * LT(j, k) - b * LT(j, k + 1)) / det;
        const double w1 = (a * LT(j, k + 1) - b * LT(j, k)) / det;
        for (int64_t i = j; i < n; ++i) LT(i, j) = LT(i, j) - LT(i, k) * w0 - LT(i, k + 1) * w1;
        LT(j, k) = w0;
        LT(j, k + 1) = w1;
      }
      ipiv[k] = ipiv[k + 1] = -(kp + 1);
    }
    k += kstep;
  }
  return info;
#undef LT
}

/* Solve with the LDL^T factors: x = P^T L^-T D^-1 L^-1 P b, the
 * interchanges applied in the factorisation's order on the way in and in
 * reverse on the way out. */
void or_ldlt_solve(const double* F, const int64_t* ipiv, int64_t n, double* B, int64_t nrhs) {
#define LT(i, j) F[(size_t)(i) + (size_t)(j) * (size_t)n]
  for (int64_t c = 0; c < nrhs; ++c) {
    double* b = B + (size_t)c * n;
    int64_t k = 0;
    while (k < n) { /* L D y = P b */
      if (ipiv[k] >= 0) {
        const int64_t kp = ipiv[k];
        if (kp != k) swap_d(&b[k], &b[kp]);
        for (int64_t i = k + 1; i < n; ++i) b[i] = b[i] - LT(i, k) * b[k];
        b[k] = b[k] / LT(k, k);
        k += 1;
      } else {
        const int64_t kp = -ipiv[k] - 1;
        if (kp != k + 1) swap_d(&b[k + 1], &b[kp]);
        for (int64_t i = k + 2; i < n; ++i) b[i] = b[i] - LT(i, k) * b[k] - LT(i, k + 1) * b[k + 1];
        const double a = LT(k, k), bb = LT(k + 1, k), cc = LT(k + 1, k + 1);
        const double det = a * cc - bb * bb;
        const double y0 = b[k], y1 = b[k + 1];
        b[k] = (cc * y0 - bb * y1) / det;
        b[k + 1] = (a * y1 - bb * y0) / det;
        k += 2;
      }
    }
    k = n - 1;
    while (k >= 0) { /* L^T x = y, then P^T */
      if (ipiv[k] >= 0) {
        double s = b[k];
        for (int64_t i = k + 1; i < n; ++i) s = s - LT(i, k) * b[i];
        b[k] = s;
        const int64_t kp = ipiv[k];
        if (kp != k) swap_d(&b[k], &b[kp]);
        k -= 1;
      } else { /* the 2 x 2 block (k-1, k) */
        double s1 = b[k], s0 = b[k - 1];
        for (int64_t i = k + 1; i < n; ++i) {
          s1 = s1 - LT(i, k) * b[i];
          s0 = s0 - LT(i, k - 1) * b[i];
        }
        b[k] = s1;
        b[k - 1] = s0;
        const int64_t kp = -ipiv[k] - 1;
        if (kp != k) swap_d(&b[k], &b[kp]);
        k -= 2;
      }
    }
  }
#undef LT
}

/* ------------------------------------------------------------------------ */
/* 1-norm estimate of inv(A) (Hager 1984; Higham 1988, the estimator LAPACK's
 * xGECON/xPOCON/xGBCON/xTRCON use).  apply(ctx, x, trans) overwrites x with
 * inv(A) x (trans = 0) or inv(A)^T x (trans = 1). */
typedef void (*or_apply_fn)(const void* ctx, double* x, int trans);

static double sum_abs(const double* x, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += fabs(x[i]);
  return s;
}
static int64_t first_argmax_abs(const double* x, int64_t n) {
  int64_t j = 0;
  double m = fabs(x[0]);
  for (int64_t i = 1; i < n; ++i)
    if (fabs(x[i]) > m) { m = fabs(x[i]); j = i; }
  return j;
}

static double est_inv_norm1(int64_t n, or_apply_fn apply, const void* ctx) {
  if (n == 0) return 0.0;
  double* x = (double*)malloc(sizeof(double) * (size_t)n);
  double* xi = (double*)malloc(sizeof(double) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) x[i] = 1.0 / (double)n;
  apply(ctx, x, 0); /* v = inv(A) (e/n) */
  double est;
  if (n == 1) {
    est = fabs(x[0]);
    free(x); free(xi);
    return est;
  }
  est = sum_abs(x, n);
  for (int64_t i = 0; i < n; ++i) { xi[i] = x[i] >= 0.0 ? 1.0 : -1.0; x[i] = xi[i]; }
  apply(ctx, x, 1); /* z = inv(A)^T sign(v) */
  int k = 2;
  for (;;) {
    int64_t j = first_argmax_abs(x, n);
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    x[j] = 1.0;
    apply(ctx, x, 0); /* v = inv(A) e_j */
    double estold = est;
    est = sum_abs(x, n);
    int same = 1;
    for (int64_t i = 0; i < n; ++i)
      if ((x[i] >= 0.0 ? 1.0 : -1.0) != xi[i]) { same = 0; break; }
    if (same || est <= estold) break; /* converged or cycling */
    for (int64_t i = 0; i < n; ++i) { xi[i] = x[i] >= 0.0 ? 1.0 : -1.0; x[i] = xi[i]; }
    apply(ctx, x, 1);
    int64_t jnew = first_argmax_abs(x, n);
    ++k;
    if (x[j] == fabs(x[jnew]) || k > 5) break;
  }
  /* alternating-sign test vector x_i = (-1)^i (1 + i/(n-1)), 0-based */
  double sgn = 1.0;
  for (int64_t i = 0; i < n; ++i) {
    x[i] = sgn * (1.0 + (double)i / (double)(n - 1));
    sgn = -sgn;
  }
  apply(ctx, x, 0);
  double temp = 2.0 * sum_abs(x, n) / (double)(3 * n);
  if (temp > est) est = temp;
  free(x); free(xi);
  return est;
}

typedef struct { const double* F; const int64_t* ipiv; int64_t n, ldab, kl, ku; int lower; } fac_ctx;

static void apply_lu(const void* c, double* x, int trans) {
  const fac_ctx* f = (const fac_ctx*)c;
  or_lu_solve(f->F, f->ipiv, f->n, x, 1, trans);
}
static void apply_chol(const void* c, double* x, int trans) {
  (void)trans; /* inv(A) is symmetric */
  const fac_ctx* f = (const fac_ctx*)c;
  or_chol_solve(f->F, f->n, x, 1);
}
static void apply_tri(const void* c, double* x, int trans) {
  const fac_ctx* f = (const fac_ctx*)c;
  or_tri_solve(f->F, f->n, f->lower, x, 1, trans);
}
static void apply_band(const void* c, double* x, int trans) {
  const fac_ctx* f = (const fac_ctx*)c;
  or_band_lu_solve(f->F, f->ldab, f->n, f->kl, f->ku, f->ipiv, x, 1, trans);
}

typedef struct { const double *dl, *d, *du, *du2; const int64_t* ipiv; int64_t n; } gt_ctx;
static void apply_gt(const void* c, double* x, int trans) {
  const gt_ctx* f = (const gt_ctx*)c;
  or_gt_solve(f->dl, f->d, f->du, f->du2, f->ipiv, f->n, x, 1, trans);
}
double or_est_inv_norm1_gt(const double* dl, const double* d, const double* du,
                           const double* du2, const int64_t* ipiv, int64_t n) {
  gt_ctx f = {dl, d, du, du2, ipiv, n};
  return est_inv_norm1(n, apply_gt, &f);
}

static void apply_ldlt(const void* c, double* x, int trans) {
  (void)trans; /* inv(A) is symmetric */
  const fac_ctx* f = (const fac_ctx*)c;
  or_ldlt_solve(f->F, f->ipiv, f->n, x, 1);
}
double or_est_inv_norm1_ldlt(const double* F, const int64_t* ipiv, int64_t n) {
  fac_ctx f = {F, ipiv, n, 0, 0, 0, 0};
  return est_inv_norm1(n, apply_ldlt, &f);
}

double or_est_inv_norm1_lu(const double* LU, const int64_t* ipiv, int64_t n) {
  fac_ctx f = {LU, ipiv, n, 0, 0, 0, 0};
  return est_inv_norm1(n, apply_lu, &f);
}
double or_est_inv_norm1_chol(const double* L, int64_t n) {
  fac_ctx f = {L, NULL, n, 0, 0, 0, 0};
  return est_inv_norm1(n, apply_chol, &f);
}
double or_est_inv_norm1_tri(const double* T, int64_t n, int lower) {
  fac_ctx f = {T, NULL, n, 0, 0, 0, lower};
  return est_inv_norm1(n, apply_tri, &f);
}
double or_est_inv_norm1_band(const double* AB, int64_t ldab, int64_t n, int64_t kl,
                             int64_t ku, const int64_t* ipiv) {
  fac_ctx f = {AB, ipiv, n, ldab, kl, ku, 0};
  return est_inv_norm1(n, apply_band, &f);
}

/* rcond = (1/||inv(A)||_1) / ||A||_1, with 0 for a zero norm or an
 * infinite estimate. */
double or_rcond_from(double anorm, double ainvnm) {
  if (anorm == 0.0 || isinf(ainvnm)) return 0.0;
  if (ainvnm == 0.0) return 0.0;
  return (1.0 / ainvnm) / anorm;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.5: one-sided Jacobi SVD (Hestenes 1958), cyclic-by-rows order.
 * A pair of columns is rotated when |g_i.g_j| > n*eps*||g_i||*||g_j||; the
 * sweeps stop after one without a rotation, or after max_sweeps. */
int or_jacobi_svd(double* G, double* V, double* sigma, int64_t n, int max_sweeps) {
  double tol = (double)n * EPS;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) AT(V, n, i, j) = (i == j) ? 1.0 : 0.0;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    int rotated = 0;
    for (int64_t p = 0; p + 1 < n; ++p)
      for (int64_t q = p + 1; q < n; ++q) {
        double alpha = 0.0, beta = 0.0, gamma = 0.0;
        for (int64_t k = 0; k < n; ++k) {
          alpha += AT(G, n, k, p) * AT(G, n, k, p);
          beta += AT(G, n, k, q) * AT(G, n, k, q);
          gamma += AT(G, n, k, p) * AT(G, n, k, q);
        }
        if (!(fabs(gamma) > tol * sqrt(alpha) * sqrt(beta))) continue;
        double zeta = (beta - alpha) / (2.0 * gamma);
        double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
        for (int64_t k = 0; k < n; ++k) {
          double gp = AT(G, n, k, p), gq = AT(G, n, k, q);
          AT(G, n, k, p) = c * gp - s * gq;
          AT(G, n, k, q) = s * gp + c * gq;
          double vp = AT(V, n, k, p), vq = AT(V, n, k, q);
          AT(V, n, k, p) = c * vp - s * vq;
          AT(V, n, k, q) = s * vp + c * vq;
        }
        rotated = 1;
      }
    if (!rotated) break;
  }
  for (int64_t j = 0; j < n; ++j) {
    double s = 0.0;
    for (int64_t k = 0; k < n; ++k) s += AT(G, n, k, j) * AT(G, n, k, j);
    sigma[j] = sqrt(s);
  }
  return sweep;
}

/* Sec. 2.5 (xGELSD): minimum-norm solution x = V pinv(Sigma) U^T b with
 * u_i = g_i / sigma_i, keeping sigma_i > tau = trunc_rel * sigma_max. */
int64_t or_svd_solve(const double* A, int64_t n, const double* B, int64_t nrhs,
                     double trunc_rel, double* X) {
  double* G = (double*)malloc(sizeof(double) * (size_t)n * n);
  double* V = (double*)malloc(sizeof(double) * (size_t)n * n);
  double* sig = (double*)malloc(sizeof(double) * (size_t)n);
  memcpy(G, A, sizeof(double) * (size_t)n * n);
  or_jacobi_svd(G, V, sig, n, 30);
  double smax = 0.0;
  for (int64_t i = 0; i < n; ++i) if (sig[i] > smax) smax = sig[i];
  double tau = (trunc_rel > 0.0 ? trunc_rel : (double)n * EPS) * smax;
  int64_t rank = 0;
  for (int64_t i = 0; i < n; ++i) if (sig[i] > tau) ++rank;
  for (int64_t c = 0; c < nrhs; ++c) {
    const double* b = B + (size_t)c * n;
    double* x = X + (size_t)c * n;
    for (int64_t k = 0; k < n; ++k) x[k] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      if (!(sig[i] > tau)) continue;
      double d = 0.0;
      for (int64_t k = 0; k < n; ++k) d += (AT(G, n, k, i) / sig[i]) * b[k];
      double w = d / sig[i];
      for (int64_t k = 0; k < n; ++k) x[k] += AT(V, n, k, i) * w;
    }
  }
  free(G); free(V); free(sig);
  return rank;
}

/* ------------------------------------------------------------------------ */
/* Compensated residual (Dot2 of Ogita, Rump and Oishi 2005). */
static void two_sum(double a, double b, double* s, double* e) {
  double x = a + b, z = x - a;
  *s = x;
  *e = (a - (x - z)) + (b - z);
}

void or_residual_dot2(const double* A, int64_t n, const double* X, const double* B,
                      int64_t nrhs, double* R, double* berr) {
  double anorm = or_norminf(A, n);
  for (int64_t c = 0; c < nrhs; ++c) {
    const double* x = X + (size_t)c * n;
    const double* b = B + (size_t)c * n;
    double* r = R + (size_t)c * n;
    double rmax = 0.0, xmax = 0.0, bmax = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      double s = b[i], comp = 0.0;
      for (int64_t j = 0; j < n; ++j) {
        double p = AT(A, n, i, j) * x[j];
        double pe = fma(AT(A, n, i, j), x[j], -p); /* exact: a*x = p + pe */
        double es;
        two_sum(s, -p, &s, &es);
        comp = comp + (es - pe);
      }
      r[i] = s + comp;
      if (fabs(r[i]) > rmax) rmax = fabs(r[i]);
      if (fabs(x[i]) > xmax) xmax = fabs(x[i]);
      if (fabs(b[i]) > bmax) bmax = fabs(b[i]);
    }
    double den = anorm * xmax + bmax;
    berr[c] = den > 0.0 ? rmax / den : (rmax > 0.0 ? INFINITY : 0.0);
  }
}

/* ------------------------------------------------------------------------ */
static void info_init(or_info_t* info) {
  info->cls = OR_CLS_NONE;
  info->route = OR_ROUTE_NONE;
  info->status = OR_OK;
  info->svd_used = 0;
  info->kl = info->ku = 0;
  info->rcond = NAN;
  info->svd_rank = -1;
}

static int all_finite(const double* x, size_t cnt) {
  for (size_t i = 0; i < cnt; ++i) if (!isfinite(x[i])) return 0;
  return 1;
}

/* After the primary route: Sec. 2.5 -- a failed solver, or rcond below the
 * threshold (or NaN), sends the system to the SVD solver unless the
 * caller disabled it. */
static int finish(const double* A, const double* B, int64_t n, int64_t nrhs,
                  uint32_t flags, const or_config_t* cfg, int failed, double* X,
                  or_info_t* info) {
  int poor = !failed && !(flags & OR_NO_RCOND) && !(info->rcond >= cfg->rcond_threshold);
  if (!failed && !poor) { info->status = OR_OK; return OR_OK; }
  if (flags & OR_NO_APPROX) {
    if (failed) {
      memset(X, 0, sizeof(double) * (size_t)n * nrhs);
      info->status = OR_E_SINGULAR;
    } else {
      info->status = OR_W_ILLCOND;
    }
    return info->status;
  }
  if (!A) { /* band input too large to densify */
    if (failed) memset(X, 0, sizeof(double) * (size_t)n * nrhs);
    info->status = failed ? OR_E_SINGULAR : OR_W_ILLCOND;
    return info->status;
  }
  info->svd_rank = or_svd_solve(A, n, B, nrhs, cfg->svd_trunc_rel, X);
  info->svd_used = 1;
  info->status = OR_W_APPROX;
  return OR_W_APPROX;
}

static int solve_lu_route(const double* A, int64_t n, int64_t nrhs, uint32_t flags,
                          double anorm, double* X, or_info_t* info) {
  double* F = (double*)malloc(sizeof(double) * (size_t)n * n);
  int64_t* ipiv = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  memcpy(F, A, sizeof(double) * (size_t)n * n);
  int failed = or_lu_factor(F, n, ipiv) != 0;
  if (!failed) {
    or_lu_solve(F, ipiv, n, X, nrhs, 0);
    if (!(flags & OR_NO_RCOND)) info->rcond = or_rcond_from(anorm, or_est_inv_norm1_lu(F, ipiv, n));
  }
  free(F); free(ipiv);
  return failed;
}

/* The symmetric-indefinite route: LDL^T of A's lower triangle. */
static int solve_ldlt_route(const double* A, int64_t n, int64_t nrhs, uint32_t flags, double anorm,
                            double* X, or_info_t* info) {
  double* F = (double*)malloc(sizeof(double) * (size_t)n * n);
  int64_t* ipiv = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  memcpy(F, A, sizeof(double) * (size_t)n * n);
  int failed = or_ldlt_factor(F, n, ipiv) != 0;
  if (!failed) {
    or_ldlt_solve(F, ipiv, n, X, nrhs);
    if (!(flags & OR_NO_RCOND)) info->rcond = or_rcond_from(anorm, or_est_inv_norm1_ldlt(F, ipiv, n));
  }
  free(F); free(ipiv);
  return failed;
}

/* The tridiagonal route: the three diagonals of A taken from dense storage
 * (dense != 0: A(i,j) at M[i + j*n]) or from band storage with leading
 * dimension ld and declared super-diagonal count kud (A(i,j) at
 * M[(kud + i - j) + j*ld]); factor, solve X in place, estimate. */
static int solve_gt_route(const double* M, int dense, int64_t ld, int64_t kud, int64_t n, double* X,
                          int64_t nrhs, uint32_t flags, double anorm, or_info_t* info) {
  double* dl = (double*)calloc((size_t)(n > 1 ? n - 1 : 1), sizeof(double));
  double* d = (double*)calloc((size_t)n, sizeof(double));
  double* du = (double*)calloc((size_t)(n > 1 ? n - 1 : 1), sizeof(double));
  double* du2 = (double*)calloc((size_t)(n > 2 ? n - 2 : 1), sizeof(double));
  int64_t* ipiv = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    d[i] = dense ? M[(size_t)i + (size_t)i * n] : M[(size_t)kud + (size_t)i * ld];
    if (i + 1 < n) {
      dl[i] = dense ? M[(size_t)(i + 1) + (size_t)i * n] : M[(size_t)(kud + 1) + (size_t)i * ld];
      du[i] = dense ? M[(size_t)i + (size_t)(i + 1) * n] : M[(size_t)(kud - 1) + (size_t)(i + 1) * ld];
    }
  }
  int failed = or_gt_factor(dl, d, du, du2, ipiv, n) != 0;
  if (!failed) {
    or_gt_solve(dl, d, du, du2, ipiv, n, X, nrhs, 0);
    if (!(flags & OR_NO_RCOND)) info->rcond = or_rcond_from(anorm, or_est_inv_norm1_gt(dl, d, du, du2, ipiv, n));
  }
  free(dl); free(d); free(du); free(du2); free(ipiv);
  return failed;
}

int or_solve(const double* A, const double* B, int64_t n, int64_t nrhs, uint32_t flags,
             const or_config_t* cfg_in, double* X, or_info_t* info) {
  or_config_t cfg;
  if (cfg_in) cfg = *cfg_in; else or_default_config(&cfg);
  info_init(info);
  if (n < 0 || nrhs < 1 || (n > 0 && (!A || !B || !X))) { info->status = OR_E_INVALID; return OR_E_INVALID; }
  if (n == 0) return OR_OK;
  if (!all_finite(A, (size_t)n * n) || !all_finite(B, (size_t)n * nrhs)) {
    info->status = OR_E_NONFINITE;
    return OR_E_NONFINITE;
  }
  or_scan_t sc;
  or_scan(A, n, &cfg, &sc);
  info->cls = sc.cls;
  info->kl = sc.kl;
  info->ku = sc.ku;
  memcpy(X, B, sizeof(double) * (size_t)n * nrhs);
  if (flags & OR_FORCE_SVD) {
    info->route = OR_ROUTE_SVD;
    info->svd_rank = or_svd_solve(A, n, B, nrhs, cfg.svd_trunc_rel, X);
    info->svd_used = 1;
    info->status = OR_W_APPROX;
    return OR_W_APPROX;
  }
  int failed = 0;
  int cls = (flags & OR_FORCE_LU) ? OR_CLS_GENERAL : sc.cls;
  if (cls == OR_CLS_BANDED && (flags & OR_TRIDIAG) && sc.kl == 1 && sc.ku == 1) {
    /* the tridiagonal specialisation: the three diagonals */
    info->route = OR_ROUTE_TRIDIAG;
    failed = solve_gt_route(A, 1, n, 0, n, X, nrhs, flags, sc.norm1, info);
  } else if (cls == OR_CLS_BANDED) { /* Sec. 2.1 */
    info->route = OR_ROUTE_BAND_LU;
    int64_t kl = sc.kl, ku = sc.ku, ldab = 2 * kl + ku + 1;
    double* AB = (double*)malloc(sizeof(double) * (size_t)ldab * n);
    int64_t* ipiv = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    or_band_pack(A, n, kl, ku, AB, ldab);
    failed = or_band_lu_factor(AB, ldab, n, kl, ku, ipiv) != 0;
    if (!failed) {
      or_band_lu_solve(AB, ldab, n, kl, ku, ipiv, X, nrhs, 0);
      if (!(flags & OR_NO_RCOND))
        info->rcond = or_rcond_from(sc.norm1, or_est_inv_norm1_band(AB, ldab, n, kl, ku, ipiv));
    }
    free(AB); free(ipiv);
  } else if (cls == OR_CLS_LOWER || cls == OR_CLS_UPPER) { /* Sec. 2.2 */
    int lower = cls == OR_CLS_LOWER;
    info->route = lower ? OR_ROUTE_TRI_LOWER : OR_ROUTE_TRI_UPPER;
    failed = or_tri_solve(A, n, lower, X, nrhs, 0) != 0;
    if (!failed && !(flags & OR_NO_RCOND))
      info->rcond = or_rcond_from(sc.norm1, or_est_inv_norm1_tri(A, n, lower));
  } else if (cls == OR_CLS_SYMPD) { /* Sec. 2.3 */
    double* F = (double*)malloc(sizeof(double) * (size_t)n * n);
    memcpy(F, A, sizeof(double) * (size_t)n * n);
    if (or_chol_factor(F, n) == 0) {
      info->route = OR_ROUTE_CHOL;
      or_chol_solve(F, n, X, nrhs);
      if (!(flags & OR_NO_RCOND)) info->rcond = or_rcond_from(sc.norm1, or_est_inv_norm1_chol(F, n));
    } else if ((flags & OR_SYM_INDEF) && n <= OR_LDLT_NMAX) {
      /* Cholesky failure, symmetric after all: the symmetric-indefinite solver */
      info->route = OR_ROUTE_CHOL_FAIL_LDLT;
      memcpy(X, B, sizeof(double) * (size_t)n * nrhs);
      failed = solve_ldlt_route(A, n, nrhs, flags, sc.norm1, X, info);
    } else { /* Cholesky failure: not sympd after all, use the general solver */
      info->route = OR_ROUTE_CHOL_FAIL_LU;
      memcpy(X, B, sizeof(double) * (size_t)n * nrhs);
      failed = solve_lu_route(A, n, nrhs, flags, sc.norm1, X, info);
    }
    free(F);
  } else if ((flags & OR_SYM_INDEF) && !(flags & OR_FORCE_LU) && n <= OR_LDLT_NMAX &&
             or_is_symmetric(A, n, cfg.sympd_tol)) {
    /* plain symmetric, not likely_sympd: the symmetric-indefinite solver */
    info->route = OR_ROUTE_LDLT;
    failed = solve_ldlt_route(A, n, nrhs, flags, sc.norm1, X, info);
  } else { /* Sec. 2.4 */
    info->route = OR_ROUTE_LU;
    failed = solve_lu_route(A, n, nrhs, flags, sc.norm1, X, info);
  }
  return finish(A, B, n, nrhs, flags, &cfg, failed, X, info);
}

/* Band-storage input: AB holds A(i,j) at AB[(ku+i-j) + j*ldab] with
 * ldab >= kl+ku+1 (declared bandwidths).  A system given in band storage
 * always takes the banded route, with the true bandwidths found inside
 * the declared band.  The SVD fallback densifies A only for
 * n <= OR_SVD_DENSIFY_NMAX (the GPU library's limit for the same step). */
int or_solve_band(const double* AB, int64_t ldab, int64_t kl, int64_t ku, const double* B,
                  int64_t n, int64_t nrhs, uint32_t flags, const or_config_t* cfg_in,
                  double* X, or_info_t* info) {
  or_config_t cfg;
  if (cfg_in) cfg = *cfg_in; else or_default_config(&cfg);
  info_init(info);
  if (n < 0 || nrhs < 1 || kl < 0 || ku < 0 || ldab < kl + ku + 1) {
    info->status = OR_E_INVALID;
    return OR_E_INVALID;
  }
  if (n == 0) return OR_OK;
  int64_t tkl = 0, tku = 0;
  double norm1 = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    double colsum = 0.0;
    for (int64_t i = (j - ku > 0 ? j - ku : 0); i <= j + kl && i < n; ++i) {
      double a = AB[(size_t)(ku + i - j) + (size_t)j * ldab];
      if (!isfinite(a)) { info->status = OR_E_NONFINITE; return OR_E_NONFINITE; }
      if (a != 0.0) {
        if (j - i > tku) tku = j - i;
        if (i - j > tkl) tkl = i - j;
      }
      colsum += fabs(a);
    }
    if (colsum > norm1) norm1 = colsum;
  }
  if (!all_finite(B, (size_t)n * nrhs)) { info->status = OR_E_NONFINITE; return OR_E_NONFINITE; }
  info->cls = OR_CLS_BANDED;
  info->route = OR_ROUTE_BAND_LU;
  info->kl = tkl;
  info->ku = tku;
  if ((flags & OR_TRIDIAG) && tkl == 1 && tku == 1) { /* the tridiagonal specialisation */
    info->route = OR_ROUTE_TRIDIAG;
    memcpy(X, B, sizeof(double) * (size_t)n * nrhs);
    int gfail = solve_gt_route(AB, 0, ldab, ku, n, X, nrhs, flags, norm1, info);
    double* dense = NULL;
    int poor = !gfail && !(flags & OR_NO_RCOND) && !(info->rcond >= cfg.rcond_threshold);
    if ((gfail || poor) && !(flags & OR_NO_APPROX) && n <= OR_SVD_DENSIFY_NMAX) {
      dense = (double*)calloc((size_t)n * n, sizeof(double));
      for (int64_t j = 0; j < n; ++j)
        for (int64_t i = (j - ku > 0 ? j - ku : 0); i <= j + kl && i < n; ++i)
          dense[(size_t)i + (size_t)j * n] = AB[(size_t)(ku + i - j) + (size_t)j * ldab];
    }
    int st = finish(dense, B, n, nrhs, flags, &cfg, gfail, X, info);
    free(dense);
    return st;
  }
  int64_t fld = 2 * tkl + tku + 1, kv = tkl + tku;
  double* F = (double*)calloc((size_t)fld * n, sizeof(double));
  int64_t* ipiv = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = (j - tku > 0 ? j - tku : 0); i <= j + tkl && i < n; ++i)
      F[(size_t)(kv + i - j) + (size_t)j * fld] = AB[(size_t)(ku + i - j) + (size_t)j * ldab];
  memcpy(X, B, sizeof(double) * (size_t)n * nrhs);
  int failed = or_band_lu_factor(F, fld, n, tkl, tku, ipiv) != 0;
  if (!failed) {
    or_band_lu_solve(F, fld, n, tkl, tku, ipiv, X, nrhs, 0);
    if (!(flags & OR_NO_RCOND))
      info->rcond = or_rcond_from(norm1, or_est_inv_norm1_band(F, fld, n, tkl, tku, ipiv));
  }
  free(F); free(ipiv);
  double* dense = NULL;
  int poor = !failed && !(flags & OR_NO_RCOND) && !(info->rcond >= cfg.rcond_threshold);
  if ((failed || poor) && !(flags & OR_NO_APPROX) && n <= OR_SVD_DENSIFY_NMAX) {
    dense = (double*)calloc((size_t)n * n, sizeof(double));
    for (int64_t j = 0; j < n; ++j)
      for (int64_t i = (j - ku > 0 ? j - ku : 0); i <= j + kl && i < n; ++i)
        dense[(size_t)i + (size_t)j * n] = AB[(size_t)(ku + i - j) + (size_t)j * ldab];
  }
  int st = finish(dense, B, n, nrhs, flags, &cfg, failed, X, info);
  free(dense);
  return st;
}
