/*
 * Oracle for the batched panel-major BLAS/LAPACK path: plain, slow, obviously
 * correct CPU routines in FP64.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg do.  It shares no code, header, helper or
 * constant with the CUDA library.
 *
 * Conventions
 *   - Matrices are column-major: element (i, j) of A is A[i + j*lda].
 *   - Every routine is the textbook definition written out as loops, in the
 *     order the definition states, with no blocking or fusion.  Compile with
 *     -O2 -ffp-contract=off so that no multiply-add is contracted and the
 *     rounding is the plain IEEE-754 one of each written operation.
 *   - Sizes equal to zero return at once and touch nothing.
 *
 * Readings of the paper where it is silent (each one is tested):
 *   - beta == 0: C is not read (the BLAS convention), so NaN in C is ignored.
 *   - syrk / potrf / syrk_potrf write only the lower triangle of D,
 *     diagonal included; the strictly upper part of D is left untouched.
 *   - potrf: the first column j whose pivot d fails (d > 0) (this includes a
 *     NaN pivot) makes the routine return j+1 and stop; columns >= j of D are
 *     then unspecified.  0 means success.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define EL(P, ld, i, j) (P)[(size_t)(i) + (size_t)(j) * (size_t)(ld)]

/* gemm_nt (Appendix A.2.1, the gemm example; Sec. 5.2.2 "gemm_nt"):
 *   D <- alpha * A * B^T + beta * C
 * A is m x k, B is n x k, C and D are m x n; C and D may coincide. */
void or_dgemm_nt(int m, int n, int k, double alpha, const double *A, int lda,
                 const double *B, int ldb, double beta, const double *C, int ldc,
                 double *D, int ldd) {
  if (m <= 0 || n <= 0) return;
  for (int j = 0; j < n; j++) {
    for (int i = 0; i < m; i++) {
      double s = 0.0;
      for (int l = 0; l < k; l++) s += EL(A, lda, i, l) * EL(B, ldb, j, l);
      double c = (beta == 0.0) ? 0.0 : beta * EL(C, ldc, i, j);
      EL(D, ldd, i, j) = alpha * s + c;
    }
  }
}

/* gemm_nn (Sec. 5.2.2 "gemm_nn"): D <- alpha * A * B + beta * C, A m x k,
 * B k x n, C and D m x n; C and D may coincide; beta == 0: C not read. */
void or_dgemm_nn(int m, int n, int k, double alpha, const double *A, int lda,
                 const double *B, int ldb, double beta, const double *C, int ldc,
                 double *D, int ldd) {
  if (m <= 0 || n <= 0) return;
  for (int j = 0; j < n; j++) {
    for (int i = 0; i < m; i++) {
      double s = 0.0;
      for (int l = 0; l < k; l++) s += EL(A, lda, i, l) * EL(B, ldb, l, j);
      double c = (beta == 0.0) ? 0.0 : beta * EL(C, ldc, i, j);
      EL(D, ldd, i, j) = alpha * s + c;
    }
  }
}

/* syrk_ln (Sec. 5.2.2 "syrk_ln"): lower(D) <- alpha * A * B^T + beta * C,
 * A and B are m x k and may differ, C and D are m x m.  Only i >= j is
 * computed and written. */
void or_dsyrk_ln(int m, int k, double alpha, const double *A, int lda,
                 const double *B, int ldb, double beta, const double *C, int ldc,
                 double *D, int ldd) {
  if (m <= 0) return;
  for (int j = 0; j < m; j++) {
    for (int i = j; i < m; i++) {
      double s = 0.0;
      for (int l = 0; l < k; l++) s += EL(A, lda, i, l) * EL(B, ldb, j, l);
      double c = (beta == 0.0) ? 0.0 : beta * EL(C, ldc, i, j);
      EL(D, ldd, i, j) = alpha * s + c;
    }
  }
}

/* potrf_l (Sec. 5.2.2 "potrf_l"; Sec. 4.6 for the factorization as a
 * sequence of column steps): the lower Cholesky factor L of the m x m SPD
 * matrix C (only its lower triangle is read), C = L * L^T, stored in lower(D).
 * Column by column (Cholesky-Crout order):
 *   d       = C[j][j] - sum_{l<j} L[j][l]^2
 *   L[j][j] = sqrt(d)                       (fails unless d > 0)
 *   L[i][j] = (C[i][j] - sum_{l<j} L[i][l] L[j][l]) / L[j][j],  i > j
 * If dinv is not NULL, dinv[j] = 1 / L[j][j] (the inverse diagonal that the
 * factorization keeps for later solves, Sec. 4.7.1).
 * C and D may coincide.  Returns 0, or j+1 for the first failing pivot. */
int or_dpotrf_l(int m, const double *C, int ldc, double *D, int ldd, double *dinv) {
  if (m <= 0) return 0;
  for (int j = 0; j < m; j++) {
    double d = EL(C, ldc, j, j);
    for (int l = 0; l < j; l++) d -= EL(D, ldd, j, l) * EL(D, ldd, j, l);
    if (!(d > 0.0)) return j + 1;
    double ljj = sqrt(d);
    EL(D, ldd, j, j) = ljj;
    for (int i = j + 1; i < m; i++) {
      double s = EL(C, ldc, i, j);
      for (int l = 0; l < j; l++) s -= EL(D, ldd, i, l) * EL(D, ldd, j, l);
      EL(D, ldd, i, j) = s / ljj;
    }
    if (dinv) dinv[j] = 1.0 / ljj;
  }
  return 0;
}

/* trsm_rltn (Sec. 5.2.2 "trsm_rltn"; right side, lower, transposed,
 * non-unit): D = X with X * L^T = alpha * B, i.e. D <- alpha * B * L^{-T}.
 * B and D are m x n, L is n x n lower triangular (strictly upper part not
 * read).  Column by column:
 *   X[i][j] = (alpha B[i][j] - sum_{l<j} X[i][l] L[j][l]) / L[j][j].
 * B and D may coincide. */
void or_dtrsm_rltn(int m, int n, double alpha, const double *L, int ldl,
                   const double *B, int ldb, double *D, int ldd) {
  if (m <= 0 || n <= 0) return;
  for (int j = 0; j < n; j++) {
    for (int i = 0; i < m; i++) {
      double s = alpha * EL(B, ldb, i, j);
      for (int l = 0; l < j; l++) s -= EL(D, ldd, i, l) * EL(L, ldl, j, l);
      EL(D, ldd, i, j) = s / EL(L, ldl, j, j);
    }
  }
}

/* syrk_potrf_ln (Sec. 4.7.2 "Concatenating updates/downdates"; Sec. 5.3,
 * the Riccati factorization step; Appendix A.3 routine list):
 *   lower(D) <- chol(C + A * B^T),  A and B m x k, C and D m x m.
 * Written as its definition: the syrk_ln sum with alpha = beta = 1 into a
 * scratch matrix, then potrf_l of that matrix.  Returns potrf's info. */
int or_dsyrk_dpotrf_ln(int m, int k, const double *A, int lda, const double *B, int ldb,
                       const double *C, int ldc, double *D, int ldd, double *dinv) {
  if (m <= 0) return 0;
  double *T = (double *)malloc((size_t)m * (size_t)m * sizeof(double));
  if (!T) return -1;
  or_dsyrk_ln(m, k, 1.0, A, lda, B, ldb, 1.0, C, ldc, T, m);
  int info = or_dpotrf_l(m, T, m, D, ldd, dinv);
  free(T);
  return info;
}

/* potrs (solve with the Cholesky factor; the two right-hand-side triangular
 * solves trsv_lnn and trsv_ltn of the BLAS level-2 list, Appendix A.3):
 * given lower L with L L^T = A, X = A^{-1} B by
 *   forward substitution  L Y = B:    Y[i] = (B[i] - sum_{l<i} L[i][l] Y[l]) / L[i][i]
 *   backward substitution L^T X = Y:  X[i] = (Y[i] - sum_{l>i} L[l][i] X[l]) / L[i][i]
 * column by column of B (n x nrhs).  Y is kept in X; B and X may coincide. */
void or_dpotrs_l(int n, int nrhs, const double *L, int ldl, const double *B, int ldb, double *X,
                 int ldx) {
  if (n <= 0 || nrhs <= 0) return;
  for (int k = 0; k < nrhs; k++) {
    for (int i = 0; i < n; i++) {
      double s = EL(B, ldb, i, k);
      for (int l = 0; l < i; l++) s -= EL(L, ldl, i, l) * EL(X, ldx, l, k);
      EL(X, ldx, i, k) = s / EL(L, ldl, i, i);
    }
    for (int i = n - 1; i >= 0; i--) {
      double s = EL(X, ldx, i, k);
      for (int l = i + 1; l < n; l++) s -= EL(L, ldl, l, i) * EL(X, ldx, l, k);
      EL(X, ldx, i, k) = s / EL(L, ldl, i, i);
    }
  }
}

/* trmm_rlnn (Sec. 5.2.2 "trmm_rlnn"; right, lower, not transposed,
 * non-unit): D <- alpha * B * L with L n x n lower triangular (strictly upper
 * part not read), B and D m x n:
 *   D[i][j] = alpha * sum_{l >= j} B[i][l] L[l][j]. */
void or_dtrmm_rlnn(int m, int n, double alpha, const double *B, int ldb, const double *L, int ldl,
                   double *D, int ldd) {
  if (m <= 0 || n <= 0) return;
  for (int j = 0; j < n; j++) {
    for (int i = 0; i < m; i++) {
      double s = 0.0;
      for (int l = j; l < n; l++) s += EL(B, ldb, i, l) * EL(L, ldl, l, j);
      EL(D, ldd, i, j) = alpha * s;
    }
  }
}

/* trsm_rlnn (right, lower, not transposed, non-unit): D = X with
 * X * L = alpha * B, L n x n lower, B and D m x n.  Column by column from
 * the last:  X[i][j] = (alpha B[i][j] - sum_{l > j} X[i][l] L[l][j]) / L[j][j].
 * B and D may coincide. */
void or_dtrsm_rlnn(int m, int n, double alpha, const double *L, int ldl, const double *B, int ldb,
                   double *D, int ldd) {
  if (m <= 0 || n <= 0) return;
  for (int j = n - 1; j >= 0; j--) {
    for (int i = 0; i < m; i++) {
      double s = alpha * EL(B, ldb, i, j);
      for (int l = j + 1; l < n; l++) s -= EL(D, ldd, i, l) * EL(L, ldl, l, j);
      EL(D, ldd, i, j) = s / EL(L, ldl, j, j);
    }
  }
}

/* Adjoint of the Cholesky factor-and-solve X = A^{-1} B (not in the paper):
 * given the factor L of A, the solution X and the cotangent Xbar (n x nrhs),
 *   Bbar = A^{-1} Xbar                          (potrs with L)
 *   Abar = -(Bbar X^T + X Bbar^T) / 2           (the symmetric part of
 *                                                -Bbar X^T; A is symmetric)
 * Abar is written in full (n x n).  Bbar must not alias X or Xbar. */
void or_dposv_adjoint(int n, int nrhs, const double *L, int ldl, const double *X, int ldx,
                      const double *Xbar, int ldxb, double *Bbar, int ldbb, double *Abar, int lda) {
  if (n <= 0 || nrhs <= 0) return;
  or_dpotrs_l(n, nrhs, L, ldl, Xbar, ldxb, Bbar, ldbb);
  for (int j = 0; j < n; j++)
    for (int i = 0; i < n; i++) {
      double s = 0.0;
      for (int k = 0; k < nrhs; k++)
        s += EL(Bbar, ldbb, i, k) * EL(X, ldx, j, k) + EL(X, ldx, i, k) * EL(Bbar, ldbb, j, k);
      EL(Abar, lda, i, j) = -0.5 * s;
    }
}

/* getrf (Sec. 5.2.2 "getrf"; LU factorization with partial pivoting, the
 * routine list of Appendix A.3): P A = L U for the n x n matrix A, in the
 * unblocked right-looking order, column by column:
 *   p      = first i >= j with |A[i][j]| maximal          (pivot row)
 *   swap rows j and p (whole rows); ipiv[j] = p           (0-based)
 *   A[i][j] = A[i][j] / A[j][j],  i > j                   (multipliers, L)
 *   A[i][c] -= A[i][j] A[j][c],   i > j, c > j            (update)
 * L (unit diagonal, not stored) and U overwrite D (a copy of C).  A zero
 * pivot sets info = j+1 (first one) and skips that column's division.
 * Returns info. */
int or_dgetrf(int n, const double *C, int ldc, double *D, int ldd, int *ipiv) {
  if (n <= 0) return 0;
  int info = 0;
  for (int j = 0; j < n; j++)
    for (int i = 0; i < n; i++) EL(D, ldd, i, j) = EL(C, ldc, i, j);
  for (int j = 0; j < n; j++) {
    int p = j;
    double best = fabs(EL(D, ldd, j, j));
    for (int i = j + 1; i < n; i++)
      if (fabs(EL(D, ldd, i, j)) > best) {
        best = fabs(EL(D, ldd, i, j));
        p = i;
      }
    ipiv[j] = p;
    if (p != j)
      for (int c = 0; c < n; c++) {
        double t = EL(D, ldd, j, c);
        EL(D, ldd, j, c) = EL(D, ldd, p, c);
        EL(D, ldd, p, c) = t;
      }
    double piv = EL(D, ldd, j, j);
    if (piv == 0.0) {
      if (info == 0) info = j + 1;
      continue;
    }
    for (int i = j + 1; i < n; i++) EL(D, ldd, i, j) = EL(D, ldd, i, j) / piv;
    for (int c = j + 1; c < n; c++)
      for (int i = j + 1; i < n; i++) EL(D, ldd, i, c) -= EL(D, ldd, i, j) * EL(D, ldd, j, c);
  }
  return info;
}

/* gelqf (Sec. 5.2.2 "gelqf"; LQ factorization, routine list of Appendix A.3):
 * A = L Q for the m x n matrix A, by Householder reflectors applied from the
 * right, row by row (i < min(m, n)):
 *   alpha = A[i][i], x = A[i][i+1:n], s = ||x||^2
 *   if s == 0:  tau[i] = 0 (H_i = I)
 *   else:       beta = -sign(alpha) sqrt(alpha^2 + s); tau[i] = (beta - alpha) / beta
 *               x = x / (alpha - beta); A[i][i] = beta
 *   H_i = I - tau[i] v v^T with v = [1, x]; rows r > i: A[r][i:n] <- A[r][i:n] H_i
 * L is the lower triangle of the result; the reflectors v (without their
 * leading 1) are left in the strictly upper part of row i, and Q =
 * H_{k-1} ... H_1 H_0 with k = min(m, n).  D is a copy of C on entry. */
void or_dgelqf(int m, int n, const double *C, int ldc, double *D, int ldd, double *tau) {
  if (m <= 0 || n <= 0) return;
  for (int j = 0; j < n; j++)
    for (int i = 0; i < m; i++) EL(D, ldd, i, j) = EL(C, ldc, i, j);
  int k = m < n ? m : n;
  for (int i = 0; i < k; i++) {
    double alpha = EL(D, ldd, i, i), s = 0.0;
    for (int c = i + 1; c < n; c++) s += EL(D, ldd, i, c) * EL(D, ldd, i, c);
    double t = 0.0;
    if (s != 0.0) {
      double beta = -copysign(sqrt(alpha * alpha + s), alpha);
      t = (beta - alpha) / beta;
      double scal = 1.0 / (alpha - beta);
      for (int c = i + 1; c < n; c++) EL(D, ldd, i, c) *= scal;
      EL(D, ldd, i, i) = beta;
    }
    tau[i] = t;
    for (int r = i + 1; r < m; r++) {
      double w = EL(D, ldd, r, i);
      for (int c = i + 1; c < n; c++) w += EL(D, ldd, r, c) * EL(D, ldd, i, c);
      EL(D, ldd, r, i) -= t * w;
      for (int c = i + 1; c < n; c++) EL(D, ldd, r, c) -= t * w * EL(D, ldd, i, c);
    }
  }
}

/* Panel-major format (Sec. 4.3.3): rows are grouped in panels of ps rows
 * (ps a power of two); each panel is a column-major ps x cn block (lda = ps)
 * and panels follow one another, ps*cn doubles apart.  Element (r, c) of the
 * panel-major matrix therefore lies at
 *   (r / ps) * ps * cn  +  c * ps  +  r % ps.
 * pack copies the m x n column-major matrix A into the panel-major matrix pA
 * at sub-matrix offset (ai, aj); unpack copies it back out. */
static size_t pm_index(int r, int c, int ps, int cn) {
  return (size_t)(r / ps) * (size_t)ps * (size_t)cn + (size_t)c * (size_t)ps + (size_t)(r % ps);
}

void or_pack(int m, int n, const double *A, int lda, int ps, int cn, double *pA, int ai, int aj) {
  for (int j = 0; j < n; j++)
    for (int i = 0; i < m; i++) pA[pm_index(ai + i, aj + j, ps, cn)] = EL(A, lda, i, j);
}

void or_unpack(int m, int n, int ps, int cn, const double *pA, int ai, int aj, double *A, int lda) {
  for (int j = 0; j < n; j++)
    for (int i = 0; i < m; i++) EL(A, lda, i, j) = pA[pm_index(ai + i, aj + j, ps, cn)];
}

/* ---- batched drivers: the same routines over independent problems ------
 * Problem b's operand X starts at X + b*sX (strides in doubles).  The loop
 * over problems runs on every OpenMP thread; the arithmetic of each problem
 * is exactly the single-problem routine above. */
int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_set_num_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

void or_dgemm_nt_batch(int batch, int m, int n, int k, double alpha,
                       const double *A, int lda, long sA, const double *B, int ldb, long sB,
                       double beta, const double *C, int ldc, long sC, double *D, int ldd, long sD) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int b = 0; b < batch; b++)
    or_dgemm_nt(m, n, k, alpha, A + (size_t)b * sA, lda, B + (size_t)b * sB, ldb, beta,
                C + (size_t)b * sC, ldc, D + (size_t)b * sD, ldd);
}

void or_dsyrk_ln_batch(int batch, int m, int k, double alpha,
                       const double *A, int lda, long sA, const double *B, int ldb, long sB,
                       double beta, const double *C, int ldc, long sC, double *D, int ldd, long sD) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int b = 0; b < batch; b++)
    or_dsyrk_ln(m, k, alpha, A + (size_t)b * sA, lda, B + (size_t)b * sB, ldb, beta,
                C + (size_t)b * sC, ldc, D + (size_t)b * sD, ldd);
}

void or_dpotrf_l_batch(int batch, int m, const double *C, int ldc, long sC,
                       double *D, int ldd, long sD, double *dinv, long sdinv, int *info) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int b = 0; b < batch; b++)
    info[b] = or_dpotrf_l(m, C + (size_t)b * sC, ldc, D + (size_t)b * sD, ldd,
                          dinv ? dinv + (size_t)b * sdinv : NULL);
}

void or_dtrsm_rltn_batch(int batch, int m, int n, double alpha, const double *L, int ldl, long sL,
                         const double *B, int ldb, long sB, double *D, int ldd, long sD) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int b = 0; b < batch; b++)
    or_dtrsm_rltn(m, n, alpha, L + (size_t)b * sL, ldl, B + (size_t)b * sB, ldb,
                  D + (size_t)b * sD, ldd);
}

void or_dpotrs_l_batch(int batch, int n, int nrhs, const double *L, int ldl, long sL,
                       const double *B, int ldb, long sB, double *X, int ldx, long sX) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int b = 0; b < batch; b++)
    or_dpotrs_l(n, nrhs, L + (size_t)b * sL, ldl, B + (size_t)b * sB, ldb, X + (size_t)b * sX, ldx);
}

void or_dsyrk_dpotrf_ln_batch(int batch, int m, int k, const double *A, int lda, long sA,
                              const double *B, int ldb, long sB, const double *C, int ldc, long sC,
                              double *D, int ldd, long sD, double *dinv, long sdinv, int *info) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int b = 0; b < batch; b++)
    info[b] = or_dsyrk_dpotrf_ln(m, k, A + (size_t)b * sA, lda, B + (size_t)b * sB, ldb,
                                 C + (size_t)b * sC, ldc, D + (size_t)b * sD, ldd,
                                 dinv ? dinv + (size_t)b * sdinv : NULL);
}
