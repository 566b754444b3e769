/*
 * oracle.c -- plain, slow CPU reference for the recursive dense factorizations
 * of Peise & Bientinesi, "Recursive Algorithms for Dense Linear Algebra: The
 * ReLAPACK Collection" (arXiv 1602.06763).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may call,
 * link or load this file: only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg do.  It shares no code, header, table or helper
 * with the CUDA implementation.
 *
 * Everything is IEEE binary64, column-major with a leading dimension (LAPACK
 * storage; Section 5 keeps LAPACK's calling conventions).  It is compiled with
 * -ffp-contract=off so that every a*b+c is two rounded operations and the
 * results are the same on x86-64 and aarch64.  OpenMP only distributes
 * independent output elements over threads; each element's arithmetic is done
 * in the order written here.
 *
 * Routines and the passages they follow:
 *   or_split        Section 3, footnote on alignment (halves that are
 *                   multiples of 8 when the size allows)
 *   or_trtri        Section 3, Fig. 4 updates (1)-(4); base case trti2 below
 *                   the crossover c (Section 3, "crossover size")
 *   or_lauum        Section 5, xlauum (A := L^T L); recursion: the standard
 *                   reading of the halving scheme of Section 3
 *   or_potrf        Section 5, xpotrf (L L^T := A); Section 3 halving scheme
 *                   with LAPACK's unblocked potf2 as base case
 *   or_getrf        Section 5, xgetrf (P L U := A, row pivoting); Section 3
 *                   halving scheme with unblocked getf2 as base case
 *   or_laswp        the row interchanges P of xgetrf
 *   or_getri        Section 5, xtrtri as the building block of xgetri:
 *                   the inverse by its definition, A X = I
 *   or_zpotrf,      complex double peers (Section 5: s, d, c and z): the
 *   or_zgetrf       same recursions with the conjugate transpose
 *   or_ztrtri,      complex inversions, each its definition written out
 *   or_zlauum,      (substitution on L X = I; L^H L; L^{-H} L^{-1}; A X = I
 *   or_zpotri,      on the factors)
 *   or_zgetri
 *   or_sygst        Section 5, xsygst (A := L^{-1} A L^{-T}, or L^T A L):
 *                   the definition, by substitution and products
 *   metrics         normwise backward errors of the pass bound (<= 10)
 *                   ||A - LL^T|| / (n eps ||A||) <= 10, computed with the
 *                   compensated dot product Dot2 of Ogita, Rump & Oishi (2005)
 *
 * Parity pins: every routine here is pinned by the "not gpu" tests (closed
 * forms, integer-exact factors, exact rational brute force, LAPACK via scipy,
 * the paper's per-level flop shares).  No function is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define AT(M, ld, i, j) (M)[(size_t)(j) * (size_t)(ld) + (size_t)(i)]

/* -------------------------------------------------------------------------- */
/* Split rule.  Section 3 footnote: the two "halves" are multiples of 8 where  */
/* possible and may differ slightly in size.  Reading: n1 = 8*floor((n+8)/16)  */
/* for n >= 16 (a multiple of 8 within 4 of n/2), else floor(n/2).             */
/* -------------------------------------------------------------------------- */
int64_t or_split(int64_t n)
{
    if (n >= 16) return 8 * ((n + 8) / 16);
    return n / 2;
}

/* -------------------------------------------------------------------------- */
/* Plain BLAS-3 building blocks (definitions written out, no blocking).        */
/* -------------------------------------------------------------------------- */

/* C(m x n) := C + alpha * op(A) * op(B), op(X) = X or X^T.
 * Element (i,j): s = sum_{p=0}^{k-1} op(A)(i,p) op(B)(p,j) accumulated in
 * increasing p from 0.0, then c_ij = c_ij + alpha*s. */
void or_gemm(int ta, int tb, int64_t m, int64_t n, int64_t k, double alpha,
             const double *A, int64_t lda, const double *B, int64_t ldb,
             double *C, int64_t ldc)
{
    if (m <= 0 || n <= 0) return;
    #pragma omp parallel
    {
        double *s = (double *)malloc(sizeof(double) * (size_t)m);
        #pragma omp for schedule(dynamic, 4)
        for (int64_t j = 0; j < n; ++j) {
            for (int64_t i = 0; i < m; ++i) s[i] = 0.0;
            for (int64_t p = 0; p < k; ++p) {
                double b = tb ? AT(B, ldb, j, p) : AT(B, ldb, p, j);
                if (!ta) {
                    for (int64_t i = 0; i < m; ++i) s[i] += AT(A, lda, i, p) * b;
                } else {
                    for (int64_t i = 0; i < m; ++i) s[i] += AT(A, lda, p, i) * b;
                }
            }
            for (int64_t i = 0; i < m; ++i) AT(C, ldc, i, j) += alpha * s[i];
        }
        free(s);
    }
}

/* Lower triangle of C(n x n) := C + alpha * op(A) op(A)^T, where op(A) is
 * A (n x k) when trans == 0 and A^T (A is k x n) when trans == 1.  Only
 * elements i >= j are read or written. */
void or_syrk_lower(int trans, int64_t n, int64_t k, double alpha,
                   const double *A, int64_t lda, double *C, int64_t ldc)
{
    if (n <= 0) return;
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t i = j; i < n; ++i) {
            double s = 0.0;
            for (int64_t p = 0; p < k; ++p) {
                double a = trans ? AT(A, lda, p, i) : AT(A, lda, i, p);
                double b = trans ? AT(A, lda, p, j) : AT(A, lda, j, p);
                s += a * b;
            }
            AT(C, ldc, i, j) += alpha * s;
        }
    }
}

/* Left, lower, no-transpose triangular solve: B(m x n) := alpha * L^{-1} B.
 * Column by column forward substitution
 *   x_i = (alpha*b_i - sum_{k<i} l_ik x_k) / l_ii   (no division if unit). */
void or_trsm_llnx(int unit, int64_t m, int64_t n, double alpha,
                  const double *L, int64_t ldl, double *B, int64_t ldb)
{
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < n; ++j) {
        double *x = &AT(B, ldb, 0, j);
        for (int64_t i = 0; i < m; ++i) {
            double s = alpha * x[i];
            for (int64_t k = 0; k < i; ++k) s -= AT(L, ldl, i, k) * x[k];
            x[i] = unit ? s : s / AT(L, ldl, i, i);
        }
    }
}

/* Right, lower, transposed, non-unit solve: B(m x n) := B L^{-T}, i.e. each
 * row x of the result satisfies x L^T = b:
 *   x_j = (b_j - sum_{k<j} x_k l_jk) / l_jj. */
void or_trsm_rltn(int64_t m, int64_t n, const double *L, int64_t ldl,
                  double *B, int64_t ldb)
{
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < m; ++r) {
        for (int64_t j = 0; j < n; ++j) {
            double s = AT(B, ldb, r, j);
            for (int64_t k = 0; k < j; ++k) s -= AT(B, ldb, r, k) * AT(L, ldl, j, k);
            AT(B, ldb, r, j) = s / AT(L, ldl, j, j);
        }
    }
}

/* Left, upper, no-transpose solve B(m x n) := U^{-1} B (back substitution)
 *   x_i = (b_i - sum_{k>i} u_ik x_k) / u_ii.  Used by the solve drivers. */
void or_trsm_lunn(int64_t m, int64_t n, const double *U, int64_t ldu,
                  double *B, int64_t ldb)
{
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < n; ++j) {
        double *x = &AT(B, ldb, 0, j);
        for (int64_t i = m - 1; i >= 0; --i) {
            double s = x[i];
            for (int64_t k = i + 1; k < m; ++k) s -= AT(U, ldu, i, k) * x[k];
            x[i] = s / AT(U, ldu, i, i);
        }
    }
}

/* Left, lower, transposed, non-unit solve B := L^{-T} B (back substitution
 * with L^T):  x_i = (b_i - sum_{k>i} l_ki x_k) / l_ii. */
void or_trsm_lltn(int64_t m, int64_t n, const double *L, int64_t ldl,
                  double *B, int64_t ldb)
{
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < n; ++j) {
        double *x = &AT(B, ldb, 0, j);
        for (int64_t i = m - 1; i >= 0; --i) {
            double s = x[i];
            for (int64_t k = i + 1; k < m; ++k) s -= AT(L, ldl, k, i) * x[k];
            x[i] = s / AT(L, ldl, i, i);
        }
    }
}

/* Right, lower, no-transpose product B(m x n) := B L with L lower (n x n):
 *   (B L)_ij = sum_{k=j}^{n-1} b_ik l_kj, computed into a copy. */
void or_trmm_rlnn(int64_t m, int64_t n, const double *L, int64_t ldl,
                  double *B, int64_t ldb)
{
    if (m <= 0 || n <= 0) return;
    double *T = (double *)malloc(sizeof(double) * (size_t)m * (size_t)n);
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t i = 0; i < m; ++i) {
            double s = 0.0;
            for (int64_t k = j; k < n; ++k) s += AT(B, ldb, i, k) * AT(L, ldl, k, j);
            T[(size_t)j * m + i] = s;
        }
    }
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i) AT(B, ldb, i, j) = T[(size_t)j * m + i];
    free(T);
}

/* Left, lower, transposed product B(m x n) := L^T B with L lower (m x m):
 *   (L^T B)_ij = sum_{k=i}^{m-1} l_ki b_kj, computed into a copy. */
void or_trmm_lltn(int64_t m, int64_t n, const double *L, int64_t ldl,
                  double *B, int64_t ldb)
{
    if (m <= 0 || n <= 0) return;
    double *T = (double *)malloc(sizeof(double) * (size_t)m * (size_t)n);
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t i = 0; i < m; ++i) {
            double s = 0.0;
            for (int64_t k = i; k < m; ++k) s += AT(L, ldl, k, i) * AT(B, ldb, k, j);
            T[(size_t)j * m + i] = s;
        }
    }
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i) AT(B, ldb, i, j) = T[(size_t)j * m + i];
    free(T);
}

/* -------------------------------------------------------------------------- */
/* Cholesky.  Section 5 (xpotrf: L L^T := A), lower storage.                   */
/* -------------------------------------------------------------------------- */

/* Unblocked base case (LAPACK potf2 semantics), column j = 0..n-1:
 *   d = a_jj - sum_{k<j} l_jk^2; if d <= 0 or d is NaN: a_jj = d, info = j+1;
 *   l_jj = sqrt(d); l_ij = (a_ij - sum_{k<j} l_ik l_jk) / l_jj for i > j.
 * Returns info (0 on success). */
int64_t or_potf2(int64_t n, double *A, int64_t lda)
{
    for (int64_t j = 0; j < n; ++j) {
        double s = 0.0;
        for (int64_t k = 0; k < j; ++k) s += AT(A, lda, j, k) * AT(A, lda, j, k);
        double d = AT(A, lda, j, j) - s;
        if (!(d > 0.0)) {            /* d <= 0 or NaN */
            AT(A, lda, j, j) = d;
            return j + 1;
        }
        double ljj = sqrt(d);
        AT(A, lda, j, j) = ljj;
        for (int64_t i = j + 1; i < n; ++i) {
            double t = 0.0;
            for (int64_t k = 0; k < j; ++k) t += AT(A, lda, i, k) * AT(A, lda, j, k);
            AT(A, lda, i, j) = (AT(A, lda, i, j) - t) / ljj;
        }
    }
    return 0;
}

/* Recursive Cholesky: recurse while n > c (reading of the Fig. 4 caption),
 * otherwise potf2.  With n1 = split(n):
 *   (1) potrf(A11)              -> L11
 *   (2) A21 := A21 L11^{-T}     (triangular solve)
 *   (3) A22 := A22 - A21 A21^T  (lower triangle only)
 *   (4) potrf(A22)              -> L22, info offset by n1. */
int64_t or_potrf(int64_t n, double *A, int64_t lda, int64_t c)
{
    if (n <= 0) return 0;
    if (c < 1) c = 1;
    if (n <= c) return or_potf2(n, A, lda);
    int64_t n1 = or_split(n), n2 = n - n1;
    double *A11 = A, *A21 = &AT(A, lda, n1, 0), *A22 = &AT(A, lda, n1, n1);
    int64_t info = or_potrf(n1, A11, lda, c);
    if (info) return info;
    or_trsm_rltn(n2, n1, A11, lda, A21, lda);
    or_syrk_lower(0, n2, n1, -1.0, A21, lda, A22, lda);
    info = or_potrf(n2, A22, lda, c);
    return info ? info + n1 : 0;
}

/* -------------------------------------------------------------------------- */
/* LU with partial (row) pivoting.  Section 5 (xgetrf: P L U := A).            */
/* ipiv is 1-based as in LAPACK: row i was interchanged with row ipiv[i]-1.    */
/* -------------------------------------------------------------------------- */

/* Apply the interchanges ipiv[k1..k2-1] (in that order) to the n columns of A:
 * for i = k1..k2-1 swap rows i and ipiv[i]-1. */
void or_laswp(int64_t n, double *A, int64_t lda, int64_t k1, int64_t k2,
              const int32_t *ipiv)
{
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t i = k1; i < k2; ++i) {
            int64_t p = (int64_t)ipiv[i] - 1;
            if (p != i) {
                double t = AT(A, lda, i, j);
                AT(A, lda, i, j) = AT(A, lda, p, j);
                AT(A, lda, p, j) = t;
            }
        }
    }
}

/* Unblocked base case (LAPACK getf2 semantics), j = 0..min(m,n)-1:
 *   p = argmax_{i>=j} |a_ij|, lowest i on exact ties (idamax);
 *   ipiv[j] = p+1;
 *   if a_pj != 0: swap rows j and p (all n columns), a_ij := a_ij / a_jj for
 *   i > j (division, not a reciprocal product); else info = j+1 if unset;
 *   rank-1 update a_ik := a_ik - a_ij a_jk for i > j, k > j.
 * Returns info. */
int64_t or_getf2(int64_t m, int64_t n, double *A, int64_t lda, int32_t *ipiv)
{
    int64_t info = 0, mn = m < n ? m : n;
    for (int64_t j = 0; j < mn; ++j) {
        int64_t p = j;
        double amax = fabs(AT(A, lda, j, j));
        for (int64_t i = j + 1; i < m; ++i) {
            double v = fabs(AT(A, lda, i, j));
            if (v > amax) { amax = v; p = i; }
        }
        ipiv[j] = (int32_t)(p + 1);
        if (AT(A, lda, p, j) != 0.0) {
            if (p != j)
                for (int64_t k = 0; k < n; ++k) {
                    double t = AT(A, lda, j, k);
                    AT(A, lda, j, k) = AT(A, lda, p, k);
                    AT(A, lda, p, k) = t;
                }
            double piv = AT(A, lda, j, j);
            for (int64_t i = j + 1; i < m; ++i) AT(A, lda, i, j) = AT(A, lda, i, j) / piv;
        } else if (info == 0) {
            info = j + 1;
        }
        for (int64_t k = j + 1; k < n; ++k) {
            double u = AT(A, lda, j, k);
            for (int64_t i = j + 1; i < m; ++i) AT(A, lda, i, k) -= AT(A, lda, i, j) * u;
        }
    }
    return info;
}

/* Recursive LU of the m x n matrix A.  Base case getf2 when n <= c or
 * min(m,n) <= c; otherwise, with n1 = split(min(m,n)), n2 = n - n1:
 *   (1) getrf(A[:, :n1])                    -> ipiv[0:n1]
 *   (2) apply ipiv[0:n1] to A[:, n1:]
 *   (3) A12 := L11^{-1} A12                  (unit lower solve)
 *   (4) A22 := A22 - A21 A12
 *   (5) getrf(A22) -> ipiv[n1:], shifted by n1; info shifted by n1
 *   (6) apply ipiv[n1:] to A[:, :n1]. */
int64_t or_getrf(int64_t m, int64_t n, double *A, int64_t lda, int32_t *ipiv,
                 int64_t c)
{
    if (m <= 0 || n <= 0) return 0;
    if (c < 1) c = 1;
    int64_t mn = m < n ? m : n;
    if (n <= c || mn <= c) return or_getf2(m, n, A, lda, ipiv);
    int64_t n1 = or_split(mn), n2 = n - n1;
    double *A12 = &AT(A, lda, 0, n1), *A21 = &AT(A, lda, n1, 0);
    double *A22 = &AT(A, lda, n1, n1);
    int64_t info = or_getrf(m, n1, A, lda, ipiv, c);
    or_laswp(n2, A12, lda, 0, n1, ipiv);
    or_trsm_llnx(1, n1, n2, 1.0, A, lda, A12, lda);
    or_gemm(0, 0, m - n1, n2, n1, -1.0, A21, lda, A12, lda, A22, lda);
    int64_t info2 = or_getrf(m - n1, n2, A22, lda, ipiv + n1, c);
    int64_t mn2 = (m - n1) < n2 ? (m - n1) : n2;
    for (int64_t i = 0; i < mn2; ++i) ipiv[n1 + i] += (int32_t)n1;
    if (info == 0 && info2 != 0) info = info2 + n1;
    or_laswp(n1, A, lda, n1, n1 + mn2, ipiv);
    return info;
}

/* -------------------------------------------------------------------------- */
/* Triangular inverse.  Section 3, Fig. 4 (lower, in place).                   */
/* -------------------------------------------------------------------------- */

/* Unblocked base case: X = L^{-1} column by column (forward substitution on
 * L x = e_j):  x_jj = 1/l_jj (1 if unit);
 *   x_ij = -(sum_{k=j}^{i-1} l_ik x_kj) / l_ii  for i > j (no division if unit). */
void or_trti2(int unit, int64_t n, double *A, int64_t lda)
{
    if (n <= 0) return;
    double *X = (double *)calloc((size_t)n * (size_t)n, sizeof(double));
    for (int64_t j = 0; j < n; ++j) {
        X[(size_t)j * n + j] = unit ? 1.0 : 1.0 / AT(A, lda, j, j);
        for (int64_t i = j + 1; i < n; ++i) {
            double s = 0.0;
            for (int64_t k = j; k < i; ++k) s += AT(A, lda, i, k) * X[(size_t)j * n + k];
            X[(size_t)j * n + i] = unit ? -s : -s / AT(A, lda, i, i);
        }
    }
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = j; i < n; ++i) AT(A, lda, i, j) = X[(size_t)j * n + i];
    free(X);
}

static void or_trtri_rec(int unit, int64_t n, double *A, int64_t lda, int64_t c)
{
    if (n <= 0) return;
    if (n <= c) { or_trti2(unit, n, A, lda); return; }
    int64_t n1 = or_split(n), n2 = n - n1;
    double *TL = A, *BL = &AT(A, lda, n1, 0), *BR = &AT(A, lda, n1, n1);
    /* (1) A_TL := A_TL^{-1} */
    or_trtri_rec(unit, n1, TL, lda, c);
    /* (2) A_BL := A_BL A_TL   (A_TL now holds its inverse) */
    if (unit) {
        /* unit diagonal: (B L)_ij = b_ij + sum_{k>j} b_ik l_kj, via a copy
           of TL with an explicit unit diagonal */
        double *T = (double *)calloc((size_t)n1 * (size_t)n1, sizeof(double));
        for (int64_t j = 0; j < n1; ++j) {
            T[(size_t)j * n1 + j] = 1.0;
            for (int64_t i = j + 1; i < n1; ++i) T[(size_t)j * n1 + i] = AT(TL, lda, i, j);
        }
        or_trmm_rlnn(n2, n1, T, n1, BL, lda);
        free(T);
    } else {
        or_trmm_rlnn(n2, n1, TL, lda, BL, lda);
    }
    /* (3) A_BL := -A_BR^{-1} A_BL   (A_BR not yet inverted) */
    or_trsm_llnx(unit, n2, n1, -1.0, BR, lda, BL, lda);
    /* (4) A_BR := A_BR^{-1} */
    or_trtri_rec(unit, n2, BR, lda, c);
}

/* Returns info = k if A(k,k) == 0 (first such k, 1-based; A is left
 * unchanged, as LAPACK's trtri does), else inverts A in place and returns 0. */
int64_t or_trtri(int unit, int64_t n, double *A, int64_t lda, int64_t c)
{
    if (n <= 0) return 0;
    if (c < 1) c = 1;
    if (!unit)
        for (int64_t i = 0; i < n; ++i)
            if (AT(A, lda, i, i) == 0.0) return i + 1;
    or_trtri_rec(unit, n, A, lda, c);
    return 0;
}

/* -------------------------------------------------------------------------- */
/* Triangular product A := L^T L (lower).  Section 5 (xlauum).                 */
/* -------------------------------------------------------------------------- */

/* Unblocked base case: (L^T L)_ij = sum_{k=i}^{n-1} l_ki l_kj for i >= j. */
void or_lauu2(int64_t n, double *A, int64_t lda)
{
    if (n <= 0) return;
    double *T = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = j; i < n; ++i) {
            double s = 0.0;
            for (int64_t k = i; k < n; ++k) s += AT(A, lda, k, i) * AT(A, lda, k, j);
            T[(size_t)j * n + i] = s;
        }
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = j; i < n; ++i) AT(A, lda, i, j) = T[(size_t)j * n + i];
    free(T);
}

/* Recursive lauum with L = [L11 0; L21 L22]:
 *   (1) lauum(A11)                 -> L11^T L11
 *   (2) A11 := A11 + A21^T A21     (lower triangle)
 *   (3) A21 := A22^T A21           (A22 still holds L22)
 *   (4) lauum(A22). */
void or_lauum(int64_t n, double *A, int64_t lda, int64_t c)
{
    if (n <= 0) return;
    if (c < 1) c = 1;
    if (n <= c) { or_lauu2(n, A, lda); return; }
    int64_t n1 = or_split(n), n2 = n - n1;
    double *A11 = A, *A21 = &AT(A, lda, n1, 0), *A22 = &AT(A, lda, n1, n1);
    or_lauum(n1, A11, lda, c);
    or_syrk_lower(1, n1, n2, 1.0, A21, lda, A11, lda);
    or_trmm_lltn(n2, n1, A22, lda, A21, lda);
    or_lauum(n2, A22, lda, c);
}

/* POTRI: A^{-1} = (L L^T)^{-1} = L^{-T} L^{-1}: trtri then lauum on L
 * (Section 5 names xtrtri as a component of the SPD inverse xpotri). */
int64_t or_potri(int64_t n, double *A, int64_t lda, int64_t c)
{
    int64_t info = or_trtri(0, n, A, lda, c);
    if (info) return info;
    or_lauum(n, A, lda, c);
    return 0;
}

/* -------------------------------------------------------------------------- */
/* Solves with the oracle's own factors (reference for refinement results).   */
/* -------------------------------------------------------------------------- */

/* getrs: X := A^{-1} B given P L U from or_getrf (square n). */
void or_getrs(int64_t n, int64_t nrhs, const double *LU, int64_t lda,
              const int32_t *ipiv, double *B, int64_t ldb)
{
    or_laswp(nrhs, B, ldb, 0, n, ipiv);
    or_trsm_llnx(1, n, nrhs, 1.0, LU, lda, B, ldb);
    or_trsm_lunn(n, nrhs, LU, lda, B, ldb);
}

/* potrs: X := A^{-1} B given lower L from or_potrf. */
void or_potrs(int64_t n, int64_t nrhs, const double *L, int64_t lda,
              double *B, int64_t ldb)
{
    or_trsm_llnx(0, n, nrhs, 1.0, L, lda, B, ldb);
    or_trsm_lltn(n, nrhs, L, lda, B, ldb);
}

/* getri: X := A^{-1} from P A = L U (or_getrf's LU and ipiv), by the       */
/* definition of the inverse: the solution of A X = I, column by column.     */
void or_getri(int64_t n, const double *LU, int64_t lda, const int32_t *ipiv, double *X, int64_t ldx)
{
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i) AT(X, ldx, i, j) = (i == j) ? 1.0 : 0.0;
    or_getrs(n, n, LU, lda, ipiv, X, ldx);
}

/* -------------------------------------------------------------------------- */
/* sygst (Section 5, xsygst): reduction of the symmetric-definite generalized */
/* problem to standard form with the Cholesky factor L of B, by definition:   */
/*   itype 1:    A := L^{-1} A L^{-T}                                         */
/*   itype 2, 3: A := L^T A L                                                 */
/* A is symmetric with its lower triangle stored; only that triangle is read */
/* and written.  Written out plainly on a full mirrored copy W:               */
/*   itype 1: W := L^{-1} W by forward substitution down each column, then    */
/*            W := W L^{-T} by forward substitution along each row;           */
/*   itype 2: W := W L (each row times L), then W := L^T W (each column).     */
/* -------------------------------------------------------------------------- */
int64_t or_sygst(int itype, int64_t n, double *A, int64_t lda, const double *L, int64_t ldl)
{
    if (itype < 1 || itype > 3) return -1;
    if (n <= 0) return 0;
    double *W = (double *)malloc((size_t)n * (size_t)n * sizeof(double));
    double *V = (double *)malloc((size_t)n * (size_t)n * sizeof(double));
    if (!W || !V) { free(W); free(V); return -2; }
#define WW(i, j) W[(size_t)(j) * (size_t)n + (size_t)(i)]
#define VV(i, j) V[(size_t)(j) * (size_t)n + (size_t)(i)]
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i)
            WW(i, j) = (i >= j) ? AT(A, lda, i, j) : AT(A, lda, j, i);
    if (itype == 1) {
        /* V := L^{-1} W, column by column */
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < n; ++j)
            for (int64_t i = 0; i < n; ++i) {
                double s = WW(i, j);
                for (int64_t k = 0; k < i; ++k) s -= AT(L, ldl, i, k) * VV(k, j);
                VV(i, j) = s / AT(L, ldl, i, i);
            }
        /* W := V L^{-T}, row by row: x L^T = v  <=>  L x^T = v^T */
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = 0; j < n; ++j) {
                double s = VV(i, j);
                for (int64_t k = 0; k < j; ++k) s -= WW(i, k) * AT(L, ldl, j, k);
                WW(i, j) = s / AT(L, ldl, j, j);
            }
    } else {
        /* V := W L */
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < n; ++j)
            for (int64_t i = 0; i < n; ++i) {
                double s = 0.0;
                for (int64_t k = j; k < n; ++k) s += WW(i, k) * AT(L, ldl, k, j);
                VV(i, j) = s;
            }
        /* W := L^T V */
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < n; ++j)
            for (int64_t i = 0; i < n; ++i) {
                double s = 0.0;
                for (int64_t k = i; k < n; ++k) s += AT(L, ldl, k, i) * VV(k, j);
                WW(i, j) = s;
            }
    }
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = j; i < n; ++i) AT(A, lda, i, j) = WW(i, j);
#undef WW
#undef VV
    free(W);
    free(V);
    return 0;
}

/* -------------------------------------------------------------------------- */
/* Error metrics.  Dot2 (Ogita, Rump & Oishi, SIAM J. Sci. Comput. 2005):     */
/* TwoSum (Knuth) and TwoProduct (Dekker, with Veltkamp's split) give a dot    */
/* product as accurate as if computed in twice the working precision.         */
/* -------------------------------------------------------------------------- */

static inline void two_sum(double a, double b, double *s, double *e)
{
    double x = a + b;
    double z = x - a;
    *e = (a - (x - z)) + (b - z);
    *s = x;
}

static inline void split(double a, double *hi, double *lo)
{
    const double factor = 134217729.0; /* 2^27 + 1 */
    double c = factor * a;
    double h = c - (c - a);
    *hi = h;
    *lo = a - h;
}

static inline void two_prod(double a, double b, double *p, double *e)
{
    double x = a * b, ah, al, bh, bl;
    split(a, &ah, &al);
    split(b, &bh, &bl);
    *e = al * bl - (((x - ah * bh) - al * bh) - ah * bl);
    *p = x;
}

typedef struct { double s, c; } dot2_t;

static inline void dot2_add(dot2_t *acc, double a, double b)
{
    double p, ep, s, es;
    two_prod(a, b, &p, &ep);
    two_sum(acc->s, p, &s, &es);
    acc->s = s;
    acc->c += ep + es;
}

static inline double dot2_val(const dot2_t *acc) { return acc->s + acc->c; }

/* 1-norm (max column sum) of a general m x n matrix. */
double or_norm1(int64_t m, int64_t n, const double *A, int64_t lda)
{
    double best = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        double s = 0.0;
        for (int64_t i = 0; i < m; ++i) s += fabs(AT(A, lda, i, j));
        if (s > best || s != s) best = s;
    }
    return best;
}

/* 1-norm of the symmetric matrix whose lower triangle is stored in A. */
double or_norm1_sym_lower(int64_t n, const double *A, int64_t lda)
{
    double best = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += fabs(i >= j ? AT(A, lda, i, j) : AT(A, lda, j, i));
        if (s > best || s != s) best = s;
    }
    return best;
}

/* 1-norm of the lower triangle of A (upper part taken as zero). */
double or_norm1_lower(int64_t n, const double *A, int64_t lda)
{
    double best = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        double s = 0.0;
        for (int64_t i = j; i < n; ++i) s += fabs(AT(A, lda, i, j));
        if (s > best || s != s) best = s;
    }
    return best;
}

/* res_chol = ||A - L L^T||_1 / (n eps ||A||_1), A symmetric (lower stored in
 * A0), L lower stored in L; eps = 2^-53. */
double or_res_chol(int64_t n, const double *A0, int64_t lda0, const double *L,
                   int64_t ldl)
{
    if (n <= 0) return 0.0;
    double *colsum = (double *)calloc((size_t)n, sizeof(double));
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < n; ++j) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            dot2_t acc = {0.0, 0.0};
            double a = i >= j ? AT(A0, lda0, i, j) : AT(A0, lda0, j, i);
            dot2_add(&acc, a, 1.0);
            int64_t kmax = i < j ? i : j;
            for (int64_t k = 0; k <= kmax; ++k)
                dot2_add(&acc, -AT(L, ldl, i, k), AT(L, ldl, j, k));
            s += fabs(dot2_val(&acc));
        }
        colsum[j] = s;
    }
    double r = 0.0;
    for (int64_t j = 0; j < n; ++j) if (colsum[j] > r || colsum[j] != colsum[j]) r = colsum[j];
    free(colsum);
    double an = or_norm1_sym_lower(n, A0, lda0);
    return r / ((double)n * ldexp(1.0, -53) * an);
}

/* res_lu = ||P A - L U||_1 / (n eps ||A||_1) for square or rectangular m x n
 * A; L unit lower m x min(m,n), U upper min(m,n) x n, both stored in LU. */
double or_res_lu(int64_t m, int64_t n, const double *A0, int64_t lda0,
                 const double *LU, int64_t ldf, const int32_t *ipiv)
{
    if (m <= 0 || n <= 0) return 0.0;
    int64_t mn = m < n ? m : n;
    /* row permutation: perm[i] = original row now at position i */
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
    for (int64_t i = 0; i < m; ++i) perm[i] = i;
    for (int64_t i = 0; i < mn; ++i) {
        int64_t p = (int64_t)ipiv[i] - 1, t = perm[i];
        perm[i] = perm[p];
        perm[p] = t;
    }
    double *colsum = (double *)calloc((size_t)n, sizeof(double));
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < n; ++j) {
        double s = 0.0;
        for (int64_t i = 0; i < m; ++i) {
            dot2_t acc = {0.0, 0.0};
            dot2_add(&acc, AT(A0, lda0, perm[i], j), 1.0);
            int64_t kmax = i < j ? i : j;
            if (kmax > mn - 1) kmax = mn - 1;
            for (int64_t k = 0; k <= kmax; ++k) {
                double l = (k == i) ? 1.0 : AT(LU, ldf, i, k);
                if (k > i) l = 0.0;
                dot2_add(&acc, -l, AT(LU, ldf, k, j));
            }
            s += fabs(dot2_val(&acc));
        }
        colsum[j] = s;
    }
    double r = 0.0;
    for (int64_t j = 0; j < n; ++j) if (colsum[j] > r || colsum[j] != colsum[j]) r = colsum[j];
    free(colsum);
    free(perm);
    double an = or_norm1(m, n, A0, lda0);
    return r / ((double)(m > n ? m : n) * ldexp(1.0, -53) * an);
}

/* res_trtri = ||L X - I||_1 / (n eps ||L||_1 ||X||_1), L and X lower
 * (non-unit). */
double or_res_trtri(int64_t n, const double *L, int64_t ldl, const double *X,
                    int64_t ldx)
{
    if (n <= 0) return 0.0;
    double *colsum = (double *)calloc((size_t)n, sizeof(double));
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < n; ++j) {
        double s = 0.0;
        for (int64_t i = j; i < n; ++i) {
            dot2_t acc = {0.0, 0.0};
            if (i == j) dot2_add(&acc, -1.0, 1.0);
            for (int64_t k = j; k <= i; ++k)
                dot2_add(&acc, AT(L, ldl, i, k), AT(X, ldx, k, j));
            s += fabs(dot2_val(&acc));
        }
        colsum[j] = s;
    }
    double r = 0.0;
    for (int64_t j = 0; j < n; ++j) if (colsum[j] > r || colsum[j] != colsum[j]) r = colsum[j];
    free(colsum);
    double ln = or_norm1_lower(n, L, ldl), xn = or_norm1_lower(n, X, ldx);
    return r / ((double)n * ldexp(1.0, -53) * ln * xn);
}

/* res_potri = ||A X - I||_1 / (n eps ||A||_1 ||X||_1), A and X symmetric
 * with their lower triangles stored. */
double or_res_potri(int64_t n, const double *A0, int64_t lda0, const double *X,
                    int64_t ldx)
{
    if (n <= 0) return 0.0;
    double *colsum = (double *)calloc((size_t)n, sizeof(double));
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < n; ++j) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            dot2_t acc = {0.0, 0.0};
            if (i == j) dot2_add(&acc, -1.0, 1.0);
            for (int64_t k = 0; k < n; ++k) {
                double a = i >= k ? AT(A0, lda0, i, k) : AT(A0, lda0, k, i);
                double x = k >= j ? AT(X, ldx, k, j) : AT(X, ldx, j, k);
                dot2_add(&acc, a, x);
            }
            s += fabs(dot2_val(&acc));
        }
        colsum[j] = s;
    }
    double r = 0.0;
    for (int64_t j = 0; j < n; ++j) if (colsum[j] > r || colsum[j] != colsum[j]) r = colsum[j];
    free(colsum);
    double an = or_norm1_sym_lower(n, A0, lda0), xn = or_norm1_sym_lower(n, X, ldx);
    return r / ((double)n * ldexp(1.0, -53) * an * xn);
}

/* Random-probe residuals for large n (O(n^2) per probe vector x):
 *   chol:  ||A x - L (L^T x)||_inf / (n eps ||A||_inf ||x||_inf)
 *   lu:    ||P A x - L (U x)||_inf / (n eps ||A||_inf ||x||_inf)
 * A symmetric lower-stored for chol; general for lu.  All sums Dot2; the
 * intermediate y = L^T x (U x) is stored in binary64, one rounding. */
static double inf_norm_sym_lower(int64_t n, const double *A, int64_t lda)
{
    double best = 0.0;
    double *rs = (double *)calloc((size_t)n, sizeof(double));
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = j; i < n; ++i) {
            double v = fabs(AT(A, lda, i, j));
            rs[i] += v;
            if (i != j) rs[j] += v;
        }
    for (int64_t i = 0; i < n; ++i) if (rs[i] > best) best = rs[i];
    free(rs);
    return best;
}

double or_probe_chol(int64_t n, const double *A0, int64_t lda0, const double *L,
                     int64_t ldl, const double *x)
{
    if (n <= 0) return 0.0;
    double *y = (double *)malloc(sizeof(double) * (size_t)n);  /* y = L^T x */
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < n; ++k) {
        dot2_t acc = {0.0, 0.0};
        for (int64_t i = k; i < n; ++i) dot2_add(&acc, AT(L, ldl, i, k), x[i]);
        y[k] = dot2_val(&acc);
    }
    double r = 0.0, xn = 0.0;
    for (int64_t i = 0; i < n; ++i) if (fabs(x[i]) > xn) xn = fabs(x[i]);
    #pragma omp parallel for schedule(dynamic, 16) reduction(max : r)
    for (int64_t i = 0; i < n; ++i) {
        dot2_t acc = {0.0, 0.0};
        for (int64_t k = 0; k < n; ++k) {
            double a = i >= k ? AT(A0, lda0, i, k) : AT(A0, lda0, k, i);
            dot2_add(&acc, a, x[k]);
        }
        for (int64_t k = 0; k <= i; ++k) dot2_add(&acc, -AT(L, ldl, i, k), y[k]);
        double v = fabs(dot2_val(&acc));
        if (v > r) r = v;
    }
    free(y);
    double an = inf_norm_sym_lower(n, A0, lda0);
    return r / ((double)n * ldexp(1.0, -53) * an * xn);
}

double or_probe_lu(int64_t n, const double *A0, int64_t lda0, const double *LU,
                   int64_t ldf, const int32_t *ipiv, const double *x)
{
    if (n <= 0) return 0.0;
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) perm[i] = i;
    for (int64_t i = 0; i < n; ++i) {
        int64_t p = (int64_t)ipiv[i] - 1, t = perm[i];
        perm[i] = perm[p];
        perm[p] = t;
    }
    double *y = (double *)malloc(sizeof(double) * (size_t)n);  /* y = U x */
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        dot2_t acc = {0.0, 0.0};
        for (int64_t k = i; k < n; ++k) dot2_add(&acc, AT(LU, ldf, i, k), x[k]);
        y[i] = dot2_val(&acc);
    }
    double r = 0.0, xn = 0.0, an = 0.0;
    for (int64_t i = 0; i < n; ++i) if (fabs(x[i]) > xn) xn = fabs(x[i]);
    #pragma omp parallel for schedule(dynamic, 16) reduction(max : r, an)
    for (int64_t i = 0; i < n; ++i) {
        dot2_t acc = {0.0, 0.0};
        double rowsum = 0.0;
        for (int64_t k = 0; k < n; ++k) {
            double a = AT(A0, lda0, perm[i], k);
            rowsum += fabs(a);
            dot2_add(&acc, a, x[k]);
        }
        for (int64_t k = 0; k < i; ++k) dot2_add(&acc, -AT(LU, ldf, i, k), y[k]);
        dot2_add(&acc, -1.0, y[i]);
        double v = fabs(dot2_val(&acc));
        if (v > r) r = v;
        if (rowsum > an) an = rowsum;
    }
    free(y);
    free(perm);
    return r / ((double)n * ldexp(1.0, -53) * an * xn);
}

/* Normwise backward error of a computed solution X of A X = B (general A),
 * per right-hand side, returning the maximum over columns:
 *   eta = ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf)
 * (Rigal and Gaches' formula for the smallest relative perturbation of A
 * and b that x solves exactly; 0 when the residual is 0). */
double or_backward_error(int64_t n, int64_t nrhs, const double *A, int64_t lda,
                         const double *X, int64_t ldx, const double *B,
                         int64_t ldb)
{
    double an = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t k = 0; k < n; ++k) s += fabs(AT(A, lda, i, k));
        if (s > an) an = s;
    }
    double worst = 0.0;
    for (int64_t j = 0; j < nrhs; ++j) {
        double rn = 0.0, xn = 0.0, bn = 0.0;
        #pragma omp parallel for schedule(dynamic, 16) reduction(max : rn)
        for (int64_t i = 0; i < n; ++i) {
            dot2_t acc = {0.0, 0.0};
            dot2_add(&acc, AT(B, ldb, i, j), 1.0);
            for (int64_t k = 0; k < n; ++k) dot2_add(&acc, -AT(A, lda, i, k), AT(X, ldx, k, j));
            double v = fabs(dot2_val(&acc));
            if (v > rn) rn = v;
        }
        for (int64_t i = 0; i < n; ++i) {
            if (fabs(AT(X, ldx, i, j)) > xn) xn = fabs(AT(X, ldx, i, j));
            if (fabs(AT(B, ldb, i, j)) > bn) bn = fabs(AT(B, ldb, i, j));
        }
        /* r = 0 is an exact solution: its backward error (the smallest
         * relative perturbation of A and b that x solves) is 0, also when
         * x = b = 0 makes the quotient 0/0 */
        double eta = (rn == 0.0) ? 0.0 : rn / (an * xn + bn);
        if (eta > worst || eta != eta) worst = eta;
    }
    return worst;
}

/* Per-level flop accounting of the recursive trtri (Section 3, the share of
 * the n^3/3 flops in the TRMM + TRSM calls of each recursion level).  Level 0
 * is the top call.  The TRMM of an n2 x n1 block with an n1 x n1 triangle and
 * the TRSM with an n2 x n2 triangle and n1 columns cost n2*n1^2 and n1*n2^2
 * flops (leading terms).  shares[l] receives the level's flops; the function
 * returns the total over all levels plus the base cases (n^3/3 each). */
double or_trtri_level_flops(int64_t n, int64_t c, double *shares, int64_t nlev,
                            int64_t level)
{
    if (n <= 0) return 0.0;
    if (n <= c) return (double)n * n * n / 3.0;
    int64_t n1 = or_split(n), n2 = n - n1;
    double here = (double)n2 * n1 * n1 + (double)n1 * n2 * n2;
    if (level < nlev) shares[level] += here;
    return here + or_trtri_level_flops(n1, c, shares, nlev, level + 1)
                + or_trtri_level_flops(n2, c, shares, nlev, level + 1);
}

/* Random-probe residuals of the inverses (O(n^2) per probe vector x):
 *   trtri: ||L (X x) - x||_inf / (n eps ||L||_inf ||X||_inf ||x||_inf)
 *   potri: ||A (X x) - x||_inf / (n eps ||A||_inf ||X||_inf ||x||_inf)
 * L, X lower triangular (trtri); A, X symmetric, lower-stored (potri). */
static double inf_norm_lower(int64_t n, const double *L, int64_t ldl)
{
    double best = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t k = 0; k <= i; ++k) s += fabs(AT(L, ldl, i, k));
        if (s > best) best = s;
    }
    return best;
}

double or_probe_trtri(int64_t n, const double *L, int64_t ldl, const double *X,
                      int64_t ldx, const double *x)
{
    if (n <= 0) return 0.0;
    double *y = (double *)malloc(sizeof(double) * (size_t)n);  /* y = X x */
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        dot2_t acc = {0.0, 0.0};
        for (int64_t k = 0; k <= i; ++k) dot2_add(&acc, AT(X, ldx, i, k), x[k]);
        y[i] = dot2_val(&acc);
    }
    double r = 0.0, xn = 0.0;
    for (int64_t i = 0; i < n; ++i) if (fabs(x[i]) > xn) xn = fabs(x[i]);
    #pragma omp parallel for schedule(dynamic, 16) reduction(max : r)
    for (int64_t i = 0; i < n; ++i) {
        dot2_t acc = {0.0, 0.0};
        dot2_add(&acc, -x[i], 1.0);
        for (int64_t k = 0; k <= i; ++k) dot2_add(&acc, AT(L, ldl, i, k), y[k]);
        double v = fabs(dot2_val(&acc));
        if (v > r) r = v;
    }
    free(y);
    return r / ((double)n * ldexp(1.0, -53) * inf_norm_lower(n, L, ldl) *
                inf_norm_lower(n, X, ldx) * xn);
}

double or_probe_potri(int64_t n, const double *A0, int64_t lda0, const double *X,
                      int64_t ldx, const double *x)
{
    if (n <= 0) return 0.0;
    double *y = (double *)malloc(sizeof(double) * (size_t)n);  /* y = X x */
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        dot2_t acc = {0.0, 0.0};
        for (int64_t k = 0; k < n; ++k)
            dot2_add(&acc, i >= k ? AT(X, ldx, i, k) : AT(X, ldx, k, i), x[k]);
        y[i] = dot2_val(&acc);
    }
    double r = 0.0, xn = 0.0;
    for (int64_t i = 0; i < n; ++i) if (fabs(x[i]) > xn) xn = fabs(x[i]);
    #pragma omp parallel for schedule(dynamic, 16) reduction(max : r)
    for (int64_t i = 0; i < n; ++i) {
        dot2_t acc = {0.0, 0.0};
        dot2_add(&acc, -x[i], 1.0);
        for (int64_t k = 0; k < n; ++k)
            dot2_add(&acc, i >= k ? AT(A0, lda0, i, k) : AT(A0, lda0, k, i), y[k]);
        double v = fabs(dot2_val(&acc));
        if (v > r) r = v;
    }
    free(y);
    return r / ((double)n * ldexp(1.0, -53) * inf_norm_sym_lower(n, A0, lda0) *
                inf_norm_sym_lower(n, X, ldx) * xn);
}


/* ========================================================================== */
/* Complex double (Section 5: every routine exists for s, d, c and z).        */
/* The same recursions with the conjugate transpose where the real ones use  */
/* the transpose: Cholesky A = L L^H (A Hermitian, lower triangle read; the  */
/* diagonal's imaginary part is ignored, as LAPACK's zpotrf does), LU with   */
/* partial pivoting on |Re| + |Im| (LAPACK's izamax), lowest row on ties.     */
/* C99 complex arithmetic; every multiply and divide is the library's.        */
/* ========================================================================== */
#include <complex.h>
typedef double complex zc_t;
#define ZT(M, ld, i, j) (M)[(size_t)(j) * (size_t)(ld) + (size_t)(i)]

static double zabs1(zc_t v) { return fabs(creal(v)) + fabs(cimag(v)); }

int64_t or_zpotf2(int64_t n, zc_t *A, int64_t lda)
{
    for (int64_t j = 0; j < n; ++j) {
        double s = 0.0;
        for (int64_t k = 0; k < j; ++k) {
            zc_t l = ZT(A, lda, j, k);
            s += creal(l) * creal(l) + cimag(l) * cimag(l);
        }
        double d = creal(ZT(A, lda, j, j)) - s;
        if (!(d > 0.0)) {
            ZT(A, lda, j, j) = d;
            return j + 1;
        }
        double ljj = sqrt(d);
        ZT(A, lda, j, j) = ljj;
        for (int64_t i = j + 1; i < n; ++i) {
            zc_t t = 0.0;
            for (int64_t k = 0; k < j; ++k) t += ZT(A, lda, i, k) * conj(ZT(A, lda, j, k));
            ZT(A, lda, i, j) = (ZT(A, lda, i, j) - t) / ljj;
        }
    }
    return 0;
}

/* B (m x n) := B L^{-H}: each row x solves x L^H = b by forward substitution. */
static void or_ztrsm_rlc(int64_t m, int64_t n, const zc_t *L, int64_t ldl, zc_t *B, int64_t ldb)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < n; ++j) {
            zc_t s = ZT(B, ldb, i, j);
            for (int64_t k = 0; k < j; ++k) s -= ZT(B, ldb, i, k) * conj(ZT(L, ldl, j, k));
            ZT(B, ldb, i, j) = s / conj(ZT(L, ldl, j, j));
        }
}

/* C (n x n, lower) -= A A^H, A n x k. */
static void or_zherk_lower(int64_t n, int64_t k, const zc_t *A, int64_t lda, zc_t *C, int64_t ldc)
{
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = j; i < n; ++i) {
            zc_t s = 0.0;
            for (int64_t p = 0; p < k; ++p) s += ZT(A, lda, i, p) * conj(ZT(A, lda, j, p));
            ZT(C, ldc, i, j) -= s;
        }
}

int64_t or_zpotrf(int64_t n, zc_t *A, int64_t lda, int64_t c)
{
    if (n <= 0) return 0;
    if (c < 1) c = 1;
    if (n <= c) return or_zpotf2(n, A, lda);
    int64_t n1 = or_split(n), n2 = n - n1;
    zc_t *A21 = &ZT(A, lda, n1, 0), *A22 = &ZT(A, lda, n1, n1);
    int64_t info = or_zpotrf(n1, A, lda, c);
    if (info) return info;
    or_ztrsm_rlc(n2, n1, A, lda, A21, lda);
    or_zherk_lower(n2, n1, A21, lda, A22, lda);
    info = or_zpotrf(n2, A22, lda, c);
    return info ? info + n1 : 0;
}

void or_zlaswp(int64_t n, zc_t *A, int64_t lda, int64_t k1, int64_t k2, const int32_t *ipiv)
{
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = k1; i < k2; ++i) {
            int64_t p = (int64_t)ipiv[i] - 1;
            if (p != i) {
                zc_t t = ZT(A, lda, i, j);
                ZT(A, lda, i, j) = ZT(A, lda, p, j);
                ZT(A, lda, p, j) = t;
            }
        }
}

int64_t or_zgetf2(int64_t m, int64_t n, zc_t *A, int64_t lda, int32_t *ipiv)
{
    int64_t info = 0, mn = m < n ? m : n;
    for (int64_t j = 0; j < mn; ++j) {
        int64_t p = j;
        double amax = zabs1(ZT(A, lda, j, j));
        for (int64_t i = j + 1; i < m; ++i) {
            double v = zabs1(ZT(A, lda, i, j));
            if (v > amax) { amax = v; p = i; }
        }
        ipiv[j] = (int32_t)(p + 1);
        if (ZT(A, lda, p, j) != 0.0) {
            if (p != j)
                for (int64_t k = 0; k < n; ++k) {
                    zc_t t = ZT(A, lda, j, k);
                    ZT(A, lda, j, k) = ZT(A, lda, p, k);
                    ZT(A, lda, p, k) = t;
                }
            zc_t piv = ZT(A, lda, j, j);
            for (int64_t i = j + 1; i < m; ++i) ZT(A, lda, i, j) = ZT(A, lda, i, j) / piv;
        } else if (info == 0) {
            info = j + 1;
        }
        for (int64_t k = j + 1; k < n; ++k) {
            zc_t u = ZT(A, lda, j, k);
            for (int64_t i = j + 1; i < m; ++i) ZT(A, lda, i, k) -= ZT(A, lda, i, j) * u;
        }
    }
    return info;
}

int64_t or_zgetrf(int64_t m, int64_t n, zc_t *A, int64_t lda, int32_t *ipiv, int64_t c)
{
    if (m <= 0 || n <= 0) return 0;
    if (c < 1) c = 1;
    int64_t mn = m < n ? m : n;
    if (n <= c || mn <= c) return or_zgetf2(m, n, A, lda, ipiv);
    int64_t n1 = or_split(mn), n2 = n - n1;
    zc_t *A12 = &ZT(A, lda, 0, n1), *A21 = &ZT(A, lda, n1, 0), *A22 = &ZT(A, lda, n1, n1);
    int64_t info = or_zgetrf(m, n1, A, lda, ipiv, c);
    or_zlaswp(n2, A12, lda, 0, n1, ipiv);
    /* A12 := L11^{-1} A12 (unit lower), column by column */
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n2; ++j)
        for (int64_t i = 0; i < n1; ++i) {
            zc_t s = ZT(A12, lda, i, j);
            for (int64_t k = 0; k < i; ++k) s -= ZT(A, lda, i, k) * ZT(A12, lda, k, j);
            ZT(A12, lda, i, j) = s;
        }
    /* A22 -= A21 A12 */
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n2; ++j)
        for (int64_t i = 0; i < m - n1; ++i) {
            zc_t s = 0.0;
            for (int64_t k = 0; k < n1; ++k) s += ZT(A21, lda, i, k) * ZT(A12, lda, k, j);
            ZT(A22, lda, i, j) -= s;
        }
    int64_t info2 = or_zgetrf(m - n1, n2, A22, lda, ipiv + n1, c);
    int64_t mn2 = (m - n1) < n2 ? (m - n1) : n2;
    for (int64_t i = 0; i < mn2; ++i) ipiv[n1 + i] += (int32_t)n1;
    if (info == 0 && info2 != 0) info = info2 + n1;
    or_zlaswp(n1, A, lda, n1, n1 + mn2, ipiv);
    return info;
}

/* ||A - L L^H||_1 / (n eps ||A||_1), A Hermitian (lower part read), Dot2
 * on the real and imaginary parts of every entry. */
double or_res_zchol(int64_t n, const zc_t *A0, int64_t lda0, const zc_t *L, int64_t ldl)
{
    if (n <= 0) return 0.0;
    double rmax = 0.0, amax = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        double s = 0.0, sa = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            const int64_t r = i >= j ? i : j, q = i >= j ? j : i;   /* lower entry (r, q) */
            zc_t a = ZT(A0, lda0, r, q);
            if (i < j) a = conj(a);
            if (i == j) a = creal(a);
            dot2_t re = {0.0, 0.0}, im = {0.0, 0.0};
            dot2_add(&re, creal(a), 1.0);
            dot2_add(&im, cimag(a), 1.0);
            const int64_t kk = (i < j ? i : j);
            for (int64_t k = 0; k <= kk; ++k) {
                zc_t x = ZT(L, ldl, i, k), y = ZT(L, ldl, j, k);   /* x conj(y) */
                dot2_add(&re, -creal(x), creal(y));
                dot2_add(&re, -cimag(x), cimag(y));
                dot2_add(&im, -cimag(x), creal(y));
                dot2_add(&im, creal(x), cimag(y));
            }
            s += hypot(dot2_val(&re), dot2_val(&im));
            sa += cabs(a);
        }
        if (s > rmax) rmax = s;
        if (sa > amax) amax = sa;
    }
    return rmax / ((double)n * 0x1p-53 * amax);
}

/* ||P A - L U||_1 / (n eps ||A||_1) for an m x n LU (P from ipiv). */
double or_res_zlu(int64_t m, int64_t n, const zc_t *A0, int64_t lda0, const zc_t *LU, int64_t ldf,
                  const int32_t *ipiv)
{
    if (m <= 0 || n <= 0) return 0.0;
    int64_t mn = m < n ? m : n;
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
    if (!perm) return -1.0;
    for (int64_t i = 0; i < m; ++i) perm[i] = i;
    for (int64_t i = 0; i < mn; ++i) {
        int64_t p = ipiv[i] - 1, t = perm[i];
        perm[i] = perm[p];
        perm[p] = t;
    }
    double rmax = 0.0, amax = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        double s = 0.0, sa = 0.0;
        for (int64_t i = 0; i < m; ++i) {
            zc_t a = ZT(A0, lda0, perm[i], j);
            dot2_t re = {0.0, 0.0}, im = {0.0, 0.0};
            dot2_add(&re, creal(a), 1.0);
            dot2_add(&im, cimag(a), 1.0);
            const int64_t kk = i < j ? i : j;
            for (int64_t k = 0; k <= kk && k < mn; ++k) {
                zc_t l = (k == i) ? 1.0 : ZT(LU, ldf, i, k), u = ZT(LU, ldf, k, j);
                dot2_add(&re, -creal(l), creal(u));
                dot2_add(&re, cimag(l), cimag(u));
                dot2_add(&im, -creal(l), cimag(u));
                dot2_add(&im, -cimag(l), creal(u));
            }
            s += hypot(dot2_val(&re), dot2_val(&im));
            sa += cabs(ZT(A0, lda0, i, j));
        }
        if (s > rmax) rmax = s;
        if (sa > amax) amax = sa;
    }
    free(perm);
    return rmax / ((double)n * 0x1p-53 * amax);
}


/* -------------------------------------------------------------------------- */
/* Complex double inversions (Section 5: the c/z peers of xtrtri, xlauum,    */
/* xpotri, xgetri), each its definition written out.                          */
/* -------------------------------------------------------------------------- */

/* X = L^{-1} (lower; unit: diagonal taken as 1) by forward substitution on
 * L x = e_j, column by column; info = first exactly-zero diagonal entry
 * (1-based, A unchanged then).  Sums accumulated in increasing k. */
int64_t or_ztrtri(int unit, int64_t n, zc_t *A, int64_t lda)
{
    if (n <= 0) return 0;
    if (!unit)
        for (int64_t i = 0; i < n; ++i)
            if (ZT(A, lda, i, i) == 0.0) return i + 1;
    zc_t *X = (zc_t *)calloc((size_t)n * (size_t)n, sizeof(zc_t));
    if (!X) return -1;
    for (int64_t j = 0; j < n; ++j) {
        X[(size_t)j * n + j] = unit ? 1.0 : 1.0 / ZT(A, lda, j, j);
        for (int64_t i = j + 1; i < n; ++i) {
            zc_t s = 0.0;
            for (int64_t k = j; k < i; ++k) s += ZT(A, lda, i, k) * X[(size_t)j * n + k];
            X[(size_t)j * n + i] = unit ? -s : -s / ZT(A, lda, i, i);
        }
    }
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = j; i < n; ++i)
            if (!(unit && i == j)) ZT(A, lda, i, j) = X[(size_t)j * n + i];
    free(X);
    return 0;
}

/* A := L^H L (lower triangle written): (L^H L)_ij = sum_{k >= i} conj(l_ki) l_kj. */
void or_zlauum(int64_t n, zc_t *A, int64_t lda)
{
    if (n <= 0) return;
    zc_t *T = (zc_t *)malloc(sizeof(zc_t) * (size_t)n * (size_t)n);
    if (!T) return;
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = j; i < n; ++i) {
            zc_t s = 0.0;
            for (int64_t k = i; k < n; ++k) s += conj(ZT(A, lda, k, i)) * ZT(A, lda, k, j);
            T[(size_t)j * n + i] = s;
        }
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = j; i < n; ++i) ZT(A, lda, i, j) = T[(size_t)j * n + i];
    free(T);
}

/* A^{-1} = (L L^H)^{-1} = L^{-H} L^{-1}: ztrtri then zlauum on the factor. */
int64_t or_zpotri(int64_t n, zc_t *A, int64_t lda)
{
    int64_t info = or_ztrtri(0, n, A, lda);
    if (info) return info;
    or_zlauum(n, A, lda);
    return 0;
}

/* X := A^{-1} from P A = L U (factors and 1-based ipiv as or_zgetrf returns
 * them), by its definition A X = I: X = I with P applied, then L Y = P,
 * then U X = Y, column by column. */
void or_zgetri(int64_t n, const zc_t *LU, int64_t lda, const int32_t *ipiv, zc_t *X, int64_t ldx)
{
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i) ZT(X, ldx, i, j) = (i == j) ? 1.0 : 0.0;
    for (int64_t i = 0; i < n; ++i) {            /* row interchanges in order */
        int64_t p = ipiv[i] - 1;
        if (p != i)
            for (int64_t j = 0; j < n; ++j) {
                zc_t t = ZT(X, ldx, i, j);
                ZT(X, ldx, i, j) = ZT(X, ldx, p, j);
                ZT(X, ldx, p, j) = t;
            }
    }
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t i = 0; i < n; ++i) {        /* L unit lower */
            zc_t s = ZT(X, ldx, i, j);
            for (int64_t k = 0; k < i; ++k) s -= ZT(LU, lda, i, k) * ZT(X, ldx, k, j);
            ZT(X, ldx, i, j) = s;
        }
        for (int64_t i = n - 1; i >= 0; --i) {   /* U upper */
            zc_t s = ZT(X, ldx, i, j);
            for (int64_t k = i + 1; k < n; ++k) s -= ZT(LU, lda, i, k) * ZT(X, ldx, k, j);
            ZT(X, ldx, i, j) = s / ZT(LU, lda, i, i);
        }
    }
}
