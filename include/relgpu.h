/*
 * relgpu.h -- C ABI of the GB300 (sm_103a) recursive dense factorizations of
 * Peise & Bientinesi, "Recursive Algorithms for Dense Linear Algebra: The
 * ReLAPACK Collection" (arXiv 1602.06763).
 *
 * The routines keep LAPACK's own argument lists (Section 5: the recursive
 * routines are drop-in replacements for LAPACK's) and add three trailing
 * arguments: a device
 * workspace, its size in bytes, and the CUDA stream to run on.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Storage: column-major with a leading dimension (LAPACK).  Element (i,j)
 *    of A is A[i + j*lda], 0-based.  Only the triangle named by `uplo` is read
 *    or written; the other triangle is left untouched.
 *  - Pointers: A, ipiv, info and work are DEVICE pointers (cudaMalloc'd or
 *    torch-allocated memory on the current device) unless the name ends in
 *    _host.  The caller owns every buffer; the library keeps no pointer after
 *    the call returns and allocates no device memory.
 *  - Streams: `stream` is a cudaStream_t (0 = legacy default stream).  The
 *    call enqueues its kernels on that stream and returns without
 *    synchronizing; results (including *info and ipiv) are valid once the
 *    stream has reached that point.  The _host variants synchronize.
 *  - Return value (host, immediate):
 *      0            success (the work was enqueued)
 *     -i            argument i is illegal, LAPACK's numbering; nothing was
 *                   enqueued and *info was not written
 *     RL_ERR_*  >0  a CUDA, workspace or support error (see rl_status_string)
 *  - Numeric result (device, asynchronous): *info (int32) is set to 0 at the
 *    start of the call and then receives LAPACK's meaning:
 *      dpotrf/dpotri: k > 0  the leading minor of order k is not positive
 *                     definite (the factorization stops there);
 *      dgetrf:        k > 0  U(k,k) is exactly zero (the factorization is
 *                     completed, as in LAPACK);
 *      dtrtri/dpotri: k > 0  A(k,k) is exactly zero (A is left unchanged);
 *      RL_INFO_DEVICE_TIMEOUT  a bounded device-side wait (the grid barrier
 *                     of the LU panel kernel) ran out; outputs are invalid.
 *  - 1-based ipiv (int32): row i was interchanged with row ipiv[i]-1.
 *  - uplo 'L' and 'U' (Section 5: LAPACK's interface).  'U' is the lower
 *    form of the transposed storage (A = U^T U with U = L^T; for complex
 *    A = U^H U with U = L^H): the call swaps A's two triangles in place
 *    (conjugating for complex), runs the lower recursion and swaps back, so
 *    the upper triangle receives the upper result and the strictly lower
 *    triangle comes back unchanged.  Inputs declared const that are
 *    transposed this way (B of rl_[ds]sygst, A of rl_[ds]potrs) are
 *    restored before the call's last kernel ends: they must be writable and
 *    must not be read by other streams while the call runs.  The BLAS-3
 *    layer (rl_dsyrk, rl_dtrsm, rl_dtrmm) keeps the subsets listed there.
 */
#ifndef RELGPU_H
#define RELGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t (CUDA's runtime declares it as this pointer). */
struct CUstream_st;
typedef struct CUstream_st *rl_stream_t;

enum {
    RL_SUCCESS = 0,
    RL_ERR_CUDA = 1,          /* a CUDA runtime call or launch failed */
    RL_ERR_WORKSPACE = 2,     /* work is NULL or lwork is below the query */
    RL_ERR_UNSUPPORTED = 3,   /* an option or a size beyond a kernel limit */
    RL_ERR_NULL_POINTER = 4,  /* info (or ipiv) is NULL */
    RL_ERR_PARAM = 5          /* rl_set_param: unknown key or bad value */
};

#define RL_INFO_DEVICE_TIMEOUT (-1000)

/* ---------------------------------------------------------------------------
 * dpotrf -- recursive Cholesky A = L L^T (Section 5, xpotrf; recursion of
 * Section 3).  With n1 ~ n/2: potrf(A11); A21 := A21 L11^{-T} (TRSM);
 * A22 := A22 - A21 A21^T (SYRK, lower triangle); potrf(A22).  Base case: an
 * unblocked Cholesky of a diagonal block in shared memory (IEEE sqrt and
 * division).  A: n x n, lower triangle overwritten by L (uplo 'L'), or
 * upper triangle by U with A = U^T U (uplo 'U', the transposed-storage form
 * described at the top of this file).
 * Argument numbers: 1 uplo, 2 n, 3 A, 4 lda, 5 info.
 * Workspace: none (work may be NULL, lwork 0).
 * ------------------------------------------------------------------------- */
int rl_dpotrf(char uplo, int64_t n, double *A, int64_t lda, int32_t *info,
              void *work, size_t lwork, rl_stream_t stream);

/* ---------------------------------------------------------------------------
 * dgetrf -- recursive LU with partial (row) pivoting, P A = L U (Section 5,
 * xgetrf; recursion of Section 3 on the columns).  With n1 ~ min(m,n)/2:
 * getrf(A[:, :n1]); apply the n1 interchanges to A[:, n1:] (LASWP);
 * A12 := L11^{-1} A12 (unit TRSM); A22 := A22 - A21 A12 (GEMM); getrf(A22);
 * apply its interchanges to A[:, :n1].  Base case: a fused panel kernel
 * (pivot search, swap, scale, rank-1 update per column) that keeps the panel
 * in shared memory across the co-resident CTAs of one cooperative launch.
 * A: m x n, overwritten by L (unit, below the diagonal) and U.
 * ipiv: min(m,n) int32, 1-based.
 * Argument numbers: 1 m, 2 n, 3 A, 4 lda, 5 ipiv, 6 info.
 * Workspace: rl_dgetrf_work_size(m, n) bytes (panel pivot exchange and the
 * grid-barrier counter); contents need not be initialized.
 * ------------------------------------------------------------------------- */
int rl_dgetrf(int64_t m, int64_t n, double *A, int64_t lda, int32_t *ipiv,
              int32_t *info, void *work, size_t lwork, rl_stream_t stream);

size_t rl_dgetrf_work_size(int64_t m, int64_t n);

/* ---------------------------------------------------------------------------
 * dtrtri -- recursive inverse of a triangular matrix in place
 * (Section 3, Fig. 4): trtri(A_TL); A_BL := A_BL A_TL (TRMM, A_TL already
 * inverted); A_BL := -A_BR^{-1} A_BL (TRSM with the not yet inverted A_BR);
 * trtri(A_BR).  Base case: an unblocked inverse in shared memory.
 * uplo 'U': the upper triangular matrix is inverted in its triangle.
 * diag: 'N' (non-unit) or 'U' (unit diagonal, not referenced).
 * Argument numbers: 1 uplo, 2 diag, 3 n, 4 A, 5 lda, 6 info.
 * Workspace: none.
 * ------------------------------------------------------------------------- */
int rl_dtrtri(char uplo, char diag, int64_t n, double *A, int64_t lda,
              int32_t *info, void *work, size_t lwork, rl_stream_t stream);

/* ---------------------------------------------------------------------------
 * dlauum -- A := L^T L for lower triangular L in place (Section 5, xlauum),
 * recursively: lauum(A11); A11 := A11 + A21^T A21 (SYRK); A21 := A22^T A21
 * (TRMM); lauum(A22).  The lower triangle of the symmetric result is
 * written (uplo 'U': A := U U^T in the upper triangle).
 * Argument numbers: 1 uplo, 2 n, 3 A, 4 lda, 5 info.
 * Workspace: none.  *info is always 0.
 * ------------------------------------------------------------------------- */
int rl_dlauum(char uplo, int64_t n, double *A, int64_t lda, int32_t *info,
              void *work, size_t lwork, rl_stream_t stream);

/* ---------------------------------------------------------------------------
 * dpotri -- inverse of an SPD matrix from its Cholesky factor: dtrtri then
 * dlauum on L (Section 5: xtrtri is the building block of xpotri), since
 * A^{-1} = L^{-T} L^{-1}.  A holds L on entry and the lower triangle of
 * A^{-1} on exit (uplo 'U': U from A = U^T U, and the upper triangle).
 * Argument numbers: 1 uplo, 2 n, 3 A, 4 lda, 5 info.
 * ------------------------------------------------------------------------- */
int rl_dpotri(char uplo, int64_t n, double *A, int64_t lda, int32_t *info,
              void *work, size_t lwork, rl_stream_t stream);

/* ---------------------------------------------------------------------------
 * Solves with computed factors (Section 5 lists xgetrf and xpotrf as the
 * building blocks of xgesv and xposv).  B (n x nrhs) is overwritten by X.
 *   rl_dgetrs: A and ipiv from rl_dgetrf: X = U^{-1} L^{-1} P B (trans 'N'),
 *     or X = P^T L^{-T} U^{-T} B (trans 'T' or 'C': A^T X = B; always the
 *     recursive TRSM, then the interchanges last first).
 *     Argument numbers: 1 trans, 2 n, 3 nrhs, 4 A, 5 lda, 6 ipiv, 7 B, 8 ldb.
 *   rl_dpotrs: A from rl_dpotrf: X = L^{-T} L^{-1} B ('L') or U^{-1} U^{-T} B ('U').
 *     Argument numbers: 1 uplo, 2 n, 3 nrhs, 4 A, 5 lda, 6 B, 7 ldb.
 * work (device, caller-owned, optional): with work == NULL both triangles
 *   are solved by the recursive TRSM (Section 3's halving on the triangle).
 *   With work != NULL and nrhs <= 64, each triangle is solved in ONE launch
 *   that streams the triangle once (64-row blocks, inverted diagonal blocks,
 *   per-block ready flags); lwork must then be >= rl_trs_work_size(n, nrhs)
 *   (a few KB), else RL_ERR_WORKSPACE.  The first int32 of work is a status:
 *   0 on completion, RL_INFO_DEVICE_TIMEOUT if a bounded device-side wait
 *   expired (read it after synchronizing).  Calls sharing one work buffer
 *   must be ordered (same stream).  With nrhs > 64, work is not used.
 * Stream-ordered; no synchronization.
 * ------------------------------------------------------------------------- */
/* dlaswp (the row interchanges of xgetrf): for k = k1..k2 (1-based, in
 * order) swap rows k and ipiv[k-1] of the m x ncols matrix A.  ipiv as
 * rl_dgetrf writes it (each target at or below its own row, <= m).  The
 * swaps are turned into their net permutation per chunk of 4096 pivots and
 * applied with one gather and one scatter per column.  Argument numbers:
 * 1 m, 2 ncols, 3 A, 4 lda, 5 k1, 6 k2.  Stream-ordered. */
int rl_dlaswp(int64_t m, int64_t ncols, double *A, int64_t lda, int64_t k1, int64_t k2,
              const int32_t *ipiv, rl_stream_t stream);
size_t rl_trs_work_size(int64_t n, int64_t nrhs);
int rl_dgetrs(char trans, int64_t n, int64_t nrhs, const double *A, int64_t lda,
              const int32_t *ipiv, double *B, int64_t ldb, void *work, size_t lwork,
              rl_stream_t stream);
int rl_dpotrs(char uplo, int64_t n, int64_t nrhs, const double *A, int64_t lda, double *B,
              int64_t ldb, void *work, size_t lwork, rl_stream_t stream);

/* ---------------------------------------------------------------------------
 * dgetri -- inverse of a general matrix from its LU factors (Section 5:
 * xtrtri is the building block of xgetri).  A and ipiv from rl_dgetrf (square
 * n); on exit A holds A^{-1} = U^{-1} L^{-1} P: U and L inverted in place by
 * the recursive TRTRI (Fig. 4 and its upper-triangular transpose), their
 * product formed in place by a recursion of GEMM/TRMM updates, then P's
 * column interchanges applied in reverse order (as LAPACK's dgetri).
 * info (device, int32): 0, or k if U(k,k) is exactly zero (A is then left
 *   unchanged, as LAPACK's dgetri leaves it when dtrtri fails).
 * work (device): rl_dgetri_work_size(n) bytes (about 8n), else
 *   RL_ERR_WORKSPACE.  n <= 40960 (the permutation plan lives in one CTA's
 *   shared memory), else RL_ERR_UNSUPPORTED.
 * Argument numbers: 1 n, 2 A, 3 lda.  Stream-ordered; no synchronization.
 * ------------------------------------------------------------------------- */
size_t rl_dgetri_work_size(int64_t n);
int rl_dgetri(int64_t n, double *A, int64_t lda, const int32_t *ipiv, int32_t *info, void *work,
              size_t lwork, rl_stream_t stream);
/* FP32 peer, same arguments and semantics. */
size_t rl_sgetri_work_size(int64_t n);
int rl_sgetri(int64_t n, float *A, int64_t lda, const int32_t *ipiv, int32_t *info, void *work,
              size_t lwork, rl_stream_t stream);

/* ---------------------------------------------------------------------------
 * dsygst (Section 5, xsygst) -- reduction of the symmetric-definite
 * generalized eigenproblem to standard form, with B's Cholesky factor L
 * (lower, from rl_dpotrf) in B:
 *   itype 1:    A := L^{-1} A L^{-T}      (A x = lambda B x)
 *   itype 2, 3: A := L^T A L              (A B x = lambda x, B A x = lambda x)
 * uplo 'L': the lower triangles of A and B are read, the lower triangle of
 * A is overwritten, the strictly upper triangles are not referenced.  uplo
 * 'U' (B = U^T U): A := U^{-T} A U^{-1} (itype 1) or U A U^T (2, 3) on the
 * upper triangles.  Recursive by halving (Section 3).
 * work (device, optional): rl_dsygst_work_size(n) bytes, about n/2 x n/2
 *   doubles, the paper's temporary buffer that saves one symmetric product
 *   per recursion level (Section 5, xsygst user note); with work == NULL the
 *   product is recomputed instead (no buffer).  A non-NULL work with lwork
 *   below the query returns RL_ERR_WORKSPACE.
 * Argument numbers: 1 itype, 2 uplo, 3 n, 4 A, 5 lda, 6 B, 7 ldb.
 * Stream-ordered; no synchronization, no numeric info (as LAPACK's dsygst).
 * ------------------------------------------------------------------------- */
size_t rl_dsygst_work_size(int64_t n);
int rl_dsygst(int itype, char uplo, int64_t n, double *A, int64_t lda, const double *B,
              int64_t ldb, void *work, size_t lwork, rl_stream_t stream);
/* FP32 peer, same arguments and semantics (work in floats: rl_ssygst_work_size). */
size_t rl_ssygst_work_size(int64_t n);
int rl_ssygst(int itype, char uplo, int64_t n, float *A, int64_t lda, const float *B,
              int64_t ldb, void *work, size_t lwork, rl_stream_t stream);

/* ---------------------------------------------------------------------------
 * Single-precision peers (Section 5: every routine exists for s, d, c and z;
 * s and d are built): the same recursions and kernels in FP32 storage and
 * arithmetic (SIMT FP32 updates).  Same arguments, numbering, workspace and
 * info semantics as the double-precision routines above.
 * ------------------------------------------------------------------------- */
int rl_spotrf(char uplo, int64_t n, float *A, int64_t lda, int32_t *info, void *work,
              size_t lwork, rl_stream_t stream);
int rl_sgetrf(int64_t m, int64_t n, float *A, int64_t lda, int32_t *ipiv, int32_t *info,
              void *work, size_t lwork, rl_stream_t stream);
int rl_strtri(char uplo, char diag, int64_t n, float *A, int64_t lda, int32_t *info,
              void *work, size_t lwork, rl_stream_t stream);
int rl_slauum(char uplo, int64_t n, float *A, int64_t lda, int32_t *info, void *work,
              size_t lwork, rl_stream_t stream);
int rl_spotri(char uplo, int64_t n, float *A, int64_t lda, int32_t *info, void *work,
              size_t lwork, rl_stream_t stream);
int rl_sgetrs(char trans, int64_t n, int64_t nrhs, const float *A, int64_t lda,
              const int32_t *ipiv, float *B, int64_t ldb, void *work, size_t lwork,
              rl_stream_t stream);
int rl_spotrs(char uplo, int64_t n, int64_t nrhs, const float *A, int64_t lda, float *B,
              int64_t ldb, void *work, size_t lwork, rl_stream_t stream);

/* ---------------------------------------------------------------------------
 * Complex double peers (Section 5: every routine exists for s, d, c and z).
 * rl_double_complex is LAPACK's complex*16 layout (re, im interleaved).
 *   rl_zpotrf: A = L L^H (Hermitian positive definite, lower triangle read;
 *     the diagonal's imaginary part is ignored), or A = U^H U (uplo 'U'),
 *     info as rl_dpotrf.
 *   rl_zgetrf: P A = L U with partial pivoting on |Re| + |Im| (LAPACK's
 *     izamax), lowest row on ties; ipiv, info and workspace
 *     (rl_dgetrf_work_size) as rl_dgetrf; panels of at most 32 columns.
 * Same recursions and argument numbering as the double-precision routines.
 * ------------------------------------------------------------------------- */
typedef struct { double re, im; } rl_double_complex;
int rl_zpotrf(char uplo, int64_t n, rl_double_complex *A, int64_t lda, int32_t *info,
              void *work, size_t lwork, rl_stream_t stream);
int rl_zgetrf(int64_t m, int64_t n, rl_double_complex *A, int64_t lda, int32_t *ipiv,
              int32_t *info, void *work, size_t lwork, rl_stream_t stream);
/* rl_zgetrs (trans 'N'; 'T'/'C' return RL_ERR_UNSUPPORTED) and rl_zpotrs
 * (uplo 'L': X = L^{-H} L^{-1} B; 'U': U^{-1} U^{-H} B): the solves of
 * rl_dgetrs / rl_dpotrs for the complex factors, by the recursive TRSM
 * (work and lwork are accepted and ignored).  Argument numbers as there. */
int rl_zgetrs(char trans, int64_t n, int64_t nrhs, const rl_double_complex *A, int64_t lda,
              const int32_t *ipiv, rl_double_complex *B, int64_t ldb, void *work, size_t lwork,
              rl_stream_t stream);
int rl_zpotrs(char uplo, int64_t n, int64_t nrhs, const rl_double_complex *A, int64_t lda,
              rl_double_complex *B, int64_t ldb, void *work, size_t lwork, rl_stream_t stream);
/* Complex double inversions, as their double-precision peers:
 *   rl_ztrtri  A := A^{-1} (lower or upper, diag 'N'/'U'), info = first
 *              zero diagonal entry (A unchanged then);
 *   rl_zlauum  A := L^H L ('L') or U U^H ('U');
 *   rl_zpotri  A := (L L^H)^{-1} from rl_zpotrf's factor (trtri + lauum);
 *   rl_zgetri  A := A^{-1} from rl_zgetrf's factors and ipiv, workspace
 *              rl_zgetri_work_size(n) bytes, n <= 40960.
 * Base cases of order <= 32 (complex elements double the shared memory per
 * entry); argument numbers as rl_dtrtri / rl_dlauum / rl_dpotri /
 * rl_dgetri. */
int rl_ztrtri(char uplo, char diag, int64_t n, rl_double_complex *A, int64_t lda, int32_t *info,
              void *work, size_t lwork, rl_stream_t stream);
int rl_zlauum(char uplo, int64_t n, rl_double_complex *A, int64_t lda, int32_t *info, void *work,
              size_t lwork, rl_stream_t stream);
int rl_zpotri(char uplo, int64_t n, rl_double_complex *A, int64_t lda, int32_t *info, void *work,
              size_t lwork, rl_stream_t stream);
size_t rl_zgetri_work_size(int64_t n);
int rl_zgetri(int64_t n, rl_double_complex *A, int64_t lda, const int32_t *ipiv, int32_t *info,
              void *work, size_t lwork, rl_stream_t stream);

/* ---------------------------------------------------------------------------
 * FP64 updates emulated on the BF16 tensor cores (the Ozaki scheme; not in
 * the paper).  Row i of op(A) and column j of op(B) are scaled by powers of
 * two 2^-eA_i, 2^-eB_j (max |entry| < 2^(e-1)), rounded to 8*slices-bit
 * fixed point and cut into `slices` signed 8-bit digits (exact in BF16);
 * the digit products of significance above 2^(-8*slices-8) are summed by
 * tcgen05 MMAs in exact FP32 blocks of 128 values of k, then in 64-bit
 * integers, and converted to FP64 once.  Error: below (slices + 1) * k *
 * 2^(-8*slices-2) * 2^(eA_i + eB_j) per entry plus the final rounding
 * (normwise like an FP64 GEMM from slices = 7 on);
 * integer inputs whose row and column maxima are below 2^(8*slices-1) give
 * the exact product wherever it is below 2^53.  Inputs must be finite (a
 * row or column holding Inf or NaN gives NaN in its row or column of C).
 *   slices: 6, 7 (FP64-level accuracy) or 8; else argument 1 is illegal.
 *   rl_dgemm_oz: C := beta C + alpha op(A) op(B) (transa/transb 'N'/'T');
 *     k <= 2^21; work >= rl_oz_work_size(m, n, k, slices) bytes (device):
 *     the digit planes, 2 * slices bytes per element of op(A) and op(B)
 *     padded to 128 x 64 tiles.  Argument numbers: 1 slices, 2 transa,
 *     3 transb, 4 m, 5 n, 6 k, 9 lda, 11 ldb, 14 ldc.
 *   rl_dpotrf_oz / rl_dgetrf_oz: rl_dpotrf / rl_dgetrf with every GEMM/SYRK
 *     update of order >= RL_PARAM_OZ_MIN (m, n and k) emulated; same
 *     results, info and ipiv semantics (within the scheme's error);
 *     workspace rl_dpotrf_oz_work_size(n, slices) /
 *     rl_dgetrf_oz_work_size(m, n, slices) (the LU's includes its panel
 *     workspace; the Cholesky's holds two sets of digit planes, one for the
 *     lookahead's side stream, whose updates then run beside the next
 *     level's).  Argument numbers shift by one (1 = slices).
 * ------------------------------------------------------------------------- */
size_t rl_oz_work_size(int64_t m, int64_t n, int64_t k, int slices);
int rl_dgemm_oz(int slices, char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                const double *A, int64_t lda, const double *B, int64_t ldb, double beta, double *C,
                int64_t ldc, void *work, size_t lwork, rl_stream_t stream);
size_t rl_dpotrf_oz_work_size(int64_t n, int slices);
size_t rl_dgetrf_oz_work_size(int64_t m, int64_t n, int slices);
int rl_dpotrf_oz(int slices, char uplo, int64_t n, double *A, int64_t lda, int32_t *info, void *work,
                 size_t lwork, rl_stream_t stream);
int rl_dgetrf_oz(int slices, int64_t m, int64_t n, double *A, int64_t lda, int32_t *ipiv, int32_t *info,
                 void *work, size_t lwork, rl_stream_t stream);

/* ---------------------------------------------------------------------------
 * Low-precision factorizations (the factorization step of the precision
 * form, callable on its own): rl_spotrf / rl_sgetrf on FP32 storage with
 * every large GEMM/SYRK update on the tensor cores (tcgen05) with operands in
 * `prec` -- RL_PREC_TF32, RL_PREC_BF16, RL_PREC_FP16S (FP16 operands; no
 * scaling here: the caller keeps |A| in FP16 range) or RL_PREC_TF32X3 (three
 * TF32 products, ~FP32 accuracy) -- and FP32 accumulation; panels, TRSM
 * leaves and small updates stay FP32 SIMT.  The paper has no precision form.
 * work (device): rl_s{potrf,getrf}_tc_work_size bytes (operand packing for the
 *   tensor cores, plus the LU panel exchange), else RL_ERR_WORKSPACE;
 *   prec RL_PREC_FP32 or unknown: RL_ERR_UNSUPPORTED (use rl_spotrf/rl_sgetrf).
 * Argument numbers: 1 prec, then those of rl_spotrf / rl_sgetrf shifted by one.
 * info as rl_spotrf / rl_sgetrf.  Stream-ordered; no synchronization.
 * ------------------------------------------------------------------------- */
size_t rl_spotrf_tc_work_size(int64_t n, int prec);
size_t rl_sgetrf_tc_work_size(int64_t m, int64_t n, int prec);
int rl_spotrf_tc(int prec, char uplo, int64_t n, float *A, int64_t lda, int32_t *info,
                 void *work, size_t lwork, rl_stream_t stream);
int rl_sgetrf_tc(int prec, int64_t m, int64_t n, float *A, int64_t lda, int32_t *ipiv,
                 int32_t *info, void *work, size_t lwork, rl_stream_t stream);

/* ---------------------------------------------------------------------------
 * Precision form: A X = B (FP64) solved with a low-precision factorization
 * and FP64 iterative refinement, following the semantics of LAPACK's dsgesv
 * (LU) and dsposv (Cholesky).  The paper has no precision form; the
 * factorization itself is the paper's recursion (Section 3) run in FP32
 * storage, with the trailing updates in the precision `prec`:
 *   RL_PREC_FP32   FP32 products and accumulation (SIMT)
 *   RL_PREC_TF32   TF32 products, FP32 accumulation (tcgen05 tensor cores)
 *   RL_PREC_BF16   BF16 products, FP32 accumulation (tcgen05)
 *   RL_PREC_FP16S  FP16 products, FP32 accumulation (tcgen05); A is scaled by
 *                  a power of two so that its entries are at most 1
 *   RL_PREC_TF32X3 three TF32 products per term (a = a_hi + a_lo split),
 *                  close to FP32 accuracy (tcgen05)
 * Updates smaller than 128 x 128 x 64 stay on the SIMT FP32 path.
 * A copy of A is converted to FP32 in `work` and factored; x0 = solve(b);
 * then r = b - A x in FP64 and x += solve(r) until, for every column,
 * ||r||_inf <= tol (||A||_inf ||x||_inf + ||b||_inf) (tol <= 0 means 1e-14),
 * or maxiter corrections were applied, or a correction reduced the largest
 * backward error by less than 10 %.  Without convergence, or when the
 * FP32 factorization fails, A is factored in FP64 in place (A then holds the
 * FP64 factors, and ipiv their pivots) and X = A^{-1} B.
 * Outputs (device, asynchronous): X (n x nrhs, ldx), ipiv (LU), *iter:
 *   >= 0  corrections applied before convergence (A unchanged)
 *   -2    an entry of A overflows FP32; -3 the FP32 factorization failed;
 *   -31   no convergence within maxiter, or a correction that reduced the
 *         largest backward error by less than 10 % (the FP64 fallback was
 *         used)
 * and *info: LAPACK's info of the FP64 fallback factorization (0 otherwise).
 * nrhs <= 512.  Workspace: rl_dsgesv_work_size / rl_dsposv_work_size bytes.
 *
 * prec | RL_REFINE_GMRES selects GMRES-based refinement (not in the paper;
 * E. Carson and N. J. Higham, SIAM J. Sci. Comput. 2017/2018, in the
 * flexible form of A. Haidar et al., SC18) for factorizations too inexact
 * for the classic loop (kappa(A) u >= 1, e.g. BF16 or FP16 updates at
 * kappa = 1e6): after x0 = solve(b), each refinement step solves the
 * correction equation A d = r by restarted flexible GMRES, right
 * preconditioned by the low-precision factors (applied in FP32), with the
 * Krylov basis, the products A z (A in FP64) and the least-squares problem
 * in FP64; a cycle ends for a column once its residual is below 1e-4 of
 * the cycle's start (or below half of what tol allows), after
 * RL_PARAM_GMRES_RESTART iterations, or when the budget is spent.  maxiter
 * then bounds the total number of GMRES iterations (preconditioner
 * applications) and *iter >= 0 reports that number; the refinement is
 * abandoned for the FP64 fallback (*iter = -31) when the budget is spent or
 * a cycle reduces the largest backward error by less than half.  nrhs <= 64
 * with this flag; the work size depends on the flag and on the restart
 * length in force when it is queried.
 *
 * prec | RL_REFINE_OZRES (with either refinement; not in the paper): the
 * FP64 products of the refinement -- the residuals b - A x and GMRES's
 * A z -- are emulated on the BF16 tensor cores (the Ozaki scheme with 7
 * digit planes, as rl_dgemm_oz): A's planes are made once per call (14 bytes
 * per element of A in the workspace) and each product slices only x.  The
 * products are exact in the digits kept: per entry the error is below
 * 8 n 2^-58 2^(e_i + e_x) (2^e_i, 2^e_x: powers of two just above the
 * largest |a_ik| of row i and the largest |x_k|), normwise the accuracy of
 * an FP64 product, so the backward-error test and the corrections keep FP64
 * accuracy; the products run at tensor-core rather than FP64-pipe rates.
 * Argument numbers (dsgesv): 1 n, 2 nrhs, 3 A, 4 lda, 5 ipiv, 6 B, 7 ldb,
 * 8 X, 9 ldx; (dsposv): 1 uplo, 2 n, 3 nrhs, 4 A, 5 lda, 6 B, 7 ldb, 8 X,
 * 9 ldx.
 * ------------------------------------------------------------------------- */
enum { RL_PREC_FP32 = 0, RL_PREC_TF32 = 1, RL_PREC_BF16 = 2, RL_PREC_FP16S = 3, RL_PREC_TF32X3 = 4 };
enum { RL_PREC_MASK = 0xff, RL_REFINE_GMRES = 0x100, RL_REFINE_OZRES = 0x200 };
size_t rl_dsgesv_work_size(int64_t n, int64_t nrhs, int prec);
size_t rl_dsposv_work_size(int64_t n, int64_t nrhs, int prec);
int rl_dsgesv(int64_t n, int64_t nrhs, double *A, int64_t lda, int32_t *ipiv, const double *B,
              int64_t ldb, double *X, int64_t ldx, int prec, double tol, int maxiter,
              int32_t *iter, int32_t *info, void *work, size_t lwork, rl_stream_t stream);
int rl_dsposv(char uplo, int64_t n, int64_t nrhs, double *A, int64_t lda, const double *B,
              int64_t ldb, double *X, int64_t ldx, int prec, double tol, int maxiter,
              int32_t *iter, int32_t *info, void *work, size_t lwork, rl_stream_t stream);

/* ---------------------------------------------------------------------------
 * BLAS-3 layer (Section 2: the Level-3 kernels the recursions are built on),
 * exported for direct use and per-kernel measurement.  BLAS semantics and
 * argument numbering; all matrices on the device, stream-ordered, no
 * workspace.  Supported options (others return RL_ERR_UNSUPPORTED):
 *   rl_dgemm  any transa/transb: C := alpha op(A) op(B) + beta C
 *   rl_dsyrk  uplo 'L', trans 'N' (C := alpha A A^T + beta C) or 'T'
 *             (C := alpha A^T A + beta C); only the lower triangle is written
 *   rl_dtrsm  uplo 'L' with (side 'L', transa 'N', diag 'N'/'U'),
 *             (side 'L', transa 'T', diag 'N'), (side 'R', transa 'T',
 *             diag 'N'); and uplo 'U', side 'L', transa 'N', diag 'N'
 *   rl_dtrmm  uplo 'L', alpha 1, with (side 'R', transa 'N', diag 'N'/'U')
 *             or (side 'L', transa 'T', diag 'N')
 * TRSM and TRMM recurse by halving the triangle (GEMM off the diagonal,
 * substitution in shared memory for blocks of order <= 64).
 * ------------------------------------------------------------------------- */
int rl_dgemm(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
             const double *A, int64_t lda, const double *B, int64_t ldb, double beta,
             double *C, int64_t ldc, rl_stream_t stream);
int rl_dsyrk(char uplo, char trans, int64_t n, int64_t k, double alpha, const double *A,
             int64_t lda, double beta, double *C, int64_t ldc, rl_stream_t stream);
/* FP32 peers of rl_dgemm / rl_dsyrk (SIMT FP32 arithmetic: the update kernels
 * of the FP32 precision form and of rl_spotrf / rl_sgetrf). */
int rl_sgemm(char transa, char transb, int64_t m, int64_t n, int64_t k, float alpha,
             const float *A, int64_t lda, const float *B, int64_t ldb, float beta, float *C,
             int64_t ldc, rl_stream_t stream);
int rl_ssyrk(char uplo, char trans, int64_t n, int64_t k, float alpha, const float *A,
             int64_t lda, float beta, float *C, int64_t ldc, rl_stream_t stream);
int rl_dtrsm(char side, char uplo, char transa, char diag, int64_t m, int64_t n,
             double alpha, const double *A, int64_t lda, double *B, int64_t ldb,
             rl_stream_t stream);
int rl_dtrmm(char side, char uplo, char transa, char diag, int64_t m, int64_t n,
             double alpha, const double *A, int64_t lda, double *B, int64_t ldb,
             rl_stream_t stream);

/* ---------------------------------------------------------------------------
 * Batching form: `batch` independent factorizations of orders up to 256 in
 * one persistent launch (the paper has no batched form; each matrix follows
 * the Section 3 scheme with 32-column halves).  Matrix b is the n[b] x n[b]
 * column-major array at A[b] with leading dimension lda[b]; n, A, lda, ipiv
 * and info are DEVICE arrays of `batch` entries (A[b] and ipiv[b] device
 * pointers).  max_n (host) bounds n[b] and must be <= 256.  info[b] follows
 * LAPACK for matrix b (dpotrf: first non-positive minor; dgetrf: first zero
 * pivot, factorization completed); ipiv[b] has n[b] 1-based entries.
 * A matrix with n[b] = 0 is left alone with info[b] = 0; one with n[b] < 0
 * or n[b] > 256 gets info[b] = -3 (potrf) / -2 (getrf), one with
 * lda[b] < max(1, n[b]) gets info[b] = -5 / -4 (LAPACK's argument numbers
 * of the order and leading-dimension arrays), and is not touched.
 * Workspace: rl_potrf_vbatched_work_size / rl_getrf_vbatched_work_size
 * bytes (the size-sorted work list and its counter).
 * Argument numbers: potrf 1 uplo, 2 batch; getrf 1 batch.
 * ------------------------------------------------------------------------- */
size_t rl_potrf_vbatched_work_size(int64_t batch);
size_t rl_getrf_vbatched_work_size(int64_t batch);
int rl_dpotrf_vbatched(char uplo, int64_t batch, const int32_t *n, double *const *A,
                       const int32_t *lda, int32_t *info, int32_t max_n, void *work,
                       size_t lwork, rl_stream_t stream);
int rl_spotrf_vbatched(char uplo, int64_t batch, const int32_t *n, float *const *A,
                       const int32_t *lda, int32_t *info, int32_t max_n, void *work,
                       size_t lwork, rl_stream_t stream);
int rl_dgetrf_vbatched(int64_t batch, const int32_t *n, double *const *A, const int32_t *lda,
                       int32_t *const *ipiv, int32_t *info, int32_t max_n, void *work,
                       size_t lwork, rl_stream_t stream);
int rl_sgetrf_vbatched(int64_t batch, const int32_t *n, float *const *A, const int32_t *lda,
                       int32_t *const *ipiv, int32_t *info, int32_t max_n, void *work,
                       size_t lwork, rl_stream_t stream);

/* ---------------------------------------------------------------------------
 * Autotuner of the batching form.  rl_vbatched_tune times each of the
 * RL_BATCH_CONFIGS candidate configurations of the batched kernels -- block
 * width NB (16 or 32: matrices are factored in NB-column halves), CTA size
 * (128 or 256 threads) and CTAs per SM -- on the caller's own batch, twice
 * each, and keeps the fastest for later rl_{d,s}{potrf,getrf}_vbatched calls
 * of that routine and element type (process-wide).  The matrices are saved
 * to `work` first and restored before every run and at the end, so A is
 * unchanged on return (ipiv and info hold the last run's values).
 *   routine 'P' (Cholesky, lower) or 'G' (LU); elem_bytes 8 (double) or 4
 *   (float); the batch arguments are those of the vbatched calls (ipiv may be
 *   NULL for 'P').  work: rl_vbatched_tune_work_size(batch, sum over the batch
 *   of n[b]^2, elem_bytes) bytes.  best (host): the chosen configuration;
 *   ms_per_config (host, RL_BATCH_CONFIGS floats, or NULL): the best of two
 *   times of each.  This call SYNCHRONIZES the stream (it reads the orders
 *   back and times with events).  The paper has no batched form.
 * rl_vbatched_config reports the configuration in use (host outputs, any may
 *   be NULL); rl_vbatched_set_config selects one (0 .. RL_BATCH_CONFIGS-1,
 *   else -3).  Argument numbers: 1 routine, 2 elem_bytes, 3 batch / cfg.
 * ------------------------------------------------------------------------- */
#define RL_BATCH_CONFIGS 8
size_t rl_vbatched_tune_work_size(int64_t batch, int64_t sum_n2, int elem_bytes);
int rl_vbatched_tune(char routine, int elem_bytes, int64_t batch, const int32_t *n, void *const *A,
                     const int32_t *lda, int32_t *const *ipiv, int32_t *info, int32_t max_n,
                     void *work, size_t lwork, int32_t *best, float *ms_per_config,
                     rl_stream_t stream);
int rl_vbatched_config(char routine, int elem_bytes, int32_t *cfg, int32_t *nb, int32_t *threads,
                       int32_t *per_sm);
int rl_vbatched_set_config(char routine, int elem_bytes, int32_t cfg);

/* ---------------------------------------------------------------------------
 * rl_dgetrf_vbatched_noalloc -- rl_dgetrf_vbatched without a workspace
 * argument.  The paper has no counterpart: it is a calling convention for
 * callers that cannot allocate device memory where they call (a cudaMalloc
 * there would synchronize the device or is not permitted, e.g. inside a
 * latency-critical loop or a host without its own device allocator).
 * Arguments and results are those of rl_dgetrf_vbatched (argument 1 batch,
 * 2 n, 3 A, 4 lda, 5 ipiv, 6 info, 7 max_n).
 * Scratch: a library-owned static device array of 256 + 4 * 65536 bytes
 *   (262,400 B) per device; batch > 65536 returns RL_ERR_UNSUPPORTED before
 *   any device work.  The first call on a device resolves the array's
 *   device address (set-up done once per device, with that device current),
 *   so make the first call before any stream capture.
 * Every call on a device shares the array: calls that may overlap in time
 *   (different streams, or host threads without ordering) race on it and
 *   must be serialized by the caller.  Nothing in it needs to start at zero
 *   (each call rewrites the order list and resets its work counter).
 * Allocates nothing (no cudaMalloc / cudaFree, no allocating library call).
 * ------------------------------------------------------------------------- */
int rl_dgetrf_vbatched_noalloc(int64_t batch, const int32_t *n, double *const *A,
                               const int32_t *lda, int32_t *const *ipiv, int32_t *info,
                               int32_t max_n, rl_stream_t stream);

/* ---------------------------------------------------------------------------
 * Tensor-core GEMM on FP32 storage (the update kernel of the precision
 * form): C(m x n) := C + alpha op(A) op(B), A, B, C single precision,
 * column-major, products in `prec` (RL_PREC_TF32, _BF16, _FP16S, _TF32X3) on
 * the tcgen05 tensor cores with FP32 accumulation.  op(A) and op(B) are first
 * packed into `work` (rl_sgemm_tc_work_size bytes).  Argument numbers:
 * 1 prec, 2 transa, 3 transb, 4 m, 5 n, 6 k, 7 alpha, 8 A, 9 lda, 10 B,
 * 11 ldb, 12 C, 13 ldc.  RL_PREC_FP32 or sizes the kernel cannot take return
 * RL_ERR_UNSUPPORTED.
 * ------------------------------------------------------------------------- */
size_t rl_sgemm_tc_work_size(int64_t m, int64_t n, int64_t k, int prec);
int rl_sgemm_tc(int prec, char transa, char transb, int64_t m, int64_t n, int64_t k, float alpha,
                const float *A, int64_t lda, const float *B, int64_t ldb, float *C, int64_t ldc,
                void *work, size_t lwork, rl_stream_t stream);

/* ---------------------------------------------------------------------------
 * Host-buffer forms (end-to-end use from host memory).  A_host (and
 * ipiv_host, info_host) are HOST pointers, ideally page-locked.  `work` is a
 * device buffer of at least rl_host_work_size(routine, m, n, lda) bytes that holds
 * the device copy of A plus the routine's workspace.  The call copies A to
 * the device, factors it on `stream`, copies the results back and
 * synchronizes the stream before returning.  Argument numbering and errors
 * as for the device forms.  routine: "dpotrf" or "dgetrf".
 * ------------------------------------------------------------------------- */
size_t rl_host_work_size(const char *routine, int64_t m, int64_t n, int64_t lda);

int rl_dpotrf_host(char uplo, int64_t n, double *A_host, int64_t lda,
                   int32_t *info_host, void *work, size_t lwork,
                   rl_stream_t stream);

int rl_dgetrf_host(int64_t m, int64_t n, double *A_host, int64_t lda,
                   int32_t *ipiv_host, int32_t *info_host, void *work,
                   size_t lwork, rl_stream_t stream);

/* ---------------------------------------------------------------------------
 * Tuning parameters (process-wide; take effect for calls enqueued after the
 * change).  The paper's crossover size c (Section 3) is set per routine.
 *   RL_PARAM_POTRF_CROSSOVER   order at or below which dpotrf runs its base
 *                              case (1..64, default 64)
 *   RL_PARAM_GETRF_PANEL       panel width of dgetrf's base case (1..64,
 *                              default 32)
 *   RL_PARAM_TRTRI_CROSSOVER   base-case order for dtrtri/dlauum (1..64,
 *                              default 64)
 *   RL_PARAM_SPIN_LIMIT_NS     bound on every device-side wait, in ns
 *                              (default 2e9); 0 makes any wait that is not
 *                              already satisfied fail with
 *                              RL_INFO_DEVICE_TIMEOUT.  The tensor-core
 *                              kernels' final waits for their own copies
 *                              and MMAs in flight (before a CTA frees its
 *                              tensor memory and exits) are never shorter
 *                              than 1 s, whatever this value
 *   RL_PARAM_BATCH_CTAS        CTAs per SM of the batched kernels (0 = as
 *                              many as fit, the default; 1..8)
 *   RL_PARAM_TRI_LANES         lanes per vector of the triangle kernels at
 *                              the TRSM/TRMM leaves: 0 (default) picks 2
 *                              for leaves of >= 12288 vectors, else 4; 2 or
 *                              4 force one; all give bit-identical results
 *   RL_PARAM_LOOKAHEAD         1 (default): the LU and Cholesky recursions
 *                              run the part of each large trailing update
 *                              that the next level needs last on an internal
 *                              stream, beside that level's first half (same
 *                              results, bit for bit); 0: the caller's stream
 *                              alone.  Factorizations whose updates run on
 *                              the tensor cores (precision form) share one
 *                              packing workspace and run on one stream.
 *   RL_PARAM_PANEL_CTAS        CTAs of the LU panel kernel: low 16 bits for
 *                              FP64 panels, high 16 bits for FP32 panels
 *                              (0, the default: one per SM; at most 256
 *                              rows each either way)
 *   RL_PARAM_OZ_MIN            smallest m, n and k of an FP64 update that
 *                              the *_oz routines emulate on the tensor
 *                              cores (default 128; smaller ones stay FP64)
 *   RL_PARAM_PANEL_CLUSTER     1 (default): FP32 LU panels (width <= 32,
 *                              at most 16384 rows) run on one cluster of
 *                              2, 4, 8 or 16 CTAs that holds the panel in
 *                              registers and exchanges the pivot candidates
 *                              through distributed shared memory (one
 *                              hardware cluster barrier per column); 0: the
 *                              cooperative one-CTA-per-SM panel kernel.
 *                              Both give the same bits.
 *   RL_PARAM_TC_PAIRS          1 (default): the tensor-core GEMM of the
 *                              precision form runs pairs of row tiles on
 *                              clusters of two CTAs that share the B tile
 *                              (each loads half and multicasts it); 0: one
 *                              CTA per tile.  Both give the same bits.
 *   RL_PARAM_GMRES_RESTART     restart length of the GMRES refinement of
 *                              rl_dsgesv / rl_dsposv (1..64, default 50)
 *   RL_PARAM_NVTX              1: every recursion node (potrf, getrf,
 *                              trtri, lauum) pushes an NVTX range named by
 *                              routine, order and depth, for timeline
 *                              tools; 0 (default): none
 * rl_set_param returns 0 or RL_ERR_PARAM; rl_get_param returns the value or
 * -1 for an unknown key.
 * ------------------------------------------------------------------------- */
enum {
    RL_PARAM_POTRF_CROSSOVER = 1,
    RL_PARAM_GETRF_PANEL = 2,
    RL_PARAM_TRTRI_CROSSOVER = 3,
    RL_PARAM_SPIN_LIMIT_NS = 4,
    RL_PARAM_BATCH_CTAS = 5,
    RL_PARAM_TRI_LANES = 6,
    RL_PARAM_LOOKAHEAD = 7,
    RL_PARAM_PANEL_CTAS = 8,
    RL_PARAM_OZ_MIN = 9,
    RL_PARAM_NVTX = 10,
    RL_PARAM_GMRES_RESTART = 11,
    RL_PARAM_PANEL_CLUSTER = 12,
    RL_PARAM_TC_PAIRS = 13
};
int rl_set_param(int key, int64_t value);
int64_t rl_get_param(int key);

/* Number of kernels this library has launched in this process (host-side
 * count, for accounting in benchmarks). */
/* rl_clear_cache: release what the library keeps between calls: the
 * internal low-priority stream of each device used by the lookahead of the
 * LU/Cholesky recursions (synchronized, then destroyed), the calling
 * thread's lookahead events, and the trace's event pool (tracing stops).
 * Each is created again on first use.  Not to be called while another
 * thread has a library call in flight.  RL_SUCCESS or RL_ERR_CUDA (the first
 * CUDA error met; the rest is released anyway).  Other host threads' event
 * pools are not reachable from here and stay until the process ends. */
int rl_clear_cache(void);
uint64_t rl_launch_count(void);

/* ---------------------------------------------------------------------------
 * Per-kernel tracing, the GPU analogue of the paper's per-kernel time and
 * efficiency breakdown (Section 3, Figs. 2 and 5).  While enabled, every
 * kernel the library launches is bracketed by two CUDA events on its stream
 * (so traced calls are not meant for graph capture) and its algorithmic
 * flops and bytes are attributed to its kind.
 *   rl_trace_enable(1) clears the totals and starts tracing; (0) stops.
 *   rl_trace_kinds() is the number of kinds; rl_trace_read(kind, ...)
 *   synchronizes on the recorded events and returns the kind's name, launch
 *   count, total device time (ms), flops and bytes.  Any output pointer may
 *   be NULL.  Returns 0 or RL_ERR_PARAM for a bad kind.
 * ------------------------------------------------------------------------- */
int rl_trace_enable(int on);
int rl_trace_kinds(void);
int rl_trace_read(int kind, const char **name, uint64_t *launches, double *ms,
                  double *flops, double *bytes);

/* Human-readable text for a return value of any entry point. */
const char *rl_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* RELGPU_H */
