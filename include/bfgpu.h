/*
 * bfgpu.h -- C ABI of the batched panel-major FP64 BLAS/LAPACK routines for
 * GB300 (sm_103a).
 *
 * The routines are the level-3 BLAS- and LAPACK-like operations that BLASFEO
 * (Frison et al., "BLASFEO: basic linear algebra subroutines for embedded
 * optimization") builds on the panel-major matrix format: gemm_nt, syrk_ln,
 * potrf_l, trsm_rltn and the fused syrk_potrf_ln.  Each routine exists in the
 * paper's single-problem form and in a batched form that runs many
 * independent problems of the same shape in one launch.
 *
 * Conventions shared by every entry point (Appendix A.2 of the paper):
 *   - Sizes come first, then the operands.  A matrix operand is a descriptor
 *     plus the row and column (ai, aj) of the first element of the
 *     sub-matrix that is the actual operand.  Option letters (n/t, l/r, ...)
 *     are part of the routine name.
 *   - Routines are non-destructive: the output has its own operand, which
 *     may coincide with an input where stated.
 *   - All matrix memory is DEVICE memory owned by the caller.  The library
 *     never allocates, frees or keeps a pointer past the call.
 *   - Descriptors are plain host structs passed by pointer; only the memory
 *     they point at lives on the device.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Every
 *     call is asynchronous on that stream.
 *   - Batched forms: problem b (0 <= b < batch) of operand X uses the matrix
 *     whose storage starts at X->pA + b * strideX (stride in doubles).  All
 *     problems share the sizes, the offsets and X's descriptor fields.
 *
 * Return value of every routine:
 *     0               success (the work is queued on `stream`)
 *    -i  (i >= 1)     argument i (1-based position in the call) is invalid;
 *                     nothing was launched
 *    BF_ERR_UNSUPPORTED  the sizes are valid but beyond what the kernels
 *                     implement (see each routine)
 *    > 0 otherwise    a cudaError_t returned by the launch
 * Numerical failure of a factorization is not an error of the call: it is
 * reported per problem in the `info` array (see bf_dpotrf_l_batched).
 */
#ifndef BFGPU_H
#define BFGPU_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Panel height ps of the GPU panel-major format (Sec. 4.3.3).  A power of
 * two, fixed at build time for every matrix, as the paper requires.  Four
 * doubles (32 bytes, one DRAM sector per panel column) keeps the padding of
 * the smallest matrices (n = 4) at zero. */
#define BF_PS 4

/* Memory alignment in bytes that bf_memsize_dmat rounds up to. */
#define BF_ALIGN 256

#define BF_ERR_UNSUPPORTED 100000

/* Returned by bf_dposv_mixed_batched_noalloc when the problem needs more
 * scratch than its fixed array holds. */
#define BF_ERR_TOO_LARGE 100001

/* Bytes of the fixed scratch array of bf_dposv_mixed_batched_noalloc. */
#define BF_NOALLOC_WORK_BYTES (16 * 1024 * 1024)

/* Matrix descriptor: the blasfeo_dmat structure of Appendix A.1.1 with the
 * members that the panel-major format needs (Sec. 4.3.3).
 *   pA      device pointer to the first element of the storage; 32-byte
 *           aligned.
 *   dA      device pointer to room for min(m, n) doubles that a
 *           factorization may fill with the inverse of the diagonal
 *           (Sec. 4.7.1), or NULL.
 *   m, n    rows and columns of the matrix.
 *   pm      storage rows: m rounded up to a multiple of ps.
 *   cn      storage columns, the panel length ("sda" in Sec. 4.3.3), >= n.
 *   ps      panel height; must equal BF_PS.
 *   memsize bytes of device memory addressed by the descriptor.
 * Element (i, j) of the matrix lies at
 *   pA[(i - i % ps) * cn + j * ps + i % ps]                      (Sec. 4.3.3)
 */
typedef struct bf_dmat {
  double *pA;
  double *dA;
  int m;
  int n;
  int pm;
  int cn;
  int ps;
  size_t memsize;
} bf_dmat;

/* ---- memory (Appendix A.1.2, externally provided memory) ----------------- */

/* Bytes of device memory that bf_create_dmat needs for an m x n matrix:
 * the panel-major storage (pm * cn doubles) followed by the inverse-diagonal
 * array (min(m, n) doubles), rounded up to a multiple of BF_ALIGN so that
 * consecutive matrices carved from one buffer stay aligned.  Returns 0 for
 * negative sizes. */
size_t bf_memsize_dmat(int m, int n);

/* Fills *sA for an m x n matrix over caller-owned device memory `mem` of at
 * least bf_memsize_dmat(m, n) bytes, aligned to BF_ALIGN.  Touches neither
 * the memory nor the device.  Returns 0, or -1/-2/-3/-4 for a bad m, n, sA or
 * mem (mem must be non-NULL and BF_ALIGN-aligned). */
int bf_create_dmat(int m, int n, bf_dmat *sA, void *mem);

/* Panel height the library was compiled with (BF_PS). */
int bf_panel_height(void);

/* ---- packing (Sec. 4.3.3; the packing routines of Appendix A.3) ---------- */

/* Packing converts between a column-major matrix (leading dimension lda:
 * element (i, j) at A[i + j*lda]) and a sub-matrix of a panel-major one
 * (Sec. 4.3.3 address formula above).  The column-major side may be
 *   - device (or managed) memory: a kernel copies;
 *   - host memory that is pinned or registered with the CUDA runtime (and so
 *     mapped into the device's address space): a kernel copies, reading or
 *     writing the host memory directly over the host link;
 *   - plain (pageable) host memory: one cudaMemcpy2DAsync per problem and
 *     group of ps rows (a panel's rows are ps consecutive doubles on both
 *     sides).  This path is slow for many small matrices; pin or register
 *     the buffer for speed.
 * The kind is found with cudaPointerGetAttributes; for a batched call it is
 * that of the first problem's matrix, and all problems must lie in one
 * allocation.  The panel-major side is device memory, as everywhere.
 * Host buffers must stay valid until the copy is done: the calls are
 * asynchronous on `stream`, except that a copy to pageable host memory
 * returns only once it is complete.  Nothing is allocated.
 * Elements of the destination outside the copied sub-matrix are not
 * written. */

/* Packs the m x n column-major matrix A (host or device, lda >= max(1, m))
 * into the sub-matrix (bi, bj) of the panel-major matrix sB. */
int bf_pack_dmat(int m, int n, const double *A, int lda, const bf_dmat *sB, int bi, int bj,
                 void *stream);

/* Unpacks the m x n sub-matrix (ai, aj) of sA into the column-major matrix
 * B (host or device, ldb >= max(1, m)). */
int bf_unpack_dmat(int m, int n, const bf_dmat *sA, int ai, int aj, double *B, int ldb,
                   void *stream);

/* Batched forms: problem b's column-major matrix is at A + b*strideA (B +
 * b*strideB for unpack; strides in doubles), its panel-major one at
 * sB->pA + b*strideB (sA->pA + b*strideA). */
int bf_pack_dmat_batched(int batch, int m, int n, const double *A, int lda, long long strideA,
                         const bf_dmat *sB, int bi, int bj, long long strideB, void *stream);

int bf_unpack_dmat_batched(int batch, int m, int n, const bf_dmat *sA, int ai, int aj,
                           long long strideA, double *B, int ldb, long long strideB, void *stream);

/* ---- level-3 BLAS ---------------------------------------------------------- */

/* gemm_nt (Appendix A.2.1; Sec. 5.2.2):
 *     D <- alpha * A * B^T + beta * C
 * A is m x k, B is n x k, C and D are m x n.  C and D may be the same
 * sub-matrix of the same storage; no other overlap is allowed.  beta == 0
 * means C is not read (it may hold NaN).  k == 0 gives D = beta * C.
 * Any size >= 0 is supported. */
int bf_dgemm_nt_batched(int batch, int m, int n, int k, double alpha,
                        const bf_dmat *sA, int ai, int aj, long long strideA,
                        const bf_dmat *sB, int bi, int bj, long long strideB, double beta,
                        const bf_dmat *sC, int ci, int cj, long long strideC,
                        const bf_dmat *sD, int di, int dj, long long strideD, void *stream);

int bf_dgemm_nt(int m, int n, int k, double alpha, const bf_dmat *sA, int ai, int aj,
                const bf_dmat *sB, int bi, int bj, double beta, const bf_dmat *sC, int ci, int cj,
                const bf_dmat *sD, int di, int dj, void *stream);

/* gemm_nn (Sec. 5.2.2 "gemm_nn"):
 *     D <- alpha * A * B + beta * C
 * A is m x k, B is k x n, C and D are m x n.  C and D may coincide; no other
 * overlap.  beta == 0 means C is not read. */
int bf_dgemm_nn_batched(int batch, int m, int n, int k, double alpha,
                        const bf_dmat *sA, int ai, int aj, long long strideA,
                        const bf_dmat *sB, int bi, int bj, long long strideB, double beta,
                        const bf_dmat *sC, int ci, int cj, long long strideC,
                        const bf_dmat *sD, int di, int dj, long long strideD, void *stream);

int bf_dgemm_nn(int m, int n, int k, double alpha, const bf_dmat *sA, int ai, int aj,
                const bf_dmat *sB, int bi, int bj, double beta, const bf_dmat *sC, int ci, int cj,
                const bf_dmat *sD, int di, int dj, void *stream);

/* trmm_rlnn (Sec. 5.2.2 "trmm_rlnn"; right, lower, not transposed,
 * non-unit):
 *     D <- alpha * B * L
 * L is the n x n lower triangle of sL at (li, lj) (its strictly upper part
 * does not affect the result); B and D are m x n and must not overlap. */
int bf_dtrmm_rlnn_batched(int batch, int m, int n, double alpha,
                          const bf_dmat *sL, int li, int lj, long long strideL,
                          const bf_dmat *sB, int bi, int bj, long long strideB,
                          const bf_dmat *sD, int di, int dj, long long strideD, void *stream);

int bf_dtrmm_rlnn(int m, int n, double alpha, const bf_dmat *sL, int li, int lj,
                  const bf_dmat *sB, int bi, int bj, const bf_dmat *sD, int di, int dj,
                  void *stream);

/* syrk_ln (Sec. 5.2.2):
 *     lower(D) <- alpha * A * B^T + beta * C
 * A and B are m x k and may be different matrices (or the same); C and D are
 * m x m.  Only the lower triangle of D, diagonal included, is computed and
 * written; the strictly upper part of D is left untouched.  C and D may
 * coincide.  beta == 0 means C is not read. */
int bf_dsyrk_ln_batched(int batch, int m, int k, double alpha,
                        const bf_dmat *sA, int ai, int aj, long long strideA,
                        const bf_dmat *sB, int bi, int bj, long long strideB, double beta,
                        const bf_dmat *sC, int ci, int cj, long long strideC,
                        const bf_dmat *sD, int di, int dj, long long strideD, void *stream);

int bf_dsyrk_ln(int m, int k, double alpha, const bf_dmat *sA, int ai, int aj,
                const bf_dmat *sB, int bi, int bj, double beta, const bf_dmat *sC, int ci, int cj,
                const bf_dmat *sD, int di, int dj, void *stream);

/* trsm_rltn (Sec. 5.2.2; right, lower, transposed, non-unit):
 *     D <- alpha * B * L^{-T},  i.e. D = X with X * L^T = alpha * B
 * L is the n x n lower triangle of sL at (li, lj) (its strictly upper part
 * is not read); B and D are m x n and may coincide.  If dinv is not NULL it
 * holds, for problem b, the n values 1/L[j][j] at dinv + b*strideDinv (as
 * written by bf_dpotrf_l_batched) and the solve uses them instead of
 * dividing (Sec. 4.7.1); without dinv the library forms the reciprocals
 * from the hardware approximation, which treats a subnormal L[j][j] as zero:
 * columns >= j of X are then NaN.  Supports n <= 4096; any m. */
int bf_dtrsm_rltn_batched(int batch, int m, int n, double alpha,
                          const bf_dmat *sL, int li, int lj, long long strideL,
                          const double *dinv, long long strideDinv,
                          const bf_dmat *sB, int bi, int bj, long long strideB,
                          const bf_dmat *sD, int di, int dj, long long strideD, void *stream);

int bf_dtrsm_rltn(int m, int n, double alpha, const bf_dmat *sL, int li, int lj,
                  const bf_dmat *sB, int bi, int bj, const bf_dmat *sD, int di, int dj,
                  void *stream);

/* ---- LAPACK-like --------------------------------------------------------- */

/* potrf_l (Sec. 5.2.2; Sec. 4.6):
 *     lower(D) <- L,  L * L^T = C,  L lower triangular with positive diagonal
 * C is m x m; only its lower triangle is read.  C and D may coincide.  The
 * strictly upper part of D is left untouched.
 * dinv (device, may be NULL): receives 1/L[j][j] for j < m at
 *   dinv + b*strideDinv (Sec. 4.7.1).
 * info (device, may be NULL): info[b] = 0 if problem b factorized, else the
 *   1-based column j+1 of the first pivot that was not > 0 (NaN included);
 *   columns >= j of that problem's D are then unspecified.  Other problems
 *   are unaffected.
 * Supports m <= 512. */
int bf_dpotrf_l_batched(int batch, int m, const bf_dmat *sC, int ci, int cj, long long strideC,
                        const bf_dmat *sD, int di, int dj, long long strideD,
                        double *dinv, long long strideDinv, int *info, void *stream);

int bf_dpotrf_l(int m, const bf_dmat *sC, int ci, int cj, const bf_dmat *sD, int di, int dj,
                int *info, void *stream);

/* getrf (Sec. 5.2.2 "getrf"; LU with partial pivoting, Appendix A.3):
 *     P A = L U  for the n x n matrix C, stored in D (L unit lower, its
 *     diagonal not stored; U upper).
 * Column by column, the pivot is the first row at or below the diagonal with
 * the largest |a(i, j)|; ipiv[b*strideIpiv + j] (device, 0-based) receives
 * it, and row j was swapped with it over the whole matrix.  info (device, may
 * be NULL): 0, or j+1 for the first exactly zero pivot (that column is then
 * neither scaled nor used to update).  C and D coincide or do not overlap.
 * Supports n <= 512.  Above n = 128 the factorization is blocked by columns
 * of 32 (the right-looking blocked form of the same algorithm: each panel
 * factorized column by column with the same pivot rule, its row swaps then
 * applied to the other columns, U12 = L11^{-1} A12, A22 -= L21 U12), so the
 * results agree with the unblocked order up to rounding; where a zero pivot
 * column meets non-finite entries the blocked update can turn 0 * inf into
 * NaN where the unblocked form skips the update. */
int bf_dgetrf_batched(int batch, int n, const bf_dmat *sC, int ci, int cj, long long strideC,
                      const bf_dmat *sD, int di, int dj, long long strideD, int *ipiv,
                      long long strideIpiv, int *info, void *stream);

int bf_dgetrf(int n, const bf_dmat *sC, int ci, int cj, const bf_dmat *sD, int di, int dj,
              int *ipiv, int *info, void *stream);

/* gelqf (Sec. 5.2.2 "gelqf"; LQ factorization, Appendix A.3):
 *     A = L Q  for the m x n matrix C, stored in D.
 * Householder reflectors H_i = I - tau_i v_i v_i^T, v_i = [1, x_i], applied
 * from the right row by row (i < min(m, n)); beta = -sign(alpha) ||(alpha,
 * x)||.  L is the lower triangle of D, x_i is left in the strictly upper
 * part of row i, tau (device) receives tau_i at tau + b*strideTau + i, and
 * Q = H_{k-1} ... H_0.  C and D coincide or do not overlap.  Supports
 * m * n <= 16384, and any m, n <= 512: there the factorization is blocked by
 * rows of 32 -- each panel by the steps above, then its reflectors applied to
 * the rows below at once as the block reflector I - V^T T V (compact WY form,
 * T upper triangular), so the results agree with the row-by-row order up to
 * rounding.  The reflector's scalars come from a reciprocal square root and
 * a reciprocal (rcp.approx and one third-order correction): a row whose
 * |alpha| + ||(alpha, x)|| is subnormal yields NaN. */
int bf_dgelqf_batched(int batch, int m, int n, const bf_dmat *sC, int ci, int cj, long long strideC,
                      const bf_dmat *sD, int di, int dj, long long strideD, double *tau,
                      long long strideTau, void *stream);

int bf_dgelqf(int m, int n, const bf_dmat *sC, int ci, int cj, const bf_dmat *sD, int di, int dj,
              double *tau, void *stream);

/* syrk_potrf_ln (Sec. 4.7.2 "concatenating updates/downdates"; Sec. 5.3;
 * routine list in Appendix A.3):
 *     lower(D) <- chol(C + A * B^T)
 * A and B are m x k (may coincide), C and D are m x m (may coincide).  The
 * sum is formed inside the factorization kernel and never stored.  dinv and
 * info as for bf_dpotrf_l_batched.  Supports m <= 512. */
int bf_dsyrk_dpotrf_ln_batched(int batch, int m, int k,
                               const bf_dmat *sA, int ai, int aj, long long strideA,
                               const bf_dmat *sB, int bi, int bj, long long strideB,
                               const bf_dmat *sC, int ci, int cj, long long strideC,
                               const bf_dmat *sD, int di, int dj, long long strideD,
                               double *dinv, long long strideDinv, int *info, void *stream);

int bf_dsyrk_dpotrf_ln(int m, int k, const bf_dmat *sA, int ai, int aj,
                       const bf_dmat *sB, int bi, int bj, const bf_dmat *sC, int ci, int cj,
                       const bf_dmat *sD, int di, int dj, int *info, void *stream);

/* ---- solves with the Cholesky factor -------------------------------------- */

/* potrs: solves A X = B for X, given the lower Cholesky factor L of A
 * (L L^T = A, as computed by bf_dpotrf_l_batched):  X = L^{-T} L^{-1} B.
 * The two triangular solves are the right-hand-side forms of trsm (trsv_lnn
 * and trsv_ltn of the paper's BLAS level-2 list, Appendix A.3).
 * L is the n x n lower triangle of sL at (li, lj); B and X are n x nrhs and
 * may coincide.  Supports n <= 216 and 1 <= nrhs <= 8 (the factor and the
 * right-hand sides of a system held in one CTA's shared memory). */
int bf_dpotrs_l_batched(int batch, int n, int nrhs, const bf_dmat *sL, int li, int lj,
                        long long strideL, const bf_dmat *sB, int bi, int bj, long long strideB,
                        const bf_dmat *sX, int xi, int xj, long long strideX, void *stream);

/* Adjoint (reverse-mode derivative) of the factor-and-solve X = A^{-1} B
 * (not in the paper): given the lower factor L of A (L L^T = A), the
 * solution X and the cotangent Xbar = d loss / d X (all n x nrhs),
 *     Bbar = A^{-1} Xbar                  (d loss / d B)
 *     Abar = -(Bbar X^T + X Bbar^T) / 2   (d loss / d A for symmetric A)
 * Bbar is n x nrhs, Abar n x n (written in full).  Outputs must not overlap
 * the inputs.  Supports n <= 208 and 1 <= nrhs <= 8. */
int bf_dposv_adjoint_batched(int batch, int n, int nrhs, const bf_dmat *sL, int li, int lj,
                             long long strideL, const bf_dmat *sX, int xi, int xj, long long strideX,
                             const bf_dmat *sXbar, int xbi, int xbj, long long strideXbar,
                             const bf_dmat *sBbar, int bbi, int bbj, long long strideBbar,
                             const bf_dmat *sAbar, int abi, int abj, long long strideAbar,
                             void *stream);

/* Bytes of device workspace bf_dposv_mixed_batched needs for `batch`
 * systems of order n (the single-precision factors and their status). */
size_t bf_dposv_mixed_worksize(int batch, int n);

/* Mixed-precision SPD solve with FP64 iterative refinement (not in the
 * paper, which has separate single- and double-precision routines,
 * Appendix A.3): the lower Cholesky factor of fl32(A) is computed in FP32
 * into `work`, then x = 0, r = b and, up to max_iter times,
 *     d = (L32 L32^T)^{-1} r (FP32),  x += d,  r = b - A x (FP64),
 * stopping once ||R||_F / (||A||_F ||X||_F) <= tol over the nrhs columns.
 * A is n x n SPD (only its lower triangle is read); B and X are n x nrhs
 * (they must not coincide).
 * iters (device, may be NULL): per system, the number of corrections taken
 *   when the tolerance was met; -1 if it was not met within max_iter (X
 *   holds the last iterate); -2 if the FP32 factorization failed (X not
 *   written).  Callers fall back to potrf + potrs for those systems.
 * resid (device, may be NULL): the final relative residual per system.
 * work: device memory of at least bf_dposv_mixed_worksize(batch, n) bytes,
 *   256-byte aligned, owned by the caller; its contents are scratch.
 * Supports n <= 256 and 1 <= nrhs <= 8. */
int bf_dposv_mixed_batched(int batch, int n, int nrhs, const bf_dmat *sA, int ai, int aj,
                           long long strideA, const bf_dmat *sB, int bi, int bj, long long strideB,
                           const bf_dmat *sX, int xi, int xj, long long strideX, double tol,
                           int max_iter, int *iters, double *resid, void *work, size_t work_bytes,
                           void *stream);

/* Bytes of device workspace bf_dposv_mixed_tc_batched needs. */
size_t bf_dposv_mixed_tc_worksize(int batch, int n);

/* Mixed-precision SPD solve whose factorization is blocked (not in the
 * paper, which has separate single- and double-precision routines, Appendix
 * A.3): for each block column of 32, the diagonal block is factored (potrf)
 * and the panel below it solved (trsm) in FP64, and the trailing matrix is
 * updated on the tensor cores in precision `prec`:
 *     0  BF16 operands, FP32 accumulation
 *     1  TF32 operands, FP32 accumulation
 *     2  3xTF32: operands split as H + R (both TF32), H H^T + H R^T + R H^T
 * (see bf_dsyrk_ln_tc_batched).  The factor, rounded to FP32, then drives the
 * FP64 iterative refinement of bf_dposv_mixed_batched, with its tolerance,
 * iteration limit and outcome codes (iters -1: not converged within
 * max_iter; -2: a pivot of the blocked factorization failed).  The lower
 * precisions converge only while cond(A) times their unit roundoff stays
 * well below one; the others report -1.
 * Arguments 1..19 as for bf_dposv_mixed_batched; work: device memory of at
 * least bf_dposv_mixed_tc_worksize(batch, n) bytes, 256-byte aligned, owned
 * by the caller.  Supports n <= 160 (its first trailing update, n - 32 rows,
 * is one 128-row tensor-core tile) and 1 <= nrhs <= 8. */
int bf_dposv_mixed_tc_batched(int batch, int n, int nrhs, const bf_dmat *sA, int ai, int aj,
                              long long strideA, const bf_dmat *sB, int bi, int bj, long long strideB,
                              const bf_dmat *sX, int xi, int xj, long long strideX, double tol,
                              int max_iter, int *iters, double *resid, int prec, void *work,
                              size_t work_bytes, void *stream);

/* syrk_ln in reduced precision on the tensor cores, the trailing update of
 * the blocked mixed-precision factorization (not in the paper, whose
 * routines come in separate single- and double-precision versions, Appendix
 * A.3):
 *     lower(D) <- C - A * A^T
 * A is m x k, C and D are m x m, all FP64; only the lower triangle of D is
 * written.  The product A A^T is formed by tcgen05 MMAs with FP32
 * accumulation from A rounded to `prec` (0 BF16, 1 TF32, 2 3xTF32 as above);
 * the subtraction is FP64.  Supports m <= 128 and 1 <= k <= 32.  A's rows
 * must start on a panel top (ai % BF_PS == 0), its storage be 16-byte
 * aligned and strideA even, else -5 (its runs of 4 rows are copied by the
 * bulk-copy engine).  C and D may coincide; A must not overlap D. */
int bf_dsyrk_ln_tc_batched(int batch, int m, int k, int prec, const bf_dmat *sA, int ai, int aj,
                           long long strideA, const bf_dmat *sC, int ci, int cj, long long strideC,
                           const bf_dmat *sD, int di, int dj, long long strideD, void *stream);

/* ---- backward Riccati recursion (Sec. 5.3) -------------------------------- */

/* One MPC instance of bf_driccati_sqrt_batched, in device memory.  All
 * matrices are panel-major (BF_PS rows per panel) with the given panel
 * lengths (cn >= the matrix's column count):
 *   BAt  (nu+nx) x nx: the stacked [B^T; A^T] of x+ = A x + B u
 *   M0   (nu+nx) x (nu+nx): [[R, S^T], [S, Q]]; only its lower triangle is read
 *   LN   nx x nx: lower Cholesky factor of the terminal cost P_N
 *   L    outputs: N lower factors nx x nx, stage k at L + k*l_stride
 *        (doubles); L_k L_k^T = P_k.  Only the lower triangles are written.
 *   Kt   outputs: N gains transposed, nx x nu, stage k at Kt + k*kt_stride;
 *        K_k = Kt_k^T is the feedback u = K_k x.
 *   info outputs (may be NULL): N ints; 0, or 1 + the column of the first
 *        non-positive pivot of stage k's factorization, or -1 if the
 *        instance's sizes exceed the call's max_nx / max_nu. */
typedef struct bf_riccati_prob {
  int nx, nu;
  const double *BAt;
  int bat_cn;
  const double *M0;
  int m0_cn;
  const double *LN;
  int ln_cn;
  double *L;
  int l_cn;
  long long l_stride;
  double *Kt;
  int kt_cn;
  long long kt_stride;
  int *info;
} bf_riccati_prob;

/* Backward Riccati recursion in the square-root form of Sec. 5.3, for
 * `batch` independent instances of possibly different sizes.  For each
 * instance and k = N-1, ..., 0, from Lc = L_{k+1} (L_N = LN):
 *     C = [B^T; A^T] Lc                                   (trmm_rlnn)
 *     [[Lam, 0], [Lo, L_k]] = chol(M0 + C C^T)            (syrk_potrf_ln)
 *     Kt_k Lam = -Lo                                      (trsm_rlnn)
 * probs: device array of the instances; order (device, may be NULL): the
 * instances to process, as indices into probs (batch of them), best sorted
 * by decreasing size so that the GPU starts the longest ones first;
 * max_nx, max_nu: bounds on the sizes of those instances (they size the
 * shared memory; instances beyond them are reported in info and skipped);
 * threads: CTA width (a multiple of 32, 32..512) or 0 for 256.
 * Returns BF_ERR_UNSUPPORTED if max_nx, max_nu need more than 200 KB of
 * shared memory (e.g. beyond nx = 64, nu = 64). */
int bf_driccati_sqrt_batched(int batch, int N, const bf_riccati_prob *probs, const int *order,
                             int max_nx, int max_nu, int threads, void *stream);

/* The mixed-precision solver above, for callers that cannot allocate
 * device memory.  The paper has no counterpart.
 *
 * Who needs it: a caller that has no way to hand over a workspace.  A
 * controller running a fixed-period loop may forbid allocation there,
 * because cudaMalloc can block the device and can fail at run time.  A
 * plugin may run inside a host application that owns all device memory.
 *
 * Same arguments, checks, results and error codes as
 * bf_dposv_mixed_batched, minus work / work_bytes.  Argument errors are
 * reported first; only a valid call that does not fit gets BF_ERR_TOO_LARGE.  The scratch is a fixed
 * array of BF_NOALLOC_WORK_BYTES (16 MiB) inside this library's device
 * memory; every GPU that loads the library holds it until the process exits.
 *   - Problems need bf_dposv_mixed_worksize(batch, n) <= BF_NOALLOC_WORK_BYTES
 *     (for n = 128, up to 255 systems).  Larger calls return
 *     BF_ERR_TOO_LARGE and launch nothing.
 *   - The first call on a device looks up the array's address
 *     (cudaGetSymbolAddress) with that device current.  Make that first call
 *     before any stream capture on the device.  The address is kept for the
 *     life of the process: no cudaDeviceReset (or other reset of the
 *     device's primary context) may come between calls.
 *   - All calls share the array, and it keeps the last call's contents.
 *     Nothing in it needs to start at zero.  Calls whose kernels overlap on
 *     the GPU race on it; serialize them (one stream, one thread at a time).
 *   - Nothing is allocated or freed. */
int bf_dposv_mixed_batched_noalloc(int batch, int n, int nrhs, const bf_dmat *sA, int ai, int aj,
                                   long long strideA, const bf_dmat *sB, int bi, int bj,
                                   long long strideB, const bf_dmat *sX, int xi, int xj,
                                   long long strideX, double tol, int max_iter, int *iters,
                                   double *resid, void *stream);

/* ---------------------------------------------------------------------------
 * Kernel layouts (the hook of the autotuner).
 *
 * The paper's library is built in size-specialized variants for each target
 * (Sec. 5.1: HP2, HP2F).  Here each routine has several kernel layouts
 * (problems per CTA, lanes per problem, a split k-loop), and a built-in rule
 * picks one from the order and the batch size.  A caller that has timed the
 * candidates -- the package's autotuner -- can force one per (routine, order,
 * batch size class).  The results do not depend on the layout beyond
 * rounding (summation order), except where a layout has no kernel for the
 * order, which bf_layout_set refuses.
 *
 * routine:  0 gemm_nt, 1 syrk_ln, 2 potrf_l, 3 trsm_rltn, 4 syrk_potrf_ln,
 *           5 getrf, 6 gelqf.
 * order:    m for gemm_nt, syrk_ln, potrf_l and syrk_potrf_ln; n (the order
 *           of L) for trsm_rltn; n for getrf; the column count n for gelqf
 *           (a forced gelqf layout that has no kernel for the call's m x n
 *           leaves that call to the rule).  Orders above 511 share one
 *           entry.
 * batch:    the entry covers the batch sizes with the same floor(log2(batch)).
 * layout:   0 = the built-in rule; 1 .. bf_layout_count(routine) - 1:
 *   gemm_nt, syrk_ln:   1, 2, 3 = the k-loop of a 4x4 block on 1, 2, 4 lanes
 *   potrf_l, syrk_potrf_ln:
 *                       1 one lane per problem, in registers (order <= 8)
 *                       2..6 a warp shared by 16, 8, 4, 2, 1 problems, the
 *                         triangles in shared memory (order <= 31)
 *                       7 one thread per row, 1, 2 or 4 problems per CTA
 *                       8 one problem per CTA of four warps (order <= 32)
 *                       9 syrk_potrf_ln only: the sum by the syrk kernel
 *                         into D, then layout 7 on D (order >= 48)
 *                       10 blocked: two diagonal blocks, potrf, trsm,
 *                         syrk, potrf (order >= 32)
 *                       11 one thread per row, eight problems per CTA,
 *                         blocks of 4 columns (order <= 64)
 *   trsm_rltn:          1 one thread per row of X
 *                       2, 3, 4 = 2, 4, 8 lanes per row (order <= 32)
 *   getrf:              1 a warp shared by 32 / G problems (order <= 128)
 *                       2 one CTA per problem, the matrix in shared
 *                         memory (order <= 128)
 *                       3, 4 blocked by columns of 32, 16: panel, swaps
 *                         and triangular solve, gemm_nn update (order <= 512)
 *   gelqf:              1, 2 as for getrf (m * n <= 16384)
 *                       3, 4 blocked by rows of 32, 16: panel, block
 *                         reflector applied to the rows below (m, n <= 512)
 * The table is process-wide (all devices) and not synchronized with calls in
 * flight: set it before the calls it should affect.
 * ------------------------------------------------------------------------ */

/* Number of layouts of `routine` (entry 0, the rule, included); 0 for an
 * unknown routine. */
int bf_layout_count(int routine);

/* Forces `layout` for (routine, order, batch class); layout 0 restores the
 * rule.  Returns 0, -1..-4 for a bad argument, or BF_ERR_UNSUPPORTED if the
 * layout has no kernel for that order. */
int bf_layout_set(int routine, int order, int batch, int layout);

/* The layout a call of `routine` with these sizes would use now (the forced
 * one, else the rule's): gemm_nt (m, n, k), syrk_ln (m, -, k), potrf_l (m),
 * trsm_rltn (m, n), syrk_potrf_ln (m, -, k), getrf (n), gelqf (m, n);
 * unused sizes are ignored.
 * Returns the layout (>= 1) or -1..-5 for a bad argument. */
int bf_layout_get(int routine, int batch, int m, int n, int k);

/* Restores the built-in rule everywhere. */
void bf_layout_reset(void);

/* ---------------------------------------------------------------------------
 * Descriptor-array batched forms: uneven sizes in one launch.
 *
 * The strided forms need every problem of a call to share sizes and layout.
 * These take, for problem b, its sizes size[b] and, for every operand, a
 * descriptor with the sub-matrix offsets that the paper's routines take
 * next to it (Sec. 3.2 and Appendix A.2: "(sA, ai, aj)"), all in DEVICE
 * arrays of length batch.  The calls are the paper's per-matrix routines
 * with one launch for the whole array.  max_m (and max_n) bound the sizes
 * and shape the launch.
 *
 * Arguments of the call itself are checked on the host (-i for argument i).
 * Each problem's record is checked on the device, with the same rules as the
 * strided forms.  A problem that fails is skipped (its output is untouched).
 * status[b] (device, may be NULL) receives 0, or -1 for bad sizes (negative,
 * or above max_m / max_n), or -(1 + p) for the p-th operand of the call
 * (counting from 1 in the order of the signature).  Calls are asynchronous.
 * ------------------------------------------------------------------------ */
typedef struct {
  bf_dmat mat; /* descriptor of the matrix */
  int i, j;    /* sub-matrix offsets (row, column) */
} bf_dsub;

typedef struct {
  int m, n, k; /* sizes of one problem; unused members are ignored */
} bf_dsize;

/* Host-side check of one operand record with the rules the kernels apply to
 * it on the device: a valid descriptor (non-NULL 8-byte-aligned pA, ps ==
 * BF_PS, 0 <= m <= pm, pm a multiple of ps, cn >= n) and a rows x cols
 * sub-matrix at (i, j) inside it (bounds compared in 64-bit arithmetic).
 * Returns 1 if the record is valid, 0 if not (or if rec is NULL).  Touches
 * neither the matrix nor the device. */
int bf_dsub_valid(const bf_dsub *rec, int rows, int cols);

/* gemm_nt per problem: D <- alpha A B^T + beta C with sizes (m, n, k); C is
 * not read (nor checked) when beta == 0.  Operands: A, B, C, D. */
int bf_dgemm_nt_vbatched(int batch, const bf_dsize *size, double alpha, const bf_dsub *A,
                         const bf_dsub *B, double beta, const bf_dsub *C, const bf_dsub *D,
                         int max_m, int max_n, int *status, void *stream);

/* syrk_ln per problem: sizes (m, -, k).  Operands: A, B, C, D. */
int bf_dsyrk_ln_vbatched(int batch, const bf_dsize *size, double alpha, const bf_dsub *A,
                         const bf_dsub *B, double beta, const bf_dsub *C, const bf_dsub *D,
                         int max_m, int *status, void *stream);

/* potrf_l per problem: size (m); m <= 512.  With want_dinv, 1/L_jj goes to
 * D[b].mat.dA[D[b].j + j] when that descriptor has an inverse-diagonal
 * array that reaches that far (D[b].j + m <= min(mat.m, mat.n)); otherwise
 * it is not written.  info[b] (device, may be NULL) as for the strided
 * form.  Operands: C, D. */
int bf_dpotrf_l_vbatched(int batch, const bf_dsize *size, const bf_dsub *C, const bf_dsub *D,
                         int want_dinv, int *info, int max_m, int *status, void *stream);

/* trsm_rltn per problem: sizes (m, n); n <= 4096.  With use_dinv the
 * reciprocals come from L[b].mat.dA[L[b].j + j] where that array reaches
 * (L[b].j + n <= min(mat.m, mat.n)); else they are formed from L.
 * Operands: L, B, D. */
int bf_dtrsm_rltn_vbatched(int batch, const bf_dsize *size, double alpha, const bf_dsub *L,
                           int use_dinv, const bf_dsub *B, const bf_dsub *D, int max_m, int max_n,
                           int *status, void *stream);

/* syrk_potrf_ln per problem: sizes (m, -, k); m <= 512.  Operands: A, B, C, D. */
int bf_dsyrk_dpotrf_ln_vbatched(int batch, const bf_dsize *size, const bf_dsub *A, const bf_dsub *B,
                                const bf_dsub *C, const bf_dsub *D, int want_dinv, int *info,
                                int max_m, int *status, void *stream);

/* Order of the records by decreasing size, for the *_vbatched_ordered calls
 * below: order (device, batch ints, 4-byte aligned) receives a permutation
 * of 0..batch-1 with size[order[q]].m non-increasing in q (records of equal
 * m in any order); records whose m is negative or above max_m come first.
 * One CTA (a counting sort over max_m + 2 keys in shared memory), no
 * workspace; its time grows with batch / 1024.  max_m <= 512. */
int bf_vbatched_order(int batch, const bf_dsize *size, int max_m, int *order, void *stream);

/* potrf_l and syrk_potrf_ln per problem, as bf_dpotrf_l_vbatched and
 * bf_dsyrk_dpotrf_ln_vbatched (same records, checks, status codes, info and
 * inverse diagonal), with the records taken in the order given by `order`
 * (device, a permutation of 0..batch-1, e.g. from bf_vbatched_order; NULL:
 * the records in their own order, which should then be sorted by size).
 * Consecutive records share a CTA: four problems per CTA when max_m <= 64
 * (or <= 128 from 24 problems per SM), else two for the orders up to 256
 * (one launch), and one per CTA above 256 (a second launch); below 12
 * problems per SM, one problem per CTA in the given order.  Sorting matters: problems of very different orders in one
 * CTA idle the smaller ones' lanes.  Entries of order outside 0..batch-1 are skipped; an order
 * that repeats a record computes it twice, concurrently (undefined).
 * Argument errors: -1 batch, -2 size, -3 order (misaligned), then the
 * remaining arguments in signature order (-4 ..). */
int bf_dpotrf_l_vbatched_ordered(int batch, const bf_dsize *size, const int *order, const bf_dsub *C,
                                 const bf_dsub *D, int want_dinv, int *info, int max_m, int *status,
                                 void *stream);

int bf_dsyrk_dpotrf_ln_vbatched_ordered(int batch, const bf_dsize *size, const int *order, const bf_dsub *A,
                                        const bf_dsub *B, const bf_dsub *C, const bf_dsub *D, int want_dinv,
                                        int *info, int max_m, int *status, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* BFGPU_H */
