// The C ABI of include/bfgpu.h: argument checking (the argument checks the
// paper mentions for its wrapper implementation, Sec. 3.1) and dispatch to
// the kernels.  Nothing here allocates memory or synchronizes.
#include <cstdint>
#include <initializer_list>

#include "bf_internal.cuh"

using namespace bf;

namespace {

inline bool aligned_to(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

// Checks one matrix operand of a batched call.  Returns 0 if valid, else
// 1 (descriptor), 2 (row offset), 3 (column offset) or 4 (stride).
int check_op(const bf_dmat *s, int ri, int cj, int rows, int cols, long long stride, int batch,
             bool output) {
  if (!s || s->ps != PS || !s->pA || !aligned_to(s->pA, 8) || s->m < 0 || s->n < 0 ||
      s->pm < s->m || s->pm % PS != 0 || s->cn < s->n)
    return 1;
  // 64-bit sums: an offset near INT_MAX must fail here, not wrap round
  if (ri < 0 || (long long)ri + rows > (long long)s->m) return 2;
  if (cj < 0 || (long long)cj + cols > (long long)s->n) return 3;
  if (stride < 0) return 4;
  if (output && batch > 1 && stride < (long long)s->pm * s->cn) return 4;
  return 0;
}

inline int pos_err(int which, int desc_pos) { return -(desc_pos + which - 1); }

Op make_op(const bf_dmat *s, int ri, int cj, long long stride) {
  Op o;
  o.p = s ? s->pA : nullptr;
  o.stride = stride;
  o.cn = s ? s->cn : 0;
  o.i0 = ri;
  o.j0 = cj;
  return o;
}

OpW make_opw(const bf_dmat *s, int ri, int cj, long long stride) {
  OpW o;
  o.p = s->pA;
  o.stride = stride;
  o.cn = s->cn;
  o.i0 = ri;
  o.j0 = cj;
  return o;
}

// The vector-load fast path needs every operand's rows to start on a panel
// top and every problem to start 16-byte aligned.
bool fast_path(std::initializer_list<const Op *> ops) {
  for (const Op *o : ops) {
    if (!o->p) continue;
    if ((o->i0 % PS) != 0 || (o->stride % 2) != 0 || !aligned_to(o->p, 16)) return false;
  }
  return true;
}

inline int status(cudaError_t e) { return e == cudaSuccess ? 0 : (int)e; }

}  // namespace

extern "C" {

size_t bf_memsize_dmat(int m, int n) {
  if (m < 0 || n < 0) return 0;
  const size_t pm = ((size_t)m + PS - 1) / PS * PS;
  const size_t cn = (size_t)n;
  const size_t nd = (size_t)(m < n ? m : n);
  const size_t bytes = (pm * cn + nd) * sizeof(double);
  return (bytes + BF_ALIGN - 1) / BF_ALIGN * BF_ALIGN;
}

int bf_create_dmat(int m, int n, bf_dmat *sA, void *mem) {
  if (m < 0) return -1;
  if (n < 0) return -2;
  if (!sA) return -3;
  if (!mem || !aligned_to(mem, BF_ALIGN)) return -4;
  const int pm = (m + PS - 1) / PS * PS;
  sA->pA = (double *)mem;
  sA->dA = (m < n ? m : n) > 0 ? (double *)mem + (size_t)pm * n : nullptr;
  sA->m = m;
  sA->n = n;
  sA->pm = pm;
  sA->cn = n;
  sA->ps = PS;
  sA->memsize = bf_memsize_dmat(m, n);
  return 0;
}

int bf_panel_height(void) { return PS; }

int bf_pack_dmat_batched(int batch, int m, int n, const double *A, int lda, long long strideA,
                         const bf_dmat *sB, int bi, int bj, long long strideB, void *stream) {
  if (batch < 0) return -1;
  if (m < 0) return -2;
  if (n < 0) return -3;
  if (batch == 0 || m == 0 || n == 0) return 0;
  if (!A || !aligned_to(A, 8)) return -4;
  if (lda < m) return -5;
  if (strideA < 0) return -6;
  if (int w = check_op(sB, bi, bj, m, n, strideB, batch, true)) return pos_err(w, 7);
  return status(launch_pack(batch, m, n, A, lda, strideA, make_opw(sB, bi, bj, strideB),
                            (cudaStream_t)stream));
}

int bf_unpack_dmat_batched(int batch, int m, int n, const bf_dmat *sA, int ai, int aj,
                           long long strideA, double *B, int ldb, long long strideB, void *stream) {
  if (batch < 0) return -1;
  if (m < 0) return -2;
  if (n < 0) return -3;
  if (batch == 0 || m == 0 || n == 0) return 0;
  if (int w = check_op(sA, ai, aj, m, n, strideA, batch, false)) return pos_err(w, 4);
  if (!B || !aligned_to(B, 8)) return -8;
  if (ldb < m) return -9;
  if (strideB < 0 || (batch > 1 && strideB < (long long)ldb * n)) return -10;
  return status(launch_unpack(batch, m, n, make_op(sA, ai, aj, strideA), B, ldb, strideB,
                              (cudaStream_t)stream));
}

int bf_pack_dmat(int m, int n, const double *A, int lda, const bf_dmat *sB, int bi, int bj, void *stream) {
  const int r = bf_pack_dmat_batched(1, m, n, A, lda, 0, sB, bi, bj, 0, stream);
  if (r >= 0) return r;
  static const int map[11] = {0, 0, 1, 2, 3, 4, 0, 5, 6, 7, 0};
  return -map[-r];
}

int bf_unpack_dmat(int m, int n, const bf_dmat *sA, int ai, int aj, double *B, int ldb, void *stream) {
  const int r = bf_unpack_dmat_batched(1, m, n, sA, ai, aj, 0, B, ldb, 0, stream);
  if (r >= 0) return r;
  static const int map[11] = {0, 0, 1, 2, 3, 4, 5, 0, 6, 7, 0};
  return -map[-r];
}

// ---------------------------------------------------------------- gemm / syrk

static int gemm_like(bool syrk, int batch, int m, int n, int k, double alpha, const bf_dmat *sA,
                     int ai, int aj, long long strideA, const bf_dmat *sB, int bi, int bj,
                     long long strideB, double beta, const bf_dmat *sC, int ci, int cj,
                     long long strideC, const bf_dmat *sD, int di, int dj, long long strideD,
                     void *stream) {
  // argument positions differ by one between gemm (m, n, k) and syrk (m, k)
  const int sh = syrk ? -1 : 0;
  if (batch < 0) return -1;
  if (m < 0) return -2;
  if (n < 0) return -3;
  if (k < 0) return -(4 + sh);
  if (batch == 0 || m == 0 || n == 0) return 0;
  if (k > 0) {
    if (int w = check_op(sA, ai, aj, m, k, strideA, batch, false)) return pos_err(w, 6 + sh);
    if (int w = check_op(sB, bi, bj, n, k, strideB, batch, false)) return pos_err(w, 10 + sh);
  }
  if (beta != 0.0)
    if (int w = check_op(sC, ci, cj, m, n, strideC, batch, false)) return pos_err(w, 15 + sh);
  if (int w = check_op(sD, di, dj, m, n, strideD, batch, true)) return pos_err(w, 19 + sh);
  const Op A = make_op(k > 0 ? sA : nullptr, ai, aj, strideA);
  const Op B = make_op(k > 0 ? sB : nullptr, bi, bj, strideB);
  const Op C = make_op(beta != 0.0 ? sC : nullptr, ci, cj, strideC);
  const OpW D = make_opw(sD, di, dj, strideD);
  const Op Dr = make_op(sD, di, dj, strideD);
  const bool fast = fast_path({&A, &B, &C, &Dr});
  return status(launch_gemm_nt(syrk, batch, m, n, k, alpha, A, B, beta, C, D, fast,
                               (cudaStream_t)stream));
}

int bf_dgemm_nt_batched(int batch, int m, int n, int k, double alpha, const bf_dmat *sA, int ai,
                        int aj, long long strideA, const bf_dmat *sB, int bi, int bj,
                        long long strideB, double beta, const bf_dmat *sC, int ci, int cj,
                        long long strideC, const bf_dmat *sD, int di, int dj, long long strideD,
                        void *stream) {
  return gemm_like(false, batch, m, n, k, alpha, sA, ai, aj, strideA, sB, bi, bj, strideB, beta,
                   sC, ci, cj, strideC, sD, di, dj, strideD, stream);
}

int bf_dgemm_nt(int m, int n, int k, double alpha, const bf_dmat *sA, int ai, int aj,
                const bf_dmat *sB, int bi, int bj, double beta, const bf_dmat *sC, int ci, int cj,
                const bf_dmat *sD, int di, int dj, void *stream) {
  const int r = bf_dgemm_nt_batched(1, m, n, k, alpha, sA, ai, aj, 0, sB, bi, bj, 0, beta, sC,
                                    ci, cj, 0, sD, di, dj, 0, stream);
  // map batched argument positions back to this signature
  if (r >= 0) return r;
  static const int map[24] = {0, 0, 1, 2, 3, 4, 5, 6, 7, 0, 8, 9, 10, 0, 11, 12, 13, 14, 0, 15, 16, 17, 0, 18};
  return -map[-r];
}

int bf_dgemm_nn_batched(int batch, int m, int n, int k, double alpha, const bf_dmat *sA, int ai,
                        int aj, long long strideA, const bf_dmat *sB, int bi, int bj,
                        long long strideB, double beta, const bf_dmat *sC, int ci, int cj,
                        long long strideC, const bf_dmat *sD, int di, int dj, long long strideD,
                        void *stream) {
  if (batch < 0) return -1;
  if (m < 0) return -2;
  if (n < 0) return -3;
  if (k < 0) return -4;
  if (batch == 0 || m == 0 || n == 0) return 0;
  if (k > 0) {
    if (int w = check_op(sA, ai, aj, m, k, strideA, batch, false)) return pos_err(w, 6);
    if (int w = check_op(sB, bi, bj, k, n, strideB, batch, false)) return pos_err(w, 10);
  }
  if (beta != 0.0)
    if (int w = check_op(sC, ci, cj, m, n, strideC, batch, false)) return pos_err(w, 15);
  if (int w = check_op(sD, di, dj, m, n, strideD, batch, true)) return pos_err(w, 19);
  const Op A = make_op(k > 0 ? sA : nullptr, ai, aj, strideA);
  const Op B = make_op(k > 0 ? sB : nullptr, bi, bj, strideB);
  const Op C = make_op(beta != 0.0 ? sC : nullptr, ci, cj, strideC);
  const bool fast = fast_path({&A});
  return status(launch_gemm_nn(false, batch, m, n, k, alpha, A, B, beta, C, make_opw(sD, di, dj, strideD),
                               fast, (cudaStream_t)stream));
}

int bf_dgemm_nn(int m, int n, int k, double alpha, const bf_dmat *sA, int ai, int aj,
                const bf_dmat *sB, int bi, int bj, double beta, const bf_dmat *sC, int ci, int cj,
                const bf_dmat *sD, int di, int dj, void *stream) {
  const int r = bf_dgemm_nn_batched(1, m, n, k, alpha, sA, ai, aj, 0, sB, bi, bj, 0, beta, sC,
                                    ci, cj, 0, sD, di, dj, 0, stream);
  if (r >= 0) return r;
  static const int map[24] = {0, 0, 1, 2, 3, 4, 5, 6, 7, 0, 8, 9, 10, 0, 11, 12, 13, 14, 0, 15, 16, 17, 0, 18};
  return -map[-r];
}

int bf_dtrmm_rlnn_batched(int batch, int m, int n, double alpha, const bf_dmat *sL, int li, int lj,
                          long long strideL, const bf_dmat *sB, int bi, int bj, long long strideB,
                          const bf_dmat *sD, int di, int dj, long long strideD, void *stream) {
  if (batch < 0) return -1;
  if (m < 0) return -2;
  if (n < 0) return -3;
  if (batch == 0 || m == 0 || n == 0) return 0;
  if (int w = check_op(sL, li, lj, n, n, strideL, batch, false)) return pos_err(w, 5);
  if (int w = check_op(sB, bi, bj, m, n, strideB, batch, false)) return pos_err(w, 9);
  if (int w = check_op(sD, di, dj, m, n, strideD, batch, true)) return pos_err(w, 13);
  if (sD->pA == sB->pA) return -13;  // D is written while B is still read
  const Op B = make_op(sB, bi, bj, strideB);
  const Op none{nullptr, 0, 0, 0, 0};
  const bool fast = fast_path({&B});
  return status(launch_gemm_nn(true, batch, m, n, n, alpha, B, make_op(sL, li, lj, strideL), 0.0, none,
                               make_opw(sD, di, dj, strideD), fast, (cudaStream_t)stream));
}

int bf_dtrmm_rlnn(int m, int n, double alpha, const bf_dmat *sL, int li, int lj, const bf_dmat *sB,
                  int bi, int bj, const bf_dmat *sD, int di, int dj, void *stream) {
  const int r = bf_dtrmm_rlnn_batched(1, m, n, alpha, sL, li, lj, 0, sB, bi, bj, 0, sD, di, dj, 0, stream);
  if (r >= 0) return r;
  static const int map[17] = {0, 0, 1, 2, 3, 4, 5, 6, 0, 7, 8, 9, 0, 10, 11, 12, 0};
  return -map[-r];
}

int bf_dsyrk_ln_batched(int batch, int m, int k, double alpha, const bf_dmat *sA, int ai, int aj,
                        long long strideA, const bf_dmat *sB, int bi, int bj, long long strideB,
                        double beta, const bf_dmat *sC, int ci, int cj, long long strideC,
                        const bf_dmat *sD, int di, int dj, long long strideD, void *stream) {
  if (batch < 0) return -1;
  if (m < 0) return -2;
  if (k < 0) return -3;
  return gemm_like(true, batch, m, m, k, alpha, sA, ai, aj, strideA, sB, bi, bj, strideB, beta, sC,
                   ci, cj, strideC, sD, di, dj, strideD, stream);
}

int bf_dsyrk_ln(int m, int k, double alpha, const bf_dmat *sA, int ai, int aj, const bf_dmat *sB,
                int bi, int bj, double beta, const bf_dmat *sC, int ci, int cj, const bf_dmat *sD,
                int di, int dj, void *stream) {
  const int r = bf_dsyrk_ln_batched(1, m, k, alpha, sA, ai, aj, 0, sB, bi, bj, 0, beta, sC, ci, cj,
                                    0, sD, di, dj, 0, stream);
  if (r >= 0) return r;
  static const int map[23] = {0, 0, 1, 2, 3, 4, 5, 6, 0, 7, 8, 9, 0, 10, 11, 12, 13, 0, 14, 15, 16, 0, 17};
  return -map[-r];
}

// ------------------------------------------------------------------ trsm

int bf_dtrsm_rltn_batched(int batch, int m, int n, double alpha, const bf_dmat *sL, int li, int lj,
                          long long strideL, const double *dinv, long long strideDinv,
                          const bf_dmat *sB, int bi, int bj, long long strideB, const bf_dmat *sD,
                          int di, int dj, long long strideD, void *stream) {
  if (batch < 0) return -1;
  if (m < 0) return -2;
  if (n < 0) return -3;
  if (batch == 0 || m == 0 || n == 0) return 0;
  if (n > TRSM_MAX_N) return BF_ERR_UNSUPPORTED;
  if (int w = check_op(sL, li, lj, n, n, strideL, batch, false)) return pos_err(w, 5);
  if (dinv && !aligned_to(dinv, 8)) return -9;
  if (strideDinv < 0 || (dinv && batch > 1 && strideDinv < n && strideDinv != 0)) return -10;
  if (int w = check_op(sB, bi, bj, m, n, strideB, batch, false)) return pos_err(w, 11);
  if (int w = check_op(sD, di, dj, m, n, strideD, batch, true)) return pos_err(w, 15);
  return status(launch_trsm_rltn(batch, m, n, alpha, make_op(sL, li, lj, strideL), dinv,
                                 strideDinv, make_op(sB, bi, bj, strideB),
                                 make_opw(sD, di, dj, strideD), (cudaStream_t)stream));
}

int bf_dtrsm_rltn(int m, int n, double alpha, const bf_dmat *sL, int li, int lj, const bf_dmat *sB,
                  int bi, int bj, const bf_dmat *sD, int di, int dj, void *stream) {
  const int r = bf_dtrsm_rltn_batched(1, m, n, alpha, sL, li, lj, 0, nullptr, 0, sB, bi, bj, 0, sD,
                                      di, dj, 0, stream);
  if (r >= 0) return r;
  static const int map[19] = {0, 0, 1, 2, 3, 4, 5, 6, 0, 0, 0, 7, 8, 9, 0, 10, 11, 12, 0};
  return -map[-r];
}

// -------------------------------------------------------- potrf / syrk_potrf

static int chol_like(bool fused, int batch, int m, int k, const bf_dmat *sA, int ai, int aj,
                     long long strideA, const bf_dmat *sB, int bi, int bj, long long strideB,
                     const bf_dmat *sC, int ci, int cj, long long strideC, const bf_dmat *sD,
                     int di, int dj, long long strideD, double *dinv, long long strideDinv,
                     int *info, void *stream, int posC) {
  // posC: argument position of sC; the rest of the positions follow it
  if (batch == 0 || m == 0) return 0;
  if (m > CHOL_MAX_N) return BF_ERR_UNSUPPORTED;
  if (fused && k > 0) {
    if (int w = check_op(sA, ai, aj, m, k, strideA, batch, false)) return pos_err(w, 4);
    if (int w = check_op(sB, bi, bj, m, k, strideB, batch, false)) return pos_err(w, 8);
  }
  if (int w = check_op(sC, ci, cj, m, m, strideC, batch, false)) return pos_err(w, posC);
  if (int w = check_op(sD, di, dj, m, m, strideD, batch, true)) return pos_err(w, posC + 4);
  if (dinv && !aligned_to(dinv, 8)) return -(posC + 8);
  if (strideDinv < 0 || (dinv && batch > 1 && strideDinv < m)) return -(posC + 9);
  if (info && !aligned_to(info, 4)) return -(posC + 10);
  const Op A = make_op(fused && k > 0 ? sA : nullptr, ai, aj, strideA);
  const Op B = make_op(fused && k > 0 ? sB : nullptr, bi, bj, strideB);
  const Op C = make_op(sC, ci, cj, strideC);
  const OpW D = make_opw(sD, di, dj, strideD);
  const Op Dr = make_op(sD, di, dj, strideD);
  const bool fast = fast_path({&A, &B, &C, &Dr});
  return status(launch_chol(fused && k > 0, batch, m, k, A, B, C, D, dinv, strideDinv, info, fast,
                            (cudaStream_t)stream));
}

int bf_dpotrf_l_batched(int batch, int m, const bf_dmat *sC, int ci, int cj, long long strideC,
                        const bf_dmat *sD, int di, int dj, long long strideD, double *dinv,
                        long long strideDinv, int *info, void *stream) {
  if (batch < 0) return -1;
  if (m < 0) return -2;
  return chol_like(false, batch, m, 0, nullptr, 0, 0, 0, nullptr, 0, 0, 0, sC, ci, cj, strideC, sD,
                   di, dj, strideD, dinv, strideDinv, info, stream, 3);
}

int bf_dpotrf_l(int m, const bf_dmat *sC, int ci, int cj, const bf_dmat *sD, int di, int dj,
                int *info, void *stream) {
  const int r = bf_dpotrf_l_batched(1, m, sC, ci, cj, 0, sD, di, dj, 0, sD ? sD->dA : nullptr, 0,
                                    info, stream);
  if (r >= 0) return r;
  static const int map[14] = {0, 0, 1, 2, 3, 4, 0, 5, 6, 7, 0, 5, 0, 8};
  return -map[-r];
}

int bf_dsyrk_dpotrf_ln_batched(int batch, int m, int k, const bf_dmat *sA, int ai, int aj,
                               long long strideA, const bf_dmat *sB, int bi, int bj,
                               long long strideB, const bf_dmat *sC, int ci, int cj,
                               long long strideC, const bf_dmat *sD, int di, int dj,
                               long long strideD, double *dinv, long long strideDinv, int *info,
                               void *stream) {
  if (batch < 0) return -1;
  if (m < 0) return -2;
  if (k < 0) return -3;
  return chol_like(true, batch, m, k, sA, ai, aj, strideA, sB, bi, bj, strideB, sC, ci, cj, strideC,
                   sD, di, dj, strideD, dinv, strideDinv, info, stream, 12);
}

int bf_dsyrk_dpotrf_ln(int m, int k, const bf_dmat *sA, int ai, int aj, const bf_dmat *sB, int bi,
                       int bj, const bf_dmat *sC, int ci, int cj, const bf_dmat *sD, int di, int dj,
                       int *info, void *stream) {
  const int r = bf_dsyrk_dpotrf_ln_batched(1, m, k, sA, ai, aj, 0, sB, bi, bj, 0, sC, ci, cj, 0, sD,
                                           di, dj, 0, sD ? sD->dA : nullptr, 0, info, stream);
  if (r >= 0) return r;
  static const int map[23] = {0, 0, 1, 2, 3, 4, 5, 0, 6, 7, 8, 0, 9, 10, 11, 0, 12, 13, 14, 0, 12, 0, 15};
  return -map[-r];
}

// ------------------------------------------------------------------ solves

int bf_dpotrs_l_batched(int batch, int n, int nrhs, const bf_dmat *sL, int li, int lj,
                        long long strideL, const bf_dmat *sB, int bi, int bj, long long strideB,
                        const bf_dmat *sX, int xi, int xj, long long strideX, void *stream) {
  if (batch < 0) return -1;
  if (n < 0) return -2;
  if (nrhs < 0) return -3;
  if (batch == 0 || n == 0 || nrhs == 0) return 0;
  if (n > POTRS_MAX_N || nrhs > POSV_MAX_NRHS) return BF_ERR_UNSUPPORTED;
  if (int w = check_op(sL, li, lj, n, n, strideL, batch, false)) return pos_err(w, 4);
  if (int w = check_op(sB, bi, bj, n, nrhs, strideB, batch, false)) return pos_err(w, 8);
  if (int w = check_op(sX, xi, xj, n, nrhs, strideX, batch, true)) return pos_err(w, 12);
  return status(launch_potrs(batch, n, nrhs, make_op(sL, li, lj, strideL), make_op(sB, bi, bj, strideB),
                             make_opw(sX, xi, xj, strideX), (cudaStream_t)stream));
}

int bf_dposv_adjoint_batched(int batch, int n, int nrhs, const bf_dmat *sL, int li, int lj,
                             long long strideL, const bf_dmat *sX, int xi, int xj, long long strideX,
                             const bf_dmat *sXbar, int xbi, int xbj, long long strideXbar,
                             const bf_dmat *sBbar, int bbi, int bbj, long long strideBbar,
                             const bf_dmat *sAbar, int abi, int abj, long long strideAbar,
                             void *stream) {
  if (batch < 0) return -1;
  if (n < 0) return -2;
  if (nrhs < 0) return -3;
  if (batch == 0 || n == 0 || nrhs == 0) return 0;
  if (n > ADJOINT_MAX_N || nrhs > POSV_MAX_NRHS) return BF_ERR_UNSUPPORTED;
  if (int w = check_op(sL, li, lj, n, n, strideL, batch, false)) return pos_err(w, 4);
  if (int w = check_op(sX, xi, xj, n, nrhs, strideX, batch, false)) return pos_err(w, 8);
  if (int w = check_op(sXbar, xbi, xbj, n, nrhs, strideXbar, batch, false)) return pos_err(w, 12);
  if (int w = check_op(sBbar, bbi, bbj, n, nrhs, strideBbar, batch, true)) return pos_err(w, 16);
  if (int w = check_op(sAbar, abi, abj, n, n, strideAbar, batch, true)) return pos_err(w, 20);
  return status(launch_posv_adjoint(batch, n, nrhs, make_op(sL, li, lj, strideL), make_op(sX, xi, xj, strideX),
                                    make_op(sXbar, xbi, xbj, strideXbar), make_opw(sBbar, bbi, bbj, strideBbar),
                                    make_opw(sAbar, abi, abj, strideAbar), (cudaStream_t)stream));
}

size_t bf_dposv_mixed_worksize(int batch, int n) {
  if (batch <= 0 || n <= 0) return 0;
  const size_t pm = ((size_t)n + PS - 1) / PS * PS;
  const size_t l32 = ((size_t)batch * pm * n * sizeof(float) + BF_ALIGN - 1) / BF_ALIGN * BF_ALIGN;
  const size_t info = ((size_t)batch * sizeof(int) + BF_ALIGN - 1) / BF_ALIGN * BF_ALIGN;
  return l32 + info;
}

}  // extern "C"

// Checks of the arguments the two mixed-precision solver entry points share
// (positions 1..19); returns 0, a negative position or BF_ERR_UNSUPPORTED.
// A zero-sized call passes, and the caller returns 0 for it.
int bf::posv_mixed_check(int batch, int n, int nrhs, const bf_dmat *sA, int ai, int aj, long long strideA,
                         const bf_dmat *sB, int bi, int bj, long long strideB, const bf_dmat *sX, int xi,
                         int xj, long long strideX, double tol, int max_iter, const int *iters,
                         const double *resid) {
  if (batch < 0) return -1;
  if (n < 0) return -2;
  if (nrhs < 0) return -3;
  if (batch == 0 || n == 0 || nrhs == 0) return 0;
  if (n > POSV_MAX_N || nrhs > POSV_MAX_NRHS) return BF_ERR_UNSUPPORTED;
  if (int w = check_op(sA, ai, aj, n, n, strideA, batch, false)) return pos_err(w, 4);
  if (int w = check_op(sB, bi, bj, n, nrhs, strideB, batch, false)) return pos_err(w, 8);
  if (int w = check_op(sX, xi, xj, n, nrhs, strideX, batch, true)) return pos_err(w, 12);
  if (sX->pA == sB->pA) return -12;
  if (!(tol >= 0.0)) return -16;
  if (max_iter < 1) return -17;
  if (iters && !aligned_to(iters, 4)) return -18;
  if (resid && !aligned_to(resid, 8)) return -19;
  return 0;
}

extern "C" {

int bf_dposv_mixed_batched(int batch, int n, int nrhs, const bf_dmat *sA, int ai, int aj,
                           long long strideA, const bf_dmat *sB, int bi, int bj, long long strideB,
                           const bf_dmat *sX, int xi, int xj, long long strideX, double tol,
                           int max_iter, int *iters, double *resid, void *work, size_t work_bytes,
                           void *stream) {
  if (int r = posv_mixed_check(batch, n, nrhs, sA, ai, aj, strideA, sB, bi, bj, strideB, sX, xi, xj,
                               strideX, tol, max_iter, iters, resid))
    return r;
  if (batch == 0 || n == 0 || nrhs == 0) return 0;
  if (!work || !aligned_to(work, BF_ALIGN)) return -20;
  if (work_bytes < bf_dposv_mixed_worksize(batch, n)) return -21;
  const size_t pm = ((size_t)n + PS - 1) / PS * PS;
  float *l32 = (float *)work;
  int *info32 = (int *)((char *)work + ((size_t)batch * pm * n * sizeof(float) + BF_ALIGN - 1) / BF_ALIGN * BF_ALIGN);
  const Op A = make_op(sA, ai, aj, strideA);
  const bool fast = fast_path({&A});
  return status(launch_posv_mixed(batch, n, nrhs, A, make_op(sB, bi, bj, strideB),
                                  make_opw(sX, xi, xj, strideX), tol, max_iter, iters, resid, l32,
                                  info32, fast, (cudaStream_t)stream));
}

static size_t round_up(size_t x) { return (x + BF_ALIGN - 1) / BF_ALIGN * BF_ALIGN; }

size_t bf_dposv_mixed_tc_worksize(int batch, int n) {
  if (batch <= 0 || n <= 0) return 0;
  const size_t pm = ((size_t)n + PS - 1) / PS * PS, nblk = ((size_t)n + 31) / 32, bt = (size_t)batch;
  return round_up(bt * pm * n * 8) + round_up(bt * n * 8) + round_up(bt * pm * n * 4) + round_up(nblk * bt * 4) +
         round_up(bt * 4);
}

int bf_dposv_mixed_tc_batched(int batch, int n, int nrhs, const bf_dmat *sA, int ai, int aj, long long strideA,
                              const bf_dmat *sB, int bi, int bj, long long strideB, const bf_dmat *sX, int xi,
                              int xj, long long strideX, double tol, int max_iter, int *iters, double *resid,
                              int prec, void *work, size_t work_bytes, void *stream) {
  if (int r = posv_mixed_check(batch, n, nrhs, sA, ai, aj, strideA, sB, bi, bj, strideB, sX, xi, xj, strideX, tol,
                               max_iter, iters, resid))
    return r;
  if (prec < 0 || prec > 2) return -20;
  if (batch == 0 || n == 0 || nrhs == 0) return 0;
  if (n > POSV_TC_MAX_N) return BF_ERR_UNSUPPORTED;
  if (!work || !aligned_to(work, BF_ALIGN)) return -21;
  if (work_bytes < bf_dposv_mixed_tc_worksize(batch, n)) return -22;
  const size_t pm = ((size_t)n + PS - 1) / PS * PS, nblk = ((size_t)n + 31) / 32, bt = (size_t)batch;
  char *w = (char *)work;
  double *W = (double *)w;
  w += round_up(bt * pm * n * 8);
  double *dinv = (double *)w;
  w += round_up(bt * n * 8);
  float *l32 = (float *)w;
  w += round_up(bt * pm * n * 4);
  int *infos = (int *)w;
  w += round_up(nblk * bt * 4);
  int *info32 = (int *)w;
  return status(launch_posv_mixed_tc(prec, batch, n, nrhs, make_op(sA, ai, aj, strideA), make_op(sB, bi, bj, strideB),
                                     make_opw(sX, xi, xj, strideX), tol, max_iter, iters, resid, W, dinv, l32, infos,
                                     info32, (cudaStream_t)stream));
}

int bf_dsyrk_ln_tc_batched(int batch, int m, int k, int prec, const bf_dmat *sA, int ai, int aj, long long strideA,
                           const bf_dmat *sC, int ci, int cj, long long strideC, const bf_dmat *sD, int di, int dj,
                           long long strideD, void *stream) {
  if (batch < 0) return -1;
  if (m < 0) return -2;
  if (k < 0) return -3;
  if (prec < 0 || prec > 2) return -4;
  if (batch == 0 || m == 0) return 0;
  if (m > 128 || k > 32 || k == 0) return BF_ERR_UNSUPPORTED;
  if (int w = check_op(sA, ai, aj, m, k, strideA, batch, false)) return pos_err(w, 5);
  if (int w = check_op(sC, ci, cj, m, m, strideC, batch, false)) return pos_err(w, 9);
  if (int w = check_op(sD, di, dj, m, m, strideD, batch, true)) return pos_err(w, 13);
  const Op A = make_op(sA, ai, aj, strideA);
  if (!syrk_tc_ok(m, k, A)) return -5;  // rows off a panel top, or runs not 16-byte aligned
  return status(launch_syrk_tc(prec, batch, m, k, A, make_op(sC, ci, cj, strideC), make_opw(sD, di, dj, strideD),
                               nullptr, (cudaStream_t)stream));
}

// ------------------------------------------------------------ getrf / gelqf

int bf_dgetrf_batched(int batch, int n, const bf_dmat *sC, int ci, int cj, long long strideC,
                      const bf_dmat *sD, int di, int dj, long long strideD, int *ipiv,
                      long long strideIpiv, int *info, void *stream) {
  if (batch < 0) return -1;
  if (n < 0) return -2;
  if (batch == 0 || n == 0) return 0;
  if (n > GETRF_MAX_N) return BF_ERR_UNSUPPORTED;
  if (int w = check_op(sC, ci, cj, n, n, strideC, batch, false)) return pos_err(w, 3);
  if (int w = check_op(sD, di, dj, n, n, strideD, batch, true)) return pos_err(w, 7);
  if (!ipiv || !aligned_to(ipiv, 4)) return -11;
  if (strideIpiv < 0 || (batch > 1 && strideIpiv < n)) return -12;
  if (info && !aligned_to(info, 4)) return -13;
  return status(launch_getrf(batch, n, make_op(sC, ci, cj, strideC), make_opw(sD, di, dj, strideD), ipiv,
                             strideIpiv, info, (cudaStream_t)stream));
}

int bf_dgetrf(int n, const bf_dmat *sC, int ci, int cj, const bf_dmat *sD, int di, int dj, int *ipiv,
              int *info, void *stream) {
  const int r = bf_dgetrf_batched(1, n, sC, ci, cj, 0, sD, di, dj, 0, ipiv, 0, info, stream);
  if (r >= 0) return r;
  static const int map[14] = {0, 0, 1, 2, 3, 4, 0, 5, 6, 7, 0, 8, 0, 9};
  return -map[-r];
}

int bf_dgelqf_batched(int batch, int m, int n, const bf_dmat *sC, int ci, int cj, long long strideC,
                      const bf_dmat *sD, int di, int dj, long long strideD, double *tau,
                      long long strideTau, void *stream) {
  if (batch < 0) return -1;
  if (m < 0) return -2;
  if (n < 0) return -3;
  if (batch == 0 || m == 0 || n == 0) return 0;
  if ((long long)m * n > GELQF_ONE_CTA_MAX_MN && (m > GELQF_MAX_DIM || n > GELQF_MAX_DIM)) return BF_ERR_UNSUPPORTED;
  if (int w = check_op(sC, ci, cj, m, n, strideC, batch, false)) return pos_err(w, 4);
  if (int w = check_op(sD, di, dj, m, n, strideD, batch, true)) return pos_err(w, 8);
  const int k = m < n ? m : n;
  if (!tau || !aligned_to(tau, 8)) return -12;
  if (strideTau < 0 || (batch > 1 && strideTau < k)) return -13;
  return status(launch_gelqf(batch, m, n, make_op(sC, ci, cj, strideC), make_opw(sD, di, dj, strideD), tau,
                             strideTau, (cudaStream_t)stream));
}

int bf_dgelqf(int m, int n, const bf_dmat *sC, int ci, int cj, const bf_dmat *sD, int di, int dj,
              double *tau, void *stream) {
  const int r = bf_dgelqf_batched(1, m, n, sC, ci, cj, 0, sD, di, dj, 0, tau, 0, stream);
  if (r >= 0) return r;
  static const int map[14] = {0, 0, 1, 2, 3, 4, 5, 0, 6, 7, 8, 0, 9, 0};
  return -map[-r];
}

int bf_dsub_valid(const bf_dsub *rec, int rows, int cols) { return rec && dsub_ok(*rec, rows, cols) ? 1 : 0; }

// ----------------------------------------------- descriptor-array batched forms
// Host checks cover the call's own arguments; each problem's record is
// checked on the device (status array).

int bf_dgemm_nt_vbatched(int batch, const bf_dsize *size, double alpha, const bf_dsub *A, const bf_dsub *B,
                         double beta, const bf_dsub *C, const bf_dsub *D, int max_m, int max_n, int *st,
                         void *stream) {
  if (batch < 0) return -1;
  if (batch > 0 && !size) return -2;
  if (batch > 0 && !A) return -4;
  if (batch > 0 && !B) return -5;
  if (batch > 0 && beta != 0.0 && !C) return -7;
  if (batch > 0 && !D) return -8;
  if (max_m < 0) return -9;
  if (max_n < 0) return -10;
  if (batch == 0 || max_m == 0 || max_n == 0) return 0;
  return status(launch_gemm_nt_v(false, batch, size, alpha, A, B, beta, C, D, max_m, max_n, st,
                                 (cudaStream_t)stream));
}

int bf_dsyrk_ln_vbatched(int batch, const bf_dsize *size, double alpha, const bf_dsub *A, const bf_dsub *B,
                         double beta, const bf_dsub *C, const bf_dsub *D, int max_m, int *st, void *stream) {
  if (batch < 0) return -1;
  if (batch > 0 && !size) return -2;
  if (batch > 0 && !A) return -4;
  if (batch > 0 && !B) return -5;
  if (batch > 0 && beta != 0.0 && !C) return -7;
  if (batch > 0 && !D) return -8;
  if (max_m < 0) return -9;
  if (batch == 0 || max_m == 0) return 0;
  return status(launch_gemm_nt_v(true, batch, size, alpha, A, B, beta, C, D, max_m, max_m, st,
                                 (cudaStream_t)stream));
}

int bf_dpotrf_l_vbatched(int batch, const bf_dsize *size, const bf_dsub *C, const bf_dsub *D, int want_dinv,
                         int *info, int max_m, int *st, void *stream) {
  if (batch < 0) return -1;
  if (batch > 0 && !size) return -2;
  if (batch > 0 && !C) return -3;
  if (batch > 0 && !D) return -4;
  if (info && !aligned_to(info, 4)) return -6;
  if (max_m < 0) return -7;
  if (max_m > CHOL_MAX_N) return BF_ERR_UNSUPPORTED;
  if (batch == 0 || max_m == 0) return 0;
  return status(launch_chol_v(false, batch, size, nullptr, nullptr, C, D, want_dinv != 0, info, max_m, st,
                              (cudaStream_t)stream));
}

int bf_dtrsm_rltn_vbatched(int batch, const bf_dsize *size, double alpha, const bf_dsub *L, int use_dinv,
                           const bf_dsub *B, const bf_dsub *D, int max_m, int max_n, int *st, void *stream) {
  if (batch < 0) return -1;
  if (batch > 0 && !size) return -2;
  if (batch > 0 && !L) return -4;
  if (batch > 0 && !B) return -6;
  if (batch > 0 && !D) return -7;
  if (max_m < 0) return -8;
  if (max_n < 0) return -9;
  if (max_n > TRSM_MAX_N) return BF_ERR_UNSUPPORTED;
  if (batch == 0 || max_m == 0 || max_n == 0) return 0;
  return status(launch_trsm_rltn_v(batch, size, alpha, L, use_dinv != 0, B, D, max_m, max_n, st,
                                   (cudaStream_t)stream));
}

int bf_dsyrk_dpotrf_ln_vbatched(int batch, const bf_dsize *size, const bf_dsub *A, const bf_dsub *B,
                                const bf_dsub *C, const bf_dsub *D, int want_dinv, int *info, int max_m,
                                int *st, void *stream) {
  if (batch < 0) return -1;
  if (batch > 0 && !size) return -2;
  if (batch > 0 && !A) return -3;
  if (batch > 0 && !B) return -4;
  if (batch > 0 && !C) return -5;
  if (batch > 0 && !D) return -6;
  if (info && !aligned_to(info, 4)) return -8;
  if (max_m < 0) return -9;
  if (max_m > CHOL_MAX_N) return BF_ERR_UNSUPPORTED;
  if (batch == 0 || max_m == 0) return 0;
  return status(launch_chol_v(true, batch, size, A, B, C, D, want_dinv != 0, info, max_m, st,
                              (cudaStream_t)stream));
}

int bf_vbatched_order(int batch, const bf_dsize *size, int max_m, int *order, void *stream) {
  if (batch < 0) return -1;
  if (batch > 0 && !size) return -2;
  if (max_m < 0) return -3;
  if (max_m > CHOL_MAX_N) return BF_ERR_UNSUPPORTED;
  if (batch > 0 && (!order || !aligned_to(order, 4))) return -4;
  if (batch == 0) return 0;
  return status(launch_vbatched_order(batch, size, max_m, order, (cudaStream_t)stream));
}

int bf_dpotrf_l_vbatched_ordered(int batch, const bf_dsize *size, const int *order, const bf_dsub *C,
                                 const bf_dsub *D, int want_dinv, int *info, int max_m, int *st, void *stream) {
  if (batch < 0) return -1;
  if (batch > 0 && !size) return -2;
  if (order && !aligned_to(order, 4)) return -3;
  if (batch > 0 && !C) return -4;
  if (batch > 0 && !D) return -5;
  if (info && !aligned_to(info, 4)) return -7;
  if (max_m < 0) return -8;
  if (max_m > CHOL_MAX_N) return BF_ERR_UNSUPPORTED;
  if (batch == 0 || max_m == 0) return 0;
  return status(launch_chol_vp(false, batch, order, size, nullptr, nullptr, C, D, want_dinv != 0, info, max_m, st,
                               (cudaStream_t)stream));
}

int bf_dsyrk_dpotrf_ln_vbatched_ordered(int batch, const bf_dsize *size, const int *order, const bf_dsub *A,
                                        const bf_dsub *B, const bf_dsub *C, const bf_dsub *D, int want_dinv,
                                        int *info, int max_m, int *st, void *stream) {
  if (batch < 0) return -1;
  if (batch > 0 && !size) return -2;
  if (order && !aligned_to(order, 4)) return -3;
  if (batch > 0 && !A) return -4;
  if (batch > 0 && !B) return -5;
  if (batch > 0 && !C) return -6;
  if (batch > 0 && !D) return -7;
  if (info && !aligned_to(info, 4)) return -9;
  if (max_m < 0) return -10;
  if (max_m > CHOL_MAX_N) return BF_ERR_UNSUPPORTED;
  if (batch == 0 || max_m == 0) return 0;
  return status(launch_chol_vp(true, batch, order, size, A, B, C, D, want_dinv != 0, info, max_m, st,
                               (cudaStream_t)stream));
}

// ---------------------------------------------------------------- Riccati

int bf_driccati_sqrt_batched(int batch, int N, const bf_riccati_prob *probs, const int *order,
                             int max_nx, int max_nu, int threads, void *stream) {
  if (batch < 0) return -1;
  if (N < 0) return -2;
  if (batch == 0 || N == 0) return 0;
  if (!probs || !aligned_to(probs, 8)) return -3;
  if (order && !aligned_to(order, 4)) return -4;
  if (max_nx < 1) return -5;
  if (max_nu < 1) return -6;
  if (threads == 0) threads = 256;
  if (threads < 32 || threads > 512 || threads % 32 != 0) return -7;
  if (riccati_smem(max_nx, max_nu) > 200 * 1024) return BF_ERR_UNSUPPORTED;
  return status(launch_riccati(batch, N, probs, order, max_nx, max_nu, threads, (cudaStream_t)stream));
}

}  // extern "C"
