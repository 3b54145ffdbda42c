// gemm_nn and trmm_rlnn, batched, FP64, panel-major operands.
//
// gemm_nn (Sec. 5.2.2 "gemm_nn"):      D <- alpha * A * B + beta * C
//   A is m x k, B is k x n.  A is read along its panels as in gemm_nt; B is
//   read across its panels (column j of the register block is one element
//   of row l of B, four columns 32 bytes apart), the access pattern the paper
//   notes for this variant.
// trmm_rlnn (Sec. 5.2.2 "trmm_rlnn"; right, lower, not transposed, non-unit):
//                                       D <- alpha * B * L
//   B is m x n, L is n x n lower triangular (its strictly upper part is not
//   read).  Column j of D only needs rows l >= j of L, so a register block's
//   k-loop starts at its first column and masks the triangle for the first
//   four steps.
//
// Same thread layout as gemm_nt: one thread per 4x4 register block of one
// problem's D, threads numbered over (problem, block) so warps stay full;
// trmm numbers a problem's blocks column by column.
#include "bf_internal.cuh"

namespace bf {
namespace {

template <bool TRMM, bool ALIGNED>
__global__ void __launch_bounds__(128)
k_gemm_nn(int batch, int m, int n, int k, double alpha, Op A, Op X, double beta, Op C, OpW D,
          int tiles_c, int tiles_pp) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)batch * tiles_pp) return;
  const int b = (int)(t / tiles_pp);
  const int tt = (int)(t - (long long)b * tiles_pp);
  // trmm: blocks numbered down the block columns, so that the lanes of a warp
  // share (nearly) the same k-range [j0, n) and none waits on a longer one
  int tr, tc;
  if (TRMM) {
    const int tiles_r = tiles_pp / tiles_c;
    tc = tt / tiles_r;
    tr = tt - tc * tiles_r;
  } else {
    tr = tt / tiles_c;
    tc = tt - tr * tiles_c;
  }
  const int i0 = tr * 4, j0 = tc * 4;
  const double *pa = A.p + b * A.stride;
  const double *px = X.p + b * X.stride;
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; r++)
#pragma unroll
    for (int c = 0; c < 4; c++) acc[r][c] = 0.0;

  // columns of the register block past n read column n-1 (never stored)
  int jc[4];
#pragma unroll
  for (int c = 0; c < 4; c++) jc[c] = min(j0 + c, n - 1);
  const int lbeg = TRMM ? j0 : 0;
  const int lend = TRMM ? n : k;

  const double *ar[4];
#pragma unroll
  for (int r = 0; r < 4; r++) ar[r] = pa + pm_off(A.i0 + min(i0 + r, m - 1), A.j0, A.cn);
  const double *ap = ALIGNED ? pa + (long long)(A.i0 + i0) * A.cn + (long long)A.j0 * PS : nullptr;

#pragma unroll 2
  for (int l = lbeg; l < lend; l++) {
    double av[4], xv[4];
    if (ALIGNED) {
      const double2 a01 = __ldg((const double2 *)(ap + (long long)l * PS));
      const double2 a23 = __ldg((const double2 *)(ap + (long long)l * PS + 2));
      av[0] = a01.x; av[1] = a01.y; av[2] = a23.x; av[3] = a23.y;
    } else {
#pragma unroll
      for (int r = 0; r < 4; r++) av[r] = __ldg(ar[r] + (long long)l * PS);
    }
    const double *xrow = px + pm_off(X.i0 + l, X.j0, X.cn);
#pragma unroll
    for (int c = 0; c < 4; c++) {
      const double v = __ldg(xrow + (long long)jc[c] * PS);
      xv[c] = (TRMM && l < j0 + c) ? 0.0 : v;  // L(l, j) = 0 above the diagonal
    }
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
      for (int c = 0; c < 4; c++) acc[r][c] = fma(av[r], xv[c], acc[r][c]);
  }

  double *pd = D.p + b * D.stride;
  const double *pc = (!TRMM && beta != 0.0) ? C.p + b * C.stride : nullptr;
#pragma unroll
  for (int r = 0; r < 4; r++)
#pragma unroll
    for (int c = 0; c < 4; c++) {
      const int i = i0 + r, j = j0 + c;
      if (i < m && j < n) {
        double v = alpha * acc[r][c];
        if (pc) v = fma(beta, pc[pm_off(C.i0 + i, C.j0 + j, C.cn)], v);
        pd[pm_off(D.i0 + i, D.j0 + j, D.cn)] = v;
      }
    }
}

}  // namespace

cudaError_t launch_gemm_nn(bool trmm, int batch, int m, int n, int k, double alpha, Op A, Op X,
                           double beta, Op C, OpW D, bool aligned, cudaStream_t s) {
  const int tcn = (n + 3) / 4;
  const int tiles_pp = ((m + 3) / 4) * tcn;
  const long long total = (long long)batch * tiles_pp;
  const long long blocks = (total + 127) / 128;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  if (trmm) {
    if (aligned)
      k_gemm_nn<true, true><<<(unsigned)blocks, 128, 0, s>>>(batch, m, n, k, alpha, A, X, beta, C, D, tcn, tiles_pp);
    else
      k_gemm_nn<true, false><<<(unsigned)blocks, 128, 0, s>>>(batch, m, n, k, alpha, A, X, beta, C, D, tcn, tiles_pp);
  } else {
    if (aligned)
      k_gemm_nn<false, true><<<(unsigned)blocks, 128, 0, s>>>(batch, m, n, k, alpha, A, X, beta, C, D, tcn, tiles_pp);
    else
      k_gemm_nn<false, false><<<(unsigned)blocks, 128, 0, s>>>(batch, m, n, k, alpha, A, X, beta, C, D, tcn, tiles_pp);
  }
  return cudaGetLastError();
}

}  // namespace bf
