// Backward Riccati recursion of linear MPC (Sec. 5.3), square-root form,
// batched over independent instances of different sizes.
//
// For dynamics x+ = A x + B u (A nx x nx, B nx x nu) and stage cost matrix
// M0 = [[R, S^T], [S, Q]], each stage k = N-1, ..., 0 computes from the
// factor Lc = chol(P_{k+1}) (P_N given by its factor LN):
//     C                 = [B^T; A^T] * Lc            (trmm_rlnn)
//     [[Lam, 0],
//      [Lo,  Lc_k]]     = chol(M0 + C C^T)           (syrk_potrf_ln, fused)
//     Kt_k * Lam        = -Lo                        (trsm_rlnn; Kt_k = K_k^T)
// so that Lc_k Lc_k^T = P_k and K_k is the feedback gain u = K_k x.
//
// GB300 design.  Instances are independent and a stage of one instance needs
// only the previous stage of the same instance, so one CTA carries one
// instance through all N stages with Lc kept in shared memory: there is no
// launch or grid-wide synchronization between stages, and only the outputs
// (Lc_k, Kt_k) go to HBM.  The block scheduler hands out CTAs in blockIdx
// order, so the caller passes the instances sorted by decreasing cost
// (`order`) and the machine balances the uneven sizes as in longest-job-first
// scheduling.  Instances are grouped in size buckets, each launch sizing its
// shared memory and CTA width for its bucket.
//
// Within a CTA, the trmm and syrk put rows on lanes (all lanes of a warp run
// dot products of the same length); the factorization is right-looking over
// the packed lower triangle of M in panels of 4 columns (warp 0 factors a
// panel, all threads apply its rank-4 update), and the gain is one thread per
// row of Kt walking the columns of Lam backwards with the saved reciprocals.
#include "bf_internal.cuh"

namespace bf {
namespace {

__device__ __forceinline__ int col_start(int l, int n) { return (l * (2 * n - l + 1)) / 2 - l; }

#ifndef BF_RICCATI_RB
#define BF_RICCATI_RB 4
#endif
constexpr int RB = BF_RICCATI_RB;  // panel width of the factorization

// column of packed lower element e in an s x s triangle (element (i, l) at col_start(l, s) + i)
__device__ __forceinline__ int packed_col(int e, int s) {
  const float q = 2.0f * s + 1.0f;
  int l = (int)((q - sqrtf(fmaxf(q * q - 8.0f * e, 0.0f))) * 0.5f);
  l = max(0, min(l, s - 1));
  while (l > 0 && col_start(l, s) + l > e) l--;
  while (l + 1 < s && col_start(l + 1, s) + l + 1 <= e) l++;
  return l;
}

__global__ void __launch_bounds__(512)
k_riccati(int batch, int N, const bf_riccati_prob *probs, const int *order, int max_nx, int max_nu) {
  extern __shared__ double sm[];
  const int t = threadIdx.x, T = blockDim.x;
  if (blockIdx.x >= (unsigned)batch) return;
  const int p = order ? order[blockIdx.x] : (int)blockIdx.x;
  const bf_riccati_prob P = probs[p];
  const int nx = P.nx, nu = P.nu, m = nx + nu;
  if (nx < 1 || nu < 1 || nx > max_nx || nu > max_nu) {
    // descriptor outside this launch's bucket: report, compute nothing
    if (P.info)
      for (int k = t; k < N; k += T) P.info[k] = -1;
    return;
  }
  const int cp = nx + 1;
  double *C = sm;                           // m x nx, row-major, pitch cp (reused for Kt)
  double *M = C + m * cp;                   // packed lower m x m, column-major
  double *rv = M + m * (m + 1) / 2;         // 1 / pivot of each column of M
  __shared__ int s_bad;
  // The factor Lc of the next stage's P is the trailing nx x nx block of M's
  // factor, so it is read in place: Lc(l, j) = M[col_start(nu + j) + nu + l].
  for (int e = t; e < nx * nx; e += T) {
    const int j = e / nx, i = e - j * nx;
    if (i >= j) M[col_start(nu + j, m) + nu + i] = P.LN[pm_off(i, j, P.ln_cn)];
  }
  __syncthreads();

  for (int k = N - 1; k >= 0; k--) {
    // (1) C = [B^T; A^T] * Lc: C(i, j) = sum_{l >= j} BAt(i, l) Lc(l, j)
    for (int e = t; e < m * nx; e += T) {
      const int j = e / m, i = e - j * m;
      const double *brow = P.BAt + pm_off(i, 0, P.bat_cn);
      const double *lcol = M + col_start(nu + j, m) + nu;  // column j of Lc, rows l >= j at lcol[l]
      double acc = 0.0;
      for (int l = j; l < nx; l++) acc = fma(__ldg(brow + (long long)l * PS), lcol[l], acc);
      C[i * cp + j] = acc;
    }
    if (t == 0) s_bad = 0;
    __syncthreads();  // M (holding Lc) is overwritten next

    // (2) M = M0 + C C^T, lower triangle
    const int NE = m * (m + 1) / 2;
    for (int e = t; e < NE; e += T) {
      const int j = packed_col(e, m), i = e - col_start(j, m);
      double acc = __ldg(P.M0 + pm_off(i, j, P.m0_cn));
      const double *ci = C + i * cp, *cj = C + j * cp;
      for (int l = 0; l < nx; l++) acc = fma(ci[l], cj[l], acc);
      M[e] = acc;
    }
    __syncthreads();

    // (3) Cholesky of M, right-looking in panels of RB columns: warp 0
    // factors the panel (rows j0..m-1) with warp-level syncs only, then all
    // threads apply its rank-RB update to the trailing triangle.  Two CTA
    // barriers per panel instead of two per column.
    for (int j0 = 0; j0 < m; j0 += RB) {
      const int jb = min(RB, m - j0);
      if (t < 32) {
        for (int jj = 0; jj < jb; jj++) {
          const int j = j0 + jj, cj = col_start(j, m);
          const double d = M[cj + j];
          const double r = rsqrt(d);
          __syncwarp();
          if (t == 0) {
            rv[j] = r;
            M[cj + j] = d * r;
            if (s_bad == 0 && not_positive(d)) s_bad = j + 1;
          }
          for (int i = j + 1 + t; i < m; i += 32) M[cj + i] *= r;
          __syncwarp();
          for (int c = j + 1; c < j0 + jb; c++) {  // the rest of the panel
            const double lc = M[cj + c];
            const int cc = col_start(c, m);
            for (int i = c + t; i < m; i += 32) M[cc + i] = fma(-M[cj + i], lc, M[cc + i]);
          }
          __syncwarp();
        }
      }
      __syncthreads();
      const int s = m - j0 - jb;  // trailing triangle rows/cols j0+jb .. m-1
      const int TE = s * (s + 1) / 2;
      for (int e = t; e < TE; e += T) {
        const int kk = packed_col(e, s), ii = e - col_start(kk, s);
        const int kc = j0 + jb + kk, ic = j0 + jb + ii;
        const int idx = col_start(kc, m) + ic;
        double v = M[idx];
        for (int jj = 0; jj < jb; jj++) {
          const int cj = col_start(j0 + jj, m);
          v = fma(-M[cj + ic], M[cj + kc], v);
        }
        M[idx] = v;
      }
      __syncthreads();
    }

    // (4) outputs: Kt * Lam = -Lo, then the new factor Lc = M[nu:, nu:]
    double *X = C;  // nx x nu, pitch nu + 1
    double *kt = P.Kt + (long long)k * P.kt_stride;
    for (int i = t; i < nx; i += T) {
      for (int j = nu - 1; j >= 0; j--) {
        double s = -M[col_start(j, m) + nu + i];
        for (int l = j + 1; l < nu; l++) s = fma(-X[i * (nu + 1) + l], M[col_start(j, m) + l], s);
        s *= rv[j];
        X[i * (nu + 1) + j] = s;
        kt[pm_off(i, j, P.kt_cn)] = s;
      }
    }
    double *lk = P.L + (long long)k * P.l_stride;
    for (int e = t; e < nx * nx; e += T) {
      const int i = e / nx, j = e - i * nx;
      if (j <= i) lk[pm_off(i, j, P.l_cn)] = M[col_start(nu + j, m) + nu + i];
    }
    if (t == 0 && P.info) P.info[k] = s_bad;
    __syncthreads();
  }
}

}  // namespace

size_t riccati_smem(int max_nx, int max_nu) {
  const size_t nx = max_nx, m = (size_t)max_nx + max_nu;
  return (m * (nx + 1) + m * (m + 1) / 2 + m) * sizeof(double);
}

cudaError_t launch_riccati(int batch, int N, const bf_riccati_prob *probs, const int *order,
                           int max_nx, int max_nu, int threads, cudaStream_t s) {
  const size_t smem = riccati_smem(max_nx, max_nu);
  static std::atomic<unsigned long long> attr{0};
  cudaError_t e = smem_attr_once((const void *)k_riccati, 200 * 1024, attr);
  if (e != cudaSuccess) return e;
  k_riccati<<<batch, threads, smem, s>>>(batch, N, probs, order, max_nx, max_nu);
  return cudaGetLastError();
}

}  // namespace bf
