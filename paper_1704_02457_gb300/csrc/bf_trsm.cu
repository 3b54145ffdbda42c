// trsm_rltn, batched, FP64, panel-major operands (Sec. 5.2.2; right, lower,
// transposed, non-unit):
//     D <- alpha * B * L^{-T}   i.e. the X with X * L^T = alpha * B.
//
// Rows of X are independent: row i solves x_i L^T = alpha b_i by forward
// substitution over the columns.  One thread owns one row and walks the
// columns in blocks of up to 32 held in registers.  For block [c0, c0+W):
//   (a) acc = alpha * B[i][c0..]
//   (b) acc -= X[i][0:c0] * L[c0..][0:c0]^T     (the gemm_nt downdate, merged
//       into the solve kernel as the paper does for trsm, Sec. 4.6)
//   (d) substitution against the diagonal block L[c0..][c0..], multiplying
//       by the inverse diagonal (Sec. 4.7.1): from the caller's dinv when
//       given (as written by potrf), else one reciprocal per column computed
//       once per CTA, so no thread divides in its inner loop.
// L's rows are shared by all threads of a problem: the diagonal block and the
// downdate chunks are staged in shared memory and read as broadcasts.  A CTA
// packs the rows of several small problems so that warps stay full; a problem
// with more than 256 rows is split over several CTAs.
#include "bf_internal.cuh"

namespace bf {
namespace {

constexpr int KC = 32;        // columns of L per staged downdate chunk
constexpr int SPITCH = 34;    // stage row pitch (even: 16-byte pair loads)
// Rows of X per CTA above which a problem's rows are split over several
// CTAs (rows are independent; each CTA stages the L blocks it needs).
// Measured with the sweep's batches: trsm n = 192 1204 -> 1225 GFLOP/s at
// 128 (n = 256 unchanged); 64 also slowed n = 96 (1216 -> 1183).
// Rows of a CTA that packs whole small problems (n <= 32).  Measured: 128
// against 256 took trsm n = 24 1049 -> 1057 and n = 32 1140 -> 1154 GFLOP/s,
// the other sweep sizes unchanged within noise.
#ifndef BF_TRSM_PACK_ROWS
#define BF_TRSM_PACK_ROWS 128
#endif
#ifndef BF_TRSM_MAX_ROWS
#define BF_TRSM_MAX_ROWS 128
#endif
constexpr int MAX_ROWS = 256;                // rows per CTA at most
constexpr int CHUNK_ROWS = BF_TRSM_MAX_ROWS;  // rows per CTA when a problem is split

__host__ __device__ __forceinline__ int ls_region(int W) { return W * (W + 1) + W + 1; }

// block width bucket: 4, 8, 16, 24 or 32 columns
__host__ __device__ __forceinline__ int w_bucket(int w) { return w <= 4 ? 4 : (w + 7) & ~7; }

template <int W>
__device__ __forceinline__ void trsm_block(double *smem, int P, int R, int c0, int m, int n,
                                           double alpha, int pb0, int batch, int r0, Op L,
                                           const double *dinv, long long sdinv, Op B, OpW D) {
  const int t = threadIdx.x;
  const int T = blockDim.x;
  const int w = min(32, n - c0);
  const int RS = ls_region(W);
  double *stage_base = smem + (((size_t)P * RS + 1) & ~(size_t)1);  // 16-byte aligned

  const int p = t / R;
  const int row = r0 + (t - p * R);
  const int b = pb0 + p;
  const bool active = (p < P) && (row < m) && (b < batch);
  double *Ls = smem + (size_t)min(p, P - 1) * RS;  // Ls[jj*(W+1) + j], then rinv[W]
  double *rinv = Ls + W * (W + 1);

  // diagonal block of L and its inverse diagonal, for every problem of the CTA
  for (int x = t; x < P * W * W; x += T) {
    const int pp = x / (W * W), jj = (x / W) % W, j = x % W;
    const int bb = pb0 + pp;
    double v = 0.0;
    if (bb < batch && jj < w && j <= jj)
      v = __ldg(L.p + bb * L.stride + pm_off(L.i0 + c0 + jj, L.j0 + c0 + j, L.cn));
    smem[(size_t)pp * RS + jj * (W + 1) + j] = v;
  }
  for (int x = t; x < P * W; x += T) {
    const int pp = x / W, j = x % W;
    const int bb = pb0 + pp;
    double r = 0.0;
    if (bb < batch && j < w) {
      if (dinv)
        r = __ldg(dinv + bb * sdinv + c0 + j);
      else
        r = recip3(__ldg(L.p + bb * L.stride + pm_off(L.i0 + c0 + j, L.j0 + c0 + j, L.cn)));
    }
    smem[(size_t)pp * RS + W * (W + 1) + j] = r;
  }

  // (a)
  double acc[W];
  const double *brow = B.p + (active ? b : 0) * B.stride + pm_off(B.i0 + (active ? row : 0), B.j0, B.cn);
  double *xrow = D.p + (active ? b : 0) * D.stride + pm_off(D.i0 + (active ? row : 0), D.j0, D.cn);
#pragma unroll
  for (int jj = 0; jj < W; jj++) acc[jj] = (active && jj < w) ? brow[(long long)(c0 + jj) * PS] : 0.0;
  if (!is_one(alpha)) {
#pragma unroll
    for (int jj = 0; jj < W; jj++) acc[jj] *= alpha;
  }

  // (b) downdate with the columns already solved
  double *stage = stage_base + (size_t)min(p, P - 1) * KC * SPITCH;
  for (int l0 = 0; l0 < c0; l0 += KC) {
    __syncthreads();
    for (int x = t; x < P * 32 * KC; x += T) {
      const int pp = x / (32 * KC);
      const int y = x - pp * 32 * KC;
      const int r4 = y % PS, ll = (y / PS) % KC, pnl = y / (PS * KC);
      const int jj = pnl * PS + r4;
      const int bb = pb0 + pp;
      stage_base[(size_t)pp * KC * SPITCH + ll * SPITCH + jj] =
          (bb < batch && jj < w) ? __ldg(L.p + bb * L.stride + pm_off(L.i0 + c0 + jj, L.j0 + l0 + ll, L.cn)) : 0.0;
    }
    __syncthreads();
    if (active) {
#pragma unroll 2
      for (int ll = 0; ll < KC; ll++) {
        const double x = xrow[(long long)(l0 + ll) * PS];
#pragma unroll
        for (int jj = 0; jj < W; jj += 2) {
          const double2 lv = *(const double2 *)&stage[ll * SPITCH + jj];
          acc[jj] = fma(-x, lv.x, acc[jj]);
          if (jj + 1 < W) acc[jj + 1] = fma(-x, lv.y, acc[jj + 1]);
        }
      }
    }
  }
  __syncthreads();

  // (d) substitution against the diagonal block
  if (active) {
#pragma unroll
    for (int j = 0; j < W; j++) {
      acc[j] *= rinv[j];
#pragma unroll
      for (int jj = j + 1; jj < W; jj++) acc[jj] = fma(-acc[j], Ls[jj * (W + 1) + j], acc[jj]);
    }
    // (e)
#pragma unroll
    for (int jj = 0; jj < W; jj++)
      if (jj < w) xrow[(long long)(c0 + jj) * PS] = acc[jj];
  }
  __syncthreads();
}

__global__ void __launch_bounds__(MAX_ROWS)
k_trsm_rltn(int batch, int m, int n, double alpha, Op L, const double *dinv, long long sdinv, Op B,
            OpW D, int P, int R, int chunks) {
  extern __shared__ double smem[];
  const int pb0 = (blockIdx.x / chunks) * P;
  const int r0 = (blockIdx.x % chunks) * R;
  for (int c0 = 0; c0 < n; c0 += 32) {
    switch (w_bucket(min(32, n - c0))) {
      case 4: trsm_block<4>(smem, P, R, c0, m, n, alpha, pb0, batch, r0, L, dinv, sdinv, B, D); break;
      case 8: trsm_block<8>(smem, P, R, c0, m, n, alpha, pb0, batch, r0, L, dinv, sdinv, B, D); break;
      case 16: trsm_block<16>(smem, P, R, c0, m, n, alpha, pb0, batch, r0, L, dinv, sdinv, B, D); break;
      case 24: trsm_block<24>(smem, P, R, c0, m, n, alpha, pb0, batch, r0, L, dinv, sdinv, B, D); break;
      default: trsm_block<32>(smem, P, R, c0, m, n, alpha, pb0, batch, r0, L, dinv, sdinv, B, D); break;
    }
  }
}

// n <= 32: a single column block of width bucket W, in a kernel of its own so
// that its register count is that of W (the blocked kernel carries the
// W = 32 path, whose register count would cap the small widths' occupancy).
template <int W>
__global__ void __launch_bounds__(MAX_ROWS)
k_trsm_rltn_w(int batch, int m, int n, double alpha, Op L, const double *dinv, long long sdinv, Op B,
              OpW D, int P, int R, int chunks) {
  extern __shared__ double smem[];
  const int pb0 = (blockIdx.x / chunks) * P;
  const int r0 = (blockIdx.x % chunks) * R;
  trsm_block<W>(smem, P, R, 0, m, n, alpha, pb0, batch, r0, L, dinv, sdinv, B, D);
}

template <int W>
cudaError_t launch_trsm_w(unsigned g, int threads, size_t smem, cudaStream_t s, int batch, int m, int n,
                          double alpha, Op L, const double *dinv, long long sdinv, Op B, OpW D, int P, int R,
                          int chunks) {
  static std::atomic<unsigned long long> attr{0};
  cudaError_t e = smem_attr_once((const void *)k_trsm_rltn_w<W>, 200 * 1024, attr);
  if (e != cudaSuccess) return e;
  k_trsm_rltn_w<W><<<g, threads, smem, s>>>(batch, m, n, alpha, L, dinv, sdinv, B, D, P, R, chunks);
  return cudaGetLastError();
}

// Descriptor-array form: CTA = (problem, chunk of MAX_ROWS rows of X), one
// problem per CTA, after checking the problem's record.
__global__ void __launch_bounds__(MAX_ROWS)
k_trsm_rltn_v(int batch, const bf_dsize *size, double alpha, const bf_dsub *Ls, int use_dinv, const bf_dsub *Bs,
              const bf_dsub *Ds, int chunks, int max_m, int max_n, int *status) {
  extern __shared__ double smem[];
  const int b = blockIdx.x / chunks, chunk = blockIdx.x - b * chunks;
  if (b >= batch) return;
  const int m = size[b].m, n = size[b].n;
  int err = 0;
  if (m < 0 || n < 0 || m > max_m || n > max_n)
    err = -1;
  else if (m > 0 && n > 0) {
    if (!dsub_ok(Ls[b], n, n))
      err = -2;
    else if (!dsub_ok(Bs[b], m, n))
      err = -3;
    else if (!dsub_ok(Ds[b], m, n))
      err = -4;
  }
  if (chunk == 0 && threadIdx.x == 0 && status) status[b] = err;
  const int R = blockDim.x, r0 = chunk * R;
  if (err != 0 || m == 0 || n == 0 || r0 >= m) return;
  const Op L = dsub_op(Ls[b]), B = dsub_op(Bs[b]);
  const OpW D = dsub_opw(Ds[b]);
  // the inverse-diagonal array holds min(m, n) entries of its matrix; outside
  // it the reciprocals are formed here
  const bf_dmat &lm = Ls[b].mat;
  const double *dinv = (use_dinv && lm.dA && Ls[b].j + n <= min(lm.m, lm.n)) ? lm.dA + Ls[b].j : nullptr;
  for (int c0 = 0; c0 < n; c0 += 32) {
    switch (w_bucket(min(32, n - c0))) {
      case 4: trsm_block<4>(smem, 1, R, c0, m, n, alpha, 0, 1, r0, L, dinv, 0, B, D); break;
      case 8: trsm_block<8>(smem, 1, R, c0, m, n, alpha, 0, 1, r0, L, dinv, 0, B, D); break;
      case 16: trsm_block<16>(smem, 1, R, c0, m, n, alpha, 0, 1, r0, L, dinv, 0, B, D); break;
      case 24: trsm_block<24>(smem, 1, R, c0, m, n, alpha, 0, 1, r0, L, dinv, 0, B, D); break;
      default: trsm_block<32>(smem, 1, R, c0, m, n, alpha, 0, 1, r0, L, dinv, 0, B, D); break;
    }
  }
}

}  // namespace

cudaError_t launch_trsm_rltn_v(int batch, const bf_dsize *size, double alpha, const bf_dsub *L, bool use_dinv,
                               const bf_dsub *B, const bf_dsub *D, int max_m, int max_n, int *status,
                               cudaStream_t s) {
  const int R = min(MAX_ROWS, ((max_m + 31) / 32) * 32);
  const int chunks = max(1, (max_m + R - 1) / R);
  const int W = w_bucket(min(max(max_n, 1), 32));
  size_t smem = ((size_t)ls_region(W) + 1) * sizeof(double);
  if (max_n > 32) smem += (size_t)KC * SPITCH * sizeof(double);
  static std::atomic<unsigned long long> attr{0};
  cudaError_t e = smem_attr_once((const void *)k_trsm_rltn_v, 200 * 1024, attr);
  if (e != cudaSuccess) return e;
  const long long blocks = (long long)batch * chunks;
  if (blocks > 0x7fffffffLL || R == 0) return cudaErrorInvalidConfiguration;
  k_trsm_rltn_v<<<(unsigned)blocks, R, smem, s>>>(batch, size, alpha, L, use_dinv ? 1 : 0, B, D, chunks, max_m,
                                                  max_n, status);
  return cudaGetLastError();
}

// The latency kernel (R lanes per row) where one thread per row would
// leave SM sub-partitions idle: at most BF_TRSM_LAT_ROWS_PER_SM rows of X
// per SM over the batch, eight lanes per row for orders above 20 with at
// most a quarter of that.  Measured single launches (n = 8..32, batch
// 64..2048): four lanes per row fastest up to 512 x 24 rows, eight lanes at
// n = 32 with 64 or 128 problems (10.1 against 14.3 us at 64).  In a CUDA
// graph, 128 problems of order 24: eight lanes 5.0, five lanes (six rows a
// warp) 5.05-5.27, four lanes 5.7 us per launch.
#ifndef BF_TRSM_LAT_ROWS_PER_SM
#define BF_TRSM_LAT_ROWS_PER_SM 128
#endif
int trsm_layout_rule(int batch, int m, int n) {
  const long long rows = (long long)batch * m, cap = (long long)BF_TRSM_LAT_ROWS_PER_SM * device_sm_count();
  if (n <= 32 && n > 20 && rows * 4 <= cap) return LAYOUT_TRSM_LAT8;
  if (n <= 32 && rows <= cap) return LAYOUT_TRSM_LAT4;
  return LAYOUT_TRSM_ROWS;
}

bool trsm_layout_ok(int layout, int n) {
  if (layout == LAYOUT_TRSM_ROWS) return n <= TRSM_MAX_N;
  return layout > LAYOUT_TRSM_ROWS && layout < LAYOUT_TRSM_COUNT && n <= 32;
}

cudaError_t launch_trsm_rltn(int batch, int m, int n, double alpha, Op L, const double *dinv,
                             long long sdinv, Op B, OpW D, cudaStream_t s) {
  int lay = layout_forced(ROUTINE_TRSM_RLTN, n, batch);
  if (lay <= 0) lay = trsm_layout_rule(batch, m, n);
  if (lay == LAYOUT_TRSM_LAT2 || lay == LAYOUT_TRSM_LAT4 || lay == LAYOUT_TRSM_LAT8)
    return launch_trsm_lat(lay == LAYOUT_TRSM_LAT2 ? 2 : (lay == LAYOUT_TRSM_LAT4 ? 4 : 8), batch, m, n, alpha, L,
                           dinv, sdinv, B, D, s);
  int P = 1, R = m, chunks = 1;
  if (m > CHUNK_ROWS) {
    chunks = (m + CHUNK_ROWS - 1) / CHUNK_ROWS;
    R = ((m + chunks - 1) / chunks + 31) / 32 * 32;  // even chunks, whole warps
  } else if (n <= 32) {
    // a single column block: pack as many problems as fit in 256 rows
    P = max(1, BF_TRSM_PACK_ROWS / m);
  } else {
    // blocked: up to 4 problems, enough to fill whole warps
    while (P < 4 && 2 * P * m <= MAX_ROWS && (P * m) % 32 != 0) P *= 2;
  }
  const int W = w_bucket(min(n, 32));
  const size_t per_problem = ((size_t)ls_region(W) + (n > 32 ? (size_t)KC * SPITCH : 0)) * sizeof(double);
  P = (int)min((size_t)P, (size_t)(96 * 1024) / per_problem);
  P = max(1, min(P, batch));
  // Small batches: if the CTAs would not cover the SMs, keep each CTA within
  // 4 warps so that no SM sub-partition serializes two warps' substitutions.
  if ((batch + P - 1) / P < device_sm_count() && P * R > 128) P = max(1, 128 / R);
  const int threads = ((P * R + 31) / 32) * 32;
  size_t smem = ((size_t)P * ls_region(W) + 1) * sizeof(double);
  if (n > 32) smem += (size_t)P * KC * SPITCH * sizeof(double);
  if (smem > 200 * 1024) return cudaErrorInvalidConfiguration;
  static std::atomic<unsigned long long> attr{0};
  cudaError_t e = smem_attr_once((const void *)k_trsm_rltn, 200 * 1024, attr);
  if (e != cudaSuccess) return e;
  const long long blocks = (long long)((batch + P - 1) / P) * chunks;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const unsigned g = (unsigned)blocks;
  if (n <= 32) {
    switch (W) {
      case 4: return launch_trsm_w<4>(g, threads, smem, s, batch, m, n, alpha, L, dinv, sdinv, B, D, P, R, chunks);
      case 8: return launch_trsm_w<8>(g, threads, smem, s, batch, m, n, alpha, L, dinv, sdinv, B, D, P, R, chunks);
      case 16: return launch_trsm_w<16>(g, threads, smem, s, batch, m, n, alpha, L, dinv, sdinv, B, D, P, R, chunks);
      case 24: return launch_trsm_w<24>(g, threads, smem, s, batch, m, n, alpha, L, dinv, sdinv, B, D, P, R, chunks);
      default: return launch_trsm_w<32>(g, threads, smem, s, batch, m, n, alpha, L, dinv, sdinv, B, D, P, R, chunks);
    }
  }
  k_trsm_rltn<<<g, threads, smem, s>>>(batch, m, n, alpha, L, dinv, sdinv, B, D, P, R, chunks);
  return cudaGetLastError();
}

}  // namespace bf
