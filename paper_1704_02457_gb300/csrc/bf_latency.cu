// Latency kernels for small batches of small problems (order <= 32):
// potrf_l / syrk_potrf_ln (k_chol_lat) and trsm_rltn (k_trsm_lat).
//
// The throughput kernels put several problems on a warp so that the
// sequential part of a factorization (a reciprocal and a square root per
// column) is shared.  With few problems that leaves most of the GPU idle and
// each warp with a long chain of FP64 instructions: on GB300 one warp-wide
// FP64 instruction occupies its SM sub-partition's FP64 pipe for the same
// time with 1 or 32 active lanes, so what bounds a small batch is the count
// of FP64 warp instructions on the busiest sub-partition.  These kernels
// spread one problem over the four sub-partitions of an SM instead.
//
// k_chol_lat: one problem per CTA of 4 warps.  The lower triangle of
//   C (+ A B^T, the fused update of Sec. 4.7.2, formed in shared memory and
//   never stored) sits in shared memory.  The factorization is the
//   right-looking square-root-free form: for column j, with d = S[j][j],
//       S[i][m] -= S[i][j] * (1/d) * S[m][j]      (j < m <= i < n)
//   so the chain from one pivot to the next holds one reciprocal (the
//   hardware approximation refined by one third-order step) and two FMAs;
//   the trailing elements are spread over the 128 threads in each step.
//   After the last step column j holds L[:, j] * sqrt(d_j), and
//   L[i][j] = S[i][j] * rsqrt(d_j) for all columns at once (Sec. 4.7.1:
//   rsqrt(d_j) is the inverse diagonal).  info = j+1 for the first pivot that
//   is not > 0, as in the other kernels.
//
// k_trsm_lat: X L^T = alpha B row by row (rows are independent), R lanes
//   per row.  Lane q of a row keeps the columns c = q (mod R) of its
//   right-hand side in registers; for column j the owner lane forms
//   X[i][j] = t_j / L[j][j] (times the inverse diagonal), hands it to the
//   row's other lanes with a shuffle, and each lane downdates its own later
//   columns: the substitution merged with the downdate (Sec. 4.6), with the
//   downdate of a row split over R lanes.
#include "bf_internal.cuh"

namespace bf {
namespace {

constexpr int LAT_T = 128;  // threads of both kernels
constexpr int LAT_N = 32;   // largest order
constexpr int LP = LAT_N + 1;

__device__ __forceinline__ const double *elem(const Op &o, int b, int r, int c) {
  return o.p + (long long)b * o.stride + pm_off(o.i0 + r, o.j0 + c, o.cn);
}
__device__ __forceinline__ double *elem(const OpW &o, int b, int r, int c) {
  return o.p + (long long)b * o.stride + pm_off(o.i0 + r, o.j0 + c, o.cn);
}

// 1/d: the hardware approximation r0 (relative error e = 1 - d r0 below
// 2^-22), then r0 (1 + e + e^2), whose error is of order e^3.
__device__ __forceinline__ double recip3(double d) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
  const double e = fma(-d, r, 1.0);
  return fma(fma(e, e, e), r, r);
}

// Columns of A and B staged per pass of the fused update.
constexpr int LAT_KC = 32;
constexpr int LKP = LAT_KC + 1;
// Off-diagonal elements go to the first three warps, the diagonal to the last.
constexpr int LAT_OFF = LAT_T - 32;
constexpr int LAT_RO = (LAT_N * (LAT_N - 1) / 2 + LAT_OFF - 1) / LAT_OFF;

// Row and column of entry e of the strictly lower triangle listed column by
// column from the last column back, e = t (t + 1) / 2 + o with o <= t:
// column n - 2 - t, row n - 1 - t + o.  The trailing part of step j (columns
// j+1 and later) is then the first (n-j-1)(n-j-2)/2 entries.
__device__ __forceinline__ void off_entry(int e, int n, int &i, int &m) {
  int t = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  if (t * (t + 1) / 2 > e) t--;
  if ((t + 1) * (t + 2) / 2 <= e) t++;
  m = n - 2 - t;
  i = m + 1 + (e - t * (t + 1) / 2);
}

template <bool FUSED>
__global__ void __launch_bounds__(LAT_T)
k_chol_lat(int n, int k, Op A, Op B, Op C, OpW D, double *dinv, long long sdinv, int *info) {
  __shared__ double S[LAT_N * LP];
  __shared__ double AB[FUSED ? 2 * LAT_N * LKP : 1];  // rows of A, then rows of B
  __shared__ double colb[2][LAT_N];                    // the current column, double buffered
  __shared__ double iv[LAT_N];                         // 1 / d_j
  __shared__ double rs[LAT_N];                         // rsqrt(d_j)
  const int b = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool diag_warp = warp == LAT_T / 32 - 1;
  const int nod = n * (n - 1) / 2;

  // C's lower triangle (a warp per column, a lane per row) and the first
  // columns of A and B, asynchronously
  for (int j = warp; j < n; j += LAT_T / 32)
    if (lane < n && lane >= j) cp_async8(&S[lane * LP + j], elem(C, b, lane, j));
  auto stage = [&](int l0, int kc) {
    for (int l = warp; l < kc; l += LAT_T / 32)
      if (lane < n) {
        cp_async8(&AB[lane * LKP + l], elem(A, b, lane, l0 + l));
        cp_async8(&AB[(LAT_N + lane) * LKP + l], elem(B, b, lane, l0 + l));
      }
  };
  if (FUSED && k > 0) stage(0, min(LAT_KC, k));

  // The elements each thread owns for the whole factorization, in
  // registers: the first three warps the strictly lower triangle (entry
  // tid + 96 r), the last warp the diagonal (lane m owns (m, m)).
  int ei[LAT_RO], em[LAT_RO];
  double v[LAT_RO];
  double dg = 0.0;
  if (!diag_warp) {
#pragma unroll
    for (int r = 0; r < LAT_RO; r++) {
      const int e = tid + LAT_OFF * r;
      ei[r] = em[r] = 0;
      if (e < nod) off_entry(e, n, ei[r], em[r]);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  if (!diag_warp) {
#pragma unroll
    for (int r = 0; r < LAT_RO; r++) v[r] = (tid + LAT_OFF * r < nod) ? S[ei[r] * LP + em[r]] : 0.0;
  } else if (lane < n) {
    dg = S[lane * LP + lane];
  }

  if (FUSED && k > 0) {
    // + A B^T on the owned elements (the fused update of Sec. 4.7.2)
    for (int l0 = 0; l0 < k; l0 += LAT_KC) {
      const int kc = min(LAT_KC, k - l0);
      if (l0 > 0) {
        __syncthreads();  // everyone is done with the previous columns
        stage(l0, kc);
        cp_async_wait_all();
        __syncthreads();
      }
      if (!diag_warp) {
#pragma unroll
        for (int r = 0; r < LAT_RO; r++) {
          if (tid + LAT_OFF * r < nod) {
            const double *ar = AB + ei[r] * LKP, *br = AB + (LAT_N + em[r]) * LKP;
            double acc = v[r];
            for (int l = 0; l < kc; l++) acc = fma(ar[l], br[l], acc);
            v[r] = acc;
          }
        }
      } else if (lane < n) {
        const double *ar = AB + lane * LKP, *br = AB + (LAT_N + lane) * LKP;
        double acc = dg;
        for (int l = 0; l < kc; l++) acc = fma(ar[l], br[l], acc);
        dg = acc;
      }
    }
  }

  // column 0, and 1 / d_0
  if (!diag_warp) {
#pragma unroll
    for (int r = 0; r < LAT_RO; r++)
      if (tid + LAT_OFF * r < nod && em[r] == 0) colb[0][ei[r]] = v[r];
  } else if (lane == 0) {
    colb[0][0] = dg;
    iv[0] = recip3(dg);
  }
  __syncthreads();

  // Right-looking, square-root free.  Step j: every owned element (i, m),
  // j < m <= i, takes S[i][m] -= S[i][j] (1/d_j) S[m][j], with column j read
  // from colb; the owners of column j+1 publish it.  The diagonal lanes use
  // S[m][m] -= S[m][j]^2 / d_j, and lane j+1, whose pivot is then final,
  // forms 1/d_{j+1} for the next step: the chain from pivot to pivot is two
  // FMAs and one reciprocal, with one barrier per column.
  for (int j = 0; j + 1 < n; j++) {
    const double invd = iv[j];
    const double *cj = colb[j & 1];
    double *cn = colb[(j + 1) & 1];
    if (diag_warp) {
      if (lane > j && lane < n) {
        const double x = cj[lane];
        dg = fma(-(x * x), invd, dg);
        if (lane == j + 1) {
          cn[lane] = dg;
          iv[lane] = recip3(dg);
        }
      }
    } else {
      const int c = (n - j - 1) * (n - j - 2) / 2;
#pragma unroll
      for (int r = 0; r < LAT_RO; r++) {
        if (tid + LAT_OFF * r < c) {
          v[r] = fma(-(cj[ei[r]] * invd), cj[em[r]], v[r]);
          if (em[r] == j + 1) cn[ei[r]] = v[r];
        }
      }
    }
    __syncthreads();
  }

  // L[i][m] = S[i][m] rsqrt(d_m); dinv = rsqrt(d_m); info = 1 + the first
  // pivot that is not > 0
  if (diag_warp) {
    const double r = lane < n ? rsqrt(dg) : 0.0;
    if (lane < n) {
      rs[lane] = r;
      *elem(D, b, lane, lane) = dg * r;
      if (dinv) dinv[(long long)b * sdinv + lane] = r;
    }
    const unsigned badm = __ballot_sync(0xffffffffu, lane < n && !(dg > 0.0));
    if (lane == 0 && info) info[b] = badm ? __ffs(badm) : 0;
  }
  __syncthreads();
  if (!diag_warp) {
#pragma unroll
    for (int r = 0; r < LAT_RO; r++)
      if (tid + LAT_OFF * r < nod) *elem(D, b, ei[r], em[r]) = v[r] * rs[em[r]];
  }
}

// NB: the order rounded up to the instantiated width; R lanes per row.
template <int NB, int R>
__global__ void __launch_bounds__(LAT_T)
k_trsm_lat(int m, int n, double alpha, Op L, const double *dinv, long long sdinv, Op B, OpW D, int chunks) {
  constexpr int S = NB / R;          // column slots per lane
  constexpr int ROWS = LAT_T / R;    // rows per CTA
  constexpr int PITCH = NB + 1;
  __shared__ double Ls[NB * PITCH];
  __shared__ double dv[NB];
  const int b = blockIdx.x / chunks;
  const int row0 = (blockIdx.x % chunks) * ROWS;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // L's lower triangle (a warp per column, a lane per row) and the inverse
  // diagonal go to shared memory asynchronously while the rows of B load
  for (int j = warp; j < n; j += LAT_T / 32)
    if (lane < n && lane >= j) cp_async8(&Ls[lane * PITCH + j], elem(L, b, lane, j));
  if (dinv)
    for (int j = tid; j < n; j += LAT_T) cp_async8(&dv[j], dinv + (long long)b * sdinv + j);
  // a warp whose rows all lie past m only helps with the loads
  const bool warp_rows = row0 + (tid & ~31) / R < m;
  const int q = tid % R;
  const int row = row0 + tid / R;
  const bool active = row < m;
  double t[S];
#pragma unroll
  for (int s = 0; s < S; s++) {
    const int c = q + R * s;
    t[s] = (active && c < n) ? alpha * *elem(B, b, row, c) : 0.0;
  }
  cp_async_wait_all();
  __syncthreads();
  if (!dinv) {
    for (int j = tid; j < n; j += LAT_T) dv[j] = recip3(Ls[j * PITCH + j]);
    __syncthreads();
  }
  if (!warp_rows) return;

  const int base = lane & ~(R - 1);
#pragma unroll
  for (int j = 0; j < NB; j++) {
    if (j >= n) break;
    const double xo = t[j / R] * dv[j];
    const double x = __shfl_sync(0xffffffffu, xo, base + j % R);
    if (active && q == j % R) *elem(D, b, row, j) = x;
#pragma unroll
    for (int s = (j + 1) / R; s < S; s++) {
      const int c = q + R * s;
      if (c > j && c < n) t[s] = fma(-x, Ls[c * PITCH + j], t[s]);
    }
  }
}

template <int NB, int R>
cudaError_t launch_trsm_lat_nb(int batch, int m, int n, double alpha, Op L, const double *dinv, long long sdinv,
                               Op B, OpW D, cudaStream_t s) {
  constexpr int ROWS = LAT_T / R;
  const int chunks = (m + ROWS - 1) / ROWS;
  const long long blocks = (long long)batch * chunks;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  k_trsm_lat<NB, R><<<(unsigned)blocks, LAT_T, 0, s>>>(m, n, alpha, L, dinv, sdinv, B, D, chunks);
  return cudaGetLastError();
}

template <int R>
cudaError_t launch_trsm_lat_r(int batch, int m, int n, double alpha, Op L, const double *dinv, long long sdinv,
                              Op B, OpW D, cudaStream_t s) {
  if (n <= 8) return launch_trsm_lat_nb<8, R>(batch, m, n, alpha, L, dinv, sdinv, B, D, s);
  if (n <= 16) return launch_trsm_lat_nb<16, R>(batch, m, n, alpha, L, dinv, sdinv, B, D, s);
  if (n <= 24) return launch_trsm_lat_nb<24, R>(batch, m, n, alpha, L, dinv, sdinv, B, D, s);
  return launch_trsm_lat_nb<32, R>(batch, m, n, alpha, L, dinv, sdinv, B, D, s);
}

}  // namespace

constexpr int CHOL_LAT_MAX_N = LAT_N;

cudaError_t launch_chol_lat(bool fused, int batch, int n, int k, Op A, Op B, Op C, OpW D, double *dinv,
                            long long sdinv, int *info, cudaStream_t s) {
  if (n > CHOL_LAT_MAX_N) return cudaErrorInvalidValue;
  if (fused)
    k_chol_lat<true><<<(unsigned)batch, LAT_T, 0, s>>>(n, k, A, B, C, D, dinv, sdinv, info);
  else
    k_chol_lat<false><<<(unsigned)batch, LAT_T, 0, s>>>(n, k, A, B, C, D, dinv, sdinv, info);
  return cudaGetLastError();
}

cudaError_t launch_trsm_lat(int lanes, int batch, int m, int n, double alpha, Op L, const double *dinv,
                            long long sdinv, Op B, OpW D, cudaStream_t s) {
  if (n > LAT_N) return cudaErrorInvalidValue;
  switch (lanes) {
    case 2: return launch_trsm_lat_r<2>(batch, m, n, alpha, L, dinv, sdinv, B, D, s);
    case 8: return launch_trsm_lat_r<8>(batch, m, n, alpha, L, dinv, sdinv, B, D, s);
    default: return launch_trsm_lat_r<4>(batch, m, n, alpha, L, dinv, sdinv, B, D, s);
  }
}

}  // namespace bf
