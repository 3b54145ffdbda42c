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
#include <type_traits>

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


// 1 when x is not zero and its magnitude lies outside 2^-480 .. 2^480
// (subnormal, inf and NaN included), from the exponent field.
__device__ __forceinline__ int far_from_one(double x) {
  const int hi = __double2hiint(x), lo = __double2loint(x);
  const int e = (hi >> 20) & 0x7ff;
  return (((hi & 0x7fffffff) | lo) != 0) && (e < 1023 - 480 || e > 1023 + 480);
}

// Columns of A and B staged per pass of the fused update.
constexpr int LAT_KC = 32;
constexpr int LKP = LAT_KC + 1;
// Off-diagonal elements go to the first three warps, the diagonal to the last.
constexpr int LAT_OFF = LAT_T - 32;

// t and o with e = t (t + 1) / 2 + o, 0 <= o <= t, for e < 528 (t < 32),
// as a table in global memory: (t << 8) | o at entry e.  A load of it
// overlaps the operand loads, where computing t from a square root cost more
// than a microsecond of dependent integer work per CTA.
struct TriTable {
  unsigned short v[LAT_N * (LAT_N + 1) / 2];
  constexpr TriTable() : v() {
    int e = 0;
    for (int t = 0; t < LAT_N; t++)
      for (int o = 0; o <= t; o++) v[e++] = (unsigned short)((t << 8) | o);
  }
};
__device__ constexpr TriTable g_tri{};

__device__ __forceinline__ void tri_split(int e, int &t, int &o) {
  const unsigned x = __ldg(&g_tri.v[e]);
  t = (int)(x >> 8);
  o = (int)(x & 255u);
}

// Row and column of entry e of the strictly lower triangle listed column by
// column from the last column back: e = t (t + 1) / 2 + o, column n - 2 - t,
// row n - 1 - t + o.  The trailing part of step j (columns j+1 and later) is
// then the first (n-j-1)(n-j-2)/2 entries.
__device__ __forceinline__ void off_entry(int e, int n, int &i, int &m) {
  int t, o;
  tri_split(e, t, o);
  m = n - 2 - t;
  i = m + 1 + o;
}

// Address of row r, column 0 of problem b's operand (column c is 4 c further:
// the panel-major column stride, Sec. 4.3.3)
__device__ __forceinline__ const double *row_base(const Op &o, int b, int r) {
  return o.p + (long long)b * o.stride + pm_off(o.i0 + r, o.j0, o.cn);
}

// NB: the order rounded up to the instantiated width (8, 16, 24 or 32), which
// sizes the per-thread slot arrays.
template <bool FUSED, int NB>
__global__ void __launch_bounds__(LAT_T)
k_chol_lat(int n, int k, Op A, Op B, Op C, OpW D, double *dinv, long long sdinv, int *info) {
  // owned off-diagonal elements and fused-update items per thread
  constexpr int RO = (NB * (NB - 1) / 2 + LAT_OFF - 1) / LAT_OFF;
  constexpr int RQ = (NB * (NB + 1) + LAT_T - 1) / LAT_T;
  __shared__ double S[LAT_N * LP];
  __shared__ double AB[FUSED ? 2 * LAT_N * LKP : 1];      // rows of A, then rows of B
  __shared__ double part[FUSED ? LAT_N * (LAT_N + 1) : 1];  // sums of the fused update's items
  __shared__ double colb[2][LAT_N];                         // the current column, double buffered
  __shared__ double iv[LAT_N];                              // 1 / d_j
  __shared__ double rs[LAT_N];                              // rsqrt(d_j)
  const int b = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool diag_warp = warp == LAT_T / 32 - 1;
  const int nod = n * (n - 1) / 2;
  const int ne = n * (n + 1) / 2;

  // C's lower triangle (a warp per column, a lane per row) and the first
  // columns of A and B, asynchronously
  const double *crow = lane < n ? row_base(C, b, lane) : nullptr;
  const double *arow = FUSED && lane < n && k > 0 ? row_base(A, b, lane) : nullptr;
  const double *brow = FUSED && lane < n && k > 0 ? row_base(B, b, lane) : nullptr;
  pdl_wait();  // launched as a programmatic dependent: the previous kernel's writes first
  for (int j = warp; j < n; j += LAT_T / 32)
    if (lane < n && lane >= j) cp_async8(&S[lane * LP + j], crow + PS * j);
  auto stage = [&](int l0, int kc) {
    if (lane < n)
      for (int l = warp; l < kc; l += LAT_T / 32) {
        cp_async8(&AB[lane * LKP + l], arow + PS * (l0 + l));
        cp_async8(&AB[(LAT_N + lane) * LKP + l], brow + PS * (l0 + l));
      }
  };
  if (FUSED && k > 0) stage(0, min(LAT_KC, k));

  // The fused update's items: an element (row-major order of the lower
  // triangle) or, when that evens out the work of the threads, half of its
  // k-range; thread t takes items t + 128 r.
  const int sp = (FUSED && k > 0 && k <= LAT_KC &&
                  ((ne * 2 + LAT_T - 1) / LAT_T) * ((k + 1) / 2) < ((ne + LAT_T - 1) / LAT_T) * k) ? 2 : 1;
  const int nq = ne * sp;
  int qi[RQ], qm[RQ], qh[RQ];
  if (FUSED && k > 0) {
#pragma unroll
    for (int r = 0; r < RQ; r++) {
      const int q = tid + LAT_T * r;
      qi[r] = qm[r] = qh[r] = 0;
      if (q < nq) {
        tri_split(sp == 2 ? q >> 1 : q, qi[r], qm[r]);
        qh[r] = sp == 2 ? (q & 1) : 0;
      }
    }
  }

  // The elements each thread owns for the whole factorization, in
  // registers: the first three warps the strictly lower triangle (entry
  // tid + 96 r), the last warp the diagonal (lane m owns (m, m)).
  int ei[RO], em[RO];
  double v[RO];
  double dg = 0.0;
  if (!diag_warp) {
#pragma unroll
    for (int r = 0; r < RO; r++) {
      const int e = tid + LAT_OFF * r;
      ei[r] = em[r] = 0;
      if (e < nod) off_entry(e, n, ei[r], em[r]);
    }
  }
  cp_async_wait_all();
  __syncthreads();

  if (FUSED && k > 0) {
    // + A B^T (the fused update of Sec. 4.7.2), items interleaved so that
    // each thread runs up to RQ independent chains of FMAs
    double acc[RQ];
#pragma unroll
    for (int r = 0; r < RQ; r++) acc[r] = 0.0;
    for (int l0 = 0; l0 < k; l0 += LAT_KC) {
      const int kc = min(LAT_KC, k - l0);
      if (l0 > 0) {
        __syncthreads();  // everyone is done with the previous columns
        stage(l0, kc);
        cp_async_wait_all();
        __syncthreads();
      }
      const int kh = (kc + sp - 1) / sp;
      int len[RQ];
      const double *pa[RQ], *pb[RQ];
#pragma unroll
      for (int r = 0; r < RQ; r++) {
        const int lo = qh[r] * kh;
        len[r] = tid + LAT_T * r < nq ? min(kh, kc - lo) : 0;
        pa[r] = AB + qi[r] * LKP + lo;
        pb[r] = AB + (LAT_N + qm[r]) * LKP + lo;
      }
      for (int l = 0; l < kh; l++) {
#pragma unroll
        for (int r = 0; r < RQ; r++)
          if (l < len[r]) acc[r] = fma(pa[r][l], pb[r][l], acc[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < RQ; r++)
      if (tid + LAT_T * r < nq) part[tid + LAT_T * r] = acc[r];
    __syncthreads();
  }

  // owned values: C, plus the item sums in order
  auto start_value = [&](int i, int m) {
    double x = S[i * LP + m];
    if (FUSED && k > 0) {
      const int e = i * (i + 1) / 2 + m;
      x += part[e * sp];
      if (sp == 2) x += part[e * sp + 1];
    }
    return x;
  };
  if (!diag_warp) {
#pragma unroll
    for (int r = 0; r < RO; r++) v[r] = (tid + LAT_OFF * r < nod) ? start_value(ei[r], em[r]) : 0.0;
  } else if (lane < n) {
    dg = start_value(lane, lane);
  }

  // column 0, and 1 / d_0; whether any entry lies outside 2^-480 .. 2^480
  // in magnitude (zeros aside), where the square of an entry could leave the
  // normal range
  int far = 0;
  if (!diag_warp) {
#pragma unroll
    for (int r = 0; r < RO; r++)
      if (tid + LAT_OFF * r < nod) {
        far |= far_from_one(v[r]);
        if (em[r] == 0) colb[0][ei[r]] = v[r];
      }
  } else if (lane < n) {
    far = far_from_one(dg);
    if (lane == 0) iv[0] = recip3(dg);
  }
  const bool wide = __syncthreads_or(far) != 0;

  // Right-looking, square-root free.  Step j: every owned element (i, m),
  // j < m <= i, takes S[i][m] -= S[i][j] (1/d_j) S[m][j], with column j read
  // from colb; the owners of column j+1 publish it.  The diagonal lanes take
  // S[m][m] -= S[m][j]^2 (1/d_j), and lane j+1, whose pivot is then final,
  // forms 1/d_{j+1} for the next step: the chain from pivot to pivot is two
  // FP64 operations and one reciprocal, with one barrier per column.  The
  // square S[m][j]^2 is formed before the pivot's reciprocal arrives; a
  // problem with entries far from unit size (wide) takes
  // (S[m][j] (1/d_j)) S[m][j] instead, which stays in range as the plain
  // form's other updates do, at one more FP64 operation on the chain.
  auto steps = [&](auto wide_tag) {
    constexpr bool WIDE = decltype(wide_tag)::value;
    for (int j = 0; j + 1 < n; j++) {
      const double invd = iv[j];
      const double *cj = colb[j & 1];
      double *cn = colb[(j + 1) & 1];
      if (diag_warp) {
        if (lane > j && lane < n) {
          const double x = cj[lane];
          dg = WIDE ? fma(-(x * invd), x, dg) : fma(-(x * x), invd, dg);
          if (lane == j + 1) iv[lane] = recip3(dg);
        }
      } else {
        const int c = (n - j - 1) * (n - j - 2) / 2;
#pragma unroll
        for (int r = 0; r < RO; r++) {
          if (tid + LAT_OFF * r < c) {
            v[r] = fma(-(cj[ei[r]] * invd), cj[em[r]], v[r]);
            if (em[r] == j + 1) cn[ei[r]] = v[r];
          }
        }
      }
      __syncthreads();
    }
  };
  if (wide)
    steps(std::true_type{});
  else
    steps(std::false_type{});

  // L[i][m] = S[i][m] rsqrt(d_m); dinv = rsqrt(d_m); info = 1 + the first
  // pivot that is not > 0
  if (diag_warp) {
    const double r = lane < n ? rsqrt(dg) : 0.0;
    if (lane < n) {
      rs[lane] = r;
      *elem(D, b, lane, lane) = dg * r;
      if (dinv) dinv[(long long)b * sdinv + lane] = r;
    }
    const unsigned badm = __ballot_sync(0xffffffffu, lane < n && not_positive(dg));
    if (lane == 0 && info) info[b] = badm ? __ffs(badm) : 0;
  }
  __syncthreads();
  if (!diag_warp) {
#pragma unroll
    for (int r = 0; r < RO; r++)
      if (tid + LAT_OFF * r < nod) *elem(D, b, ei[r], em[r]) = v[r] * rs[em[r]];
  }
  pdl_allow();  // the next kernel may be scheduled once every CTA is here
}

// NB: the order rounded up to the instantiated width; R lanes per row, a
// warp holding 32/R rows.
// The columns of L below the diagonal are scaled by the inverse diagonal in
// shared memory, L'[c][j] = L[c][j] / L[j][j], so that a lane carries the
// unscaled t_j = (B - sum_{l<j} X_l L^T_l)_j, the downdate reads
// t_c -= t_j L'[c][j], and X_j = alpha t_j / L[j][j] is formed once at the
// end (alpha folded into the inverse diagonal: one product per column of L
// instead of one per element of B): the chain from one column to the next
// is one shuffle and one FMA.
template <int NB, int R>
__global__ void __launch_bounds__(LAT_T)
k_trsm_lat(int m, int n, double alpha, Op L, const double *dinv, long long sdinv, Op B, OpW D, int chunks) {
  constexpr int S = (NB + R - 1) / R;     // column slots per lane
  constexpr int RPW = 32 / R;             // rows per warp
  constexpr int ROWS = (LAT_T / 32) * RPW;  // rows per CTA
  constexpr int PITCH = NB + 1;
  constexpr int NT = (NB * (NB - 1) / 2 + LAT_T - 1) / LAT_T;  // strictly lower entries per thread
  __shared__ double Ls[NB * PITCH];
  __shared__ double dv[NB], adv[NB];
  const int b = blockIdx.x / chunks;
  const int row0 = (blockIdx.x % chunks) * ROWS;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nod = n * (n - 1) / 2;
  // the strictly lower entries this thread scales (a constant table, read
  // before the wait for the previous kernel)
  int si[NT], sj[NT];
#pragma unroll
  for (int r = 0; r < NT; r++) {
    si[r] = sj[r] = 0;
    if (tid + LAT_T * r < nod) off_entry(tid + LAT_T * r, n, si[r], sj[r]);
  }
  // L's lower triangle (a warp per column, a lane per row) and the inverse
  // diagonal go to shared memory asynchronously while the rows of B load
  const double *lrow = lane < n ? row_base(L, b, lane) : nullptr;
  pdl_wait();  // launched as a programmatic dependent: the previous kernel's writes first
  for (int j = warp; j < n; j += LAT_T / 32)
    if (lane < n && lane >= j) cp_async8(&Ls[lane * PITCH + j], lrow + PS * j);
  if (dinv)
    for (int j = tid; j < n; j += LAT_T) cp_async8(&dv[j], dinv + (long long)b * sdinv + j);
  const int q = lane % R, rw = lane / R;
  const int row = row0 + warp * RPW + rw;
  // a warp whose rows all lie past m only helps with the set-up
  const bool warp_rows = row0 + warp * RPW < m;
  const bool active = rw < RPW && row < m;
  double t[S];
  {
    const double *brow = active ? row_base(B, b, row) : nullptr;
#pragma unroll
    for (int s = 0; s < S; s++) {
      const int c = q + R * s;
      t[s] = (active && c < n) ? brow[PS * c] : 0.0;
    }
  }
  cp_async_wait_all();
  __syncthreads();
  if (!dinv) {
    for (int j = tid; j < n; j += LAT_T) dv[j] = recip3(Ls[j * PITCH + j]);
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < NT; r++)
    if (tid + LAT_T * r < nod) Ls[si[r] * PITCH + sj[r]] *= dv[sj[r]];
  if (tid < n) adv[tid] = alpha * dv[tid];
  __syncthreads();
  if (!warp_rows) return;

  const int base = lane - q;
#pragma unroll
  for (int j = 0; j < NB; j++) {
    if (j >= n) break;
    const double x = __shfl_sync(0xffffffffu, t[j / R], (base + j % R) & 31);
#pragma unroll
    for (int s = (j + 1) / R; s < S; s++) {
      const int c = q + R * s;
      if (c > j && c < n) t[s] = fma(-x, Ls[c * PITCH + j], t[s]);
    }
  }
  if (active) {
    double *drow = D.p + (long long)b * D.stride + pm_off(D.i0 + row, D.j0, D.cn);
#pragma unroll
    for (int s = 0; s < S; s++) {
      const int c = q + R * s;
      if (c < n) drow[PS * c] = t[s] * adv[c];
    }
  }
  pdl_allow();  // the next kernel may be scheduled once every CTA is here
}

template <int NB, int R>
cudaError_t launch_trsm_lat_nb(int batch, int m, int n, double alpha, Op L, const double *dinv, long long sdinv,
                               Op B, OpW D, cudaStream_t s) {
  constexpr int ROWS = (LAT_T / 32) * (32 / R);
  const int chunks = (m + ROWS - 1) / ROWS;
  const long long blocks = (long long)batch * chunks;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  return launch_pdl(k_trsm_lat<NB, R>, dim3((unsigned)blocks), dim3(LAT_T), 0, s, m, n, alpha, L, dinv, sdinv, B, D,
                    chunks);
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

template <bool FUSED>
cudaError_t launch_chol_lat_f(int batch, int n, int k, Op A, Op B, Op C, OpW D, double *dinv, long long sdinv,
                              int *info, cudaStream_t s) {
  const dim3 grid((unsigned)batch), block(LAT_T);
  if (n <= 8) return launch_pdl(k_chol_lat<FUSED, 8>, grid, block, 0, s, n, k, A, B, C, D, dinv, sdinv, info);
  if (n <= 16) return launch_pdl(k_chol_lat<FUSED, 16>, grid, block, 0, s, n, k, A, B, C, D, dinv, sdinv, info);
  if (n <= 24) return launch_pdl(k_chol_lat<FUSED, 24>, grid, block, 0, s, n, k, A, B, C, D, dinv, sdinv, info);
  return launch_pdl(k_chol_lat<FUSED, 32>, grid, block, 0, s, n, k, A, B, C, D, dinv, sdinv, info);
}

cudaError_t launch_chol_lat(bool fused, int batch, int n, int k, Op A, Op B, Op C, OpW D, double *dinv,
                            long long sdinv, int *info, cudaStream_t s) {
  if (n > CHOL_LAT_MAX_N) return cudaErrorInvalidValue;
  return fused ? launch_chol_lat_f<true>(batch, n, k, A, B, C, D, dinv, sdinv, info, s)
               : launch_chol_lat_f<false>(batch, n, k, A, B, C, D, dinv, sdinv, info, s);
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
