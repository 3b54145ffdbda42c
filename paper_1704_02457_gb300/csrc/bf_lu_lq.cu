// getrf (LU with partial pivoting) and gelqf (Householder LQ), batched,
// FP64, panel-major operands (Sec. 5.2.2 "getrf" and "gelqf"; routine list
// of Appendix A.3).
//
// getrf:  P A = L U for square A, column by column: the pivot is the first
//         row with the largest |a(i, j)| at or below the diagonal, rows j and
//         p are swapped whole, the multipliers below the pivot are scaled by
//         its reciprocal and the trailing matrix takes a rank-1 update.
// gelqf:  A = L Q, row by row: the reflector H_i = I - tau v v^T (v = [1, x])
//         annihilates a(i, i+1:n) with beta = -sign(alpha) ||(alpha, x)||,
//         x is scaled by 1 / (alpha - beta), and the rows below are updated
//         from the right.  L is the lower triangle of the result; the
//         reflectors stay in the strictly upper part, tau alongside.
//
// Layout: a CTA is one warp holding Q = 32/G problems, G lanes each, whole
// matrices in shared memory (problem q's element (i, j) at
// sm[(j*rows + i)*Q + q]).  As in the small Cholesky, the sequential part of
// each step (pivot choice, reciprocal, norm and square root) is one warp
// instruction for all Q problems; a problem's G lanes split the rows (or
// columns) of the step's updates.
#include <math_constants.h>

#include "bf_internal.cuh"

namespace bf {
namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ void cp_async8(double *dst, const double *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// whole m x n matrices of the warp's problems in and out of shared memory
template <int Q>
__device__ __forceinline__ void load_all(double *sm, int b0, int batch, int m, int n, const Op &C) {
  const int lane = threadIdx.x;
  for (int qq = 0; qq < Q; qq++) {
    const int bb = b0 + qq;
    if (bb >= batch) break;
    const double *pc = C.p + bb * C.stride;
    for (int x = lane; x < m * n; x += 32) {
      const int j = x / m, i = x - j * m;
      cp_async8(&sm[(j * m + i) * Q + qq], pc + pm_off(C.i0 + i, C.j0 + j, C.cn));
    }
  }
  cp_async_wait_all();
  __syncwarp();
}

template <int Q>
__device__ __forceinline__ void store_all(const double *sm, int b0, int batch, int m, int n, const OpW &D) {
  const int lane = threadIdx.x;
  __syncwarp();
  for (int qq = 0; qq < Q; qq++) {
    const int bb = b0 + qq;
    if (bb >= batch) break;
    double *pd = D.p + bb * D.stride;
    for (int x = lane; x < m * n; x += 32) {
      const int j = x / m, i = x - j * m;
      pd[pm_off(D.i0 + i, D.j0 + j, D.cn)] = sm[(j * m + i) * Q + qq];
    }
  }
}

template <int G>
__global__ void __launch_bounds__(32)
k_getrf(int batch, int n, Op C, OpW D, int *ipiv, long long sipiv, int *info) {
  constexpr int Q = 32 / G;
  extern __shared__ double sm[];
  const int lane = threadIdx.x, q = lane / G, s = lane % G;
  const int b0 = blockIdx.x * Q, b = b0 + q;
  const bool valid = b < batch;
#define A_(i, j) sm[((j) * n + (i)) * Q + q]
  load_all<Q>(sm, b0, batch, n, n, C);
  int first_zero = 0;
  for (int j = 0; j < n; j++) {
    // pivot: largest |a(i, j)|, i >= j, first such row
    const bool diag_nan = isnan(A_(j, j));  // read before any lane can swap
    double best = -1.0;
    int bi = j;  // stays the diagonal if nothing compares larger (e.g. NaN)
    for (int i = j + s; i < n; i += G) {
      const double v = fabs(A_(i, j));
      if (v > best) {
        best = v;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
      const double ov = __shfl_xor_sync(FULL, best, o);
      const int oi = __shfl_xor_sync(FULL, bi, o);
      if (ov > best || (ov == best && oi < bi)) {
        best = ov;
        bi = oi;
      }
    }
    const int p = diag_nan ? j : bi;  // a NaN diagonal keeps its row
    if (p != j)
      for (int c = s; c < n; c += G) {
        const double t = A_(j, c);
        A_(j, c) = A_(p, c);
        A_(p, c) = t;
      }
    __syncwarp();
    const double piv = A_(j, j);
    if (valid && s == 0) ipiv[b * sipiv + j] = p;
    if (piv == 0.0) {
      if (first_zero == 0) first_zero = j + 1;
    } else {
      const double r = recip_newton(piv);
      for (int i = j + 1 + s; i < n; i += G) {
        const double l = A_(i, j) * r;
        A_(i, j) = l;
        for (int c = j + 1; c < n; c++) A_(i, c) = fma(-l, A_(j, c), A_(i, c));
      }
    }
    __syncwarp();
  }
#undef A_
  store_all<Q>(sm, b0, batch, n, n, D);
  if (info && valid && s == 0) info[b] = first_zero;
}

template <int G>
__global__ void __launch_bounds__(32)
k_gelqf(int batch, int m, int n, Op C, OpW D, double *tau, long long stau) {
  constexpr int Q = 32 / G;
  extern __shared__ double sm[];
  const int lane = threadIdx.x, q = lane / G, s = lane % G;
  const int b0 = blockIdx.x * Q, b = b0 + q;
  const bool valid = b < batch;
#define A_(i, j) sm[((j) * m + (i)) * Q + q]
  load_all<Q>(sm, b0, batch, m, n, C);
  const int k = min(m, n);
  for (int i = 0; i < k; i++) {
    double ss = 0.0;
    for (int c = i + 1 + s; c < n; c += G) ss = fma(A_(i, c), A_(i, c), ss);
#pragma unroll
    for (int o = 1; o < G; o <<= 1) ss += __shfl_xor_sync(FULL, ss, o);
    const double alpha = A_(i, i);
    double t = 0.0;
    __syncwarp();
    if (ss != 0.0) {
      const double beta = -copysign(sqrt(fma(alpha, alpha, ss)), alpha);
      t = (beta - alpha) / beta;
      const double scal = 1.0 / (alpha - beta);
      for (int c = i + 1 + s; c < n; c += G) A_(i, c) *= scal;
      if (s == 0) A_(i, i) = beta;
    }
    if (valid && s == 0) tau[b * stau + i] = t;
    __syncwarp();
    for (int r = i + 1 + s; r < m; r += G) {
      double w = A_(r, i);
      for (int c = i + 1; c < n; c++) w = fma(A_(r, c), A_(i, c), w);
      const double tw = t * w;
      A_(r, i) -= tw;
      for (int c = i + 1; c < n; c++) A_(r, c) = fma(-tw, A_(i, c), A_(r, c));
    }
    __syncwarp();
  }
#undef A_
  store_all<Q>(sm, b0, batch, m, n, D);
}

// ---------------------------------------------------------------------------
// Row kernels (one CTA per problem, one thread per row, 32 <= rows): the
// matrix sits in shared memory column-major with an odd leading dimension
// ld, so a warp walking down a column (thread-per-row updates) or along a
// row (swaps, the reflector's row) touches distinct banks.
// ---------------------------------------------------------------------------

// (value, row) arg-max over the CTA; ties go to the smaller row.  red holds
// one slot per warp; every thread returns the same row.
__device__ __forceinline__ int cta_argmax(double v, int idx, double *red_v, int *red_i) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(FULL, v, o);
    const int oi = __shfl_xor_sync(FULL, idx, o);
    if (ov > v || (ov == v && oi < idx)) {
      v = ov;
      idx = oi;
    }
  }
  if (lane == 0) {
    red_v[wid] = v;
    red_i[wid] = idx;
  }
  __syncthreads();
  double bv = red_v[0];
  int bi = red_i[0];
  for (int w = 1; w < nw; w++) {
    const double ov = red_v[w];
    const int oi = red_i[w];
    if (ov > bv || (ov == bv && oi < bi)) {
      bv = ov;
      bi = oi;
    }
  }
  return bi;
}

__device__ __forceinline__ double cta_sum(double v, double *red_v) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  if (lane == 0) red_v[wid] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < nw; w++) s += red_v[w];
  return s;
}

// panel-major <-> shared memory (column-major, leading dimension ld), walked
// in panel-major order so that consecutive threads touch consecutive words
__device__ __forceinline__ void rows_load(double *sm, int ld, int m, int n, const double *pc, const Op &C) {
  const int mp = (m + PS - 1) / PS;
  for (int x = threadIdx.x; x < mp * PS * n; x += blockDim.x) {
    const int r4 = x % PS, j = (x / PS) % n, i = (x / (PS * n)) * PS + r4;
    if (i < m) cp_async8(&sm[j * ld + i], pc + pm_off(C.i0 + i, C.j0 + j, C.cn));
  }
  cp_async_wait_all();
  __syncthreads();
}

__device__ __forceinline__ void rows_store(const double *sm, int ld, int m, int n, double *pd, const OpW &D) {
  __syncthreads();
  const int mp = (m + PS - 1) / PS;
  for (int x = threadIdx.x; x < mp * PS * n; x += blockDim.x) {
    const int r4 = x % PS, j = (x / PS) % n, i = (x / (PS * n)) * PS + r4;
    if (i < m) pd[pm_off(D.i0 + i, D.j0 + j, D.cn)] = sm[j * ld + i];
  }
}

__global__ void __launch_bounds__(128)
k_getrf_rows(int n, int ld, Op C, OpW D, int *ipiv, long long sipiv, int *info) {
  extern __shared__ double sm[];
  __shared__ double red_v[4];
  __shared__ int red_i[4];
  const int b = blockIdx.x, t = threadIdx.x;
  rows_load(sm, ld, n, n, C.p + b * C.stride, C);
  int first_zero = 0;
  for (int j = 0; j < n; j++) {
    // NaN entries never win; a NaN diagonal keeps its row.  Both reads come
    // before the barrier inside cta_argmax, so before any swap.
    const double x = (t >= j && t < n) ? sm[j * ld + t] : CUDART_NAN;
    const bool diag_nan = isnan(sm[j * ld + j]);
    const bool cand = !isnan(x);
    const int p = cta_argmax(cand ? fabs(x) : -1.0, cand ? t : n, red_v, red_i);
    const int pr = (p < n && !diag_nan) ? p : j;
    if (pr != j && t < n) {
      const double x = sm[t * ld + j];
      sm[t * ld + j] = sm[t * ld + pr];
      sm[t * ld + pr] = x;
    }
    if (t == 0) ipiv[b * sipiv + j] = pr;
    __syncthreads();
    const double piv = sm[j * ld + j];
    if (piv == 0.0) {
      if (first_zero == 0) first_zero = j + 1;
    } else if (t > j && t < n) {
      const double l = sm[j * ld + t] * recip_newton(piv);
      sm[j * ld + t] = l;
      for (int c = j + 1; c < n; c++) sm[c * ld + t] = fma(-l, sm[c * ld + j], sm[c * ld + t]);
    }
    __syncthreads();
  }
  rows_store(sm, ld, n, n, D.p + b * D.stride, D);
  if (info && t == 0) info[b] = first_zero;
}

__global__ void __launch_bounds__(128)
k_gelqf_rows(int m, int n, int ld, Op C, OpW D, double *tau, long long stau) {
  extern __shared__ double sm[];
  __shared__ double red_v[4];
  const int b = blockIdx.x, t = threadIdx.x, T_ = blockDim.x;
  rows_load(sm, ld, m, n, C.p + b * C.stride, C);
  const int k = min(m, n);
  for (int i = 0; i < k; i++) {
    double part = 0.0;
    for (int c = i + 1 + t; c < n; c += T_) part = fma(sm[c * ld + i], sm[c * ld + i], part);
    const double alpha = sm[i * ld + i];  // read before the barrier in cta_sum: thread 0 overwrites it
    const double ss = cta_sum(part, red_v);
    double tv = 0.0;
    if (ss != 0.0) {
      const double beta = -copysign(sqrt(fma(alpha, alpha, ss)), alpha);
      tv = (beta - alpha) / beta;
      const double scal = 1.0 / (alpha - beta);
      for (int c = i + 1 + t; c < n; c += T_) sm[c * ld + i] *= scal;
      if (t == 0) sm[i * ld + i] = beta;
    }
    if (t == 0) tau[b * stau + i] = tv;
    __syncthreads();
    for (int r = i + 1 + t; r < m; r += T_) {
      double w = sm[i * ld + r];
      for (int c = i + 1; c < n; c++) w = fma(sm[c * ld + r], sm[c * ld + i], w);
      const double tw = tv * w;
      sm[i * ld + r] -= tw;
      for (int c = i + 1; c < n; c++) sm[c * ld + r] = fma(-tw, sm[c * ld + i], sm[c * ld + r]);
    }
    __syncthreads();
  }
  rows_store(sm, ld, m, n, D.p + b * D.stride, D);
}

// Lanes per problem of the one-warp kernels: the smallest G whose matrices
// for the warp's 32/G problems fit 20 KB (many resident warps per SM hide the
// latency of the per-column pivot and reciprocal); else one problem per warp.
int pick_g(size_t bytes_per_problem) {
  for (int g = 1; g <= 32; g *= 2)
    if (bytes_per_problem * (32 / g) <= 20 * 1024) return g;
  return 32;
}

#ifndef BF_LU_ROWS_MIN
#define BF_LU_ROWS_MIN 32  // rows from which the one-CTA-per-problem kernels are used
#endif

cudaError_t set_smem(const void *fn, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <int G>
cudaError_t run_getrf(int batch, int n, Op C, OpW D, int *ipiv, long long sipiv, int *info, cudaStream_t s) {
  constexpr int Q = 32 / G;
  const size_t smem = (size_t)n * n * Q * sizeof(double);
  cudaError_t e = set_smem((const void *)k_getrf<G>, smem);
  if (e != cudaSuccess) return e;
  k_getrf<G><<<(batch + Q - 1) / Q, 32, smem, s>>>(batch, n, C, D, ipiv, sipiv, info);
  return cudaGetLastError();
}

template <int G>
cudaError_t run_gelqf(int batch, int m, int n, Op C, OpW D, double *tau, long long stau, cudaStream_t s) {
  constexpr int Q = 32 / G;
  const size_t smem = (size_t)m * n * Q * sizeof(double);
  cudaError_t e = set_smem((const void *)k_gelqf<G>, smem);
  if (e != cudaSuccess) return e;
  k_gelqf<G><<<(batch + Q - 1) / Q, 32, smem, s>>>(batch, m, n, C, D, tau, stau);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_getrf(int batch, int n, Op C, OpW D, int *ipiv, long long sipiv, int *info, cudaStream_t s) {
  if (n >= BF_LU_ROWS_MIN) {
    const int ld = n | 1;
    const size_t smem = (size_t)ld * n * sizeof(double);
    cudaError_t e = set_smem((const void *)k_getrf_rows, smem);
    if (e != cudaSuccess) return e;
    k_getrf_rows<<<batch, ((n + 31) / 32) * 32, smem, s>>>(n, ld, C, D, ipiv, sipiv, info);
    return cudaGetLastError();
  }
  switch (pick_g((size_t)n * n * 8)) {
    case 1: return run_getrf<1>(batch, n, C, D, ipiv, sipiv, info, s);
    case 2: return run_getrf<2>(batch, n, C, D, ipiv, sipiv, info, s);
    case 4: return run_getrf<4>(batch, n, C, D, ipiv, sipiv, info, s);
    case 8: return run_getrf<8>(batch, n, C, D, ipiv, sipiv, info, s);
    case 16: return run_getrf<16>(batch, n, C, D, ipiv, sipiv, info, s);
    default: return run_getrf<32>(batch, n, C, D, ipiv, sipiv, info, s);
  }
}

cudaError_t launch_gelqf(int batch, int m, int n, Op C, OpW D, double *tau, long long stau, cudaStream_t s) {
  if (m >= BF_LU_ROWS_MIN) {
    const int ld = m | 1;
    const size_t smem = (size_t)ld * n * sizeof(double);
    cudaError_t e = set_smem((const void *)k_gelqf_rows, smem);
    if (e != cudaSuccess) return e;
    k_gelqf_rows<<<batch, min(128, ((m + 31) / 32) * 32), smem, s>>>(m, n, ld, C, D, tau, stau);
    return cudaGetLastError();
  }
  switch (pick_g((size_t)m * n * 8)) {
    case 1: return run_gelqf<1>(batch, m, n, C, D, tau, stau, s);
    case 2: return run_gelqf<2>(batch, m, n, C, D, tau, stau, s);
    case 4: return run_gelqf<4>(batch, m, n, C, D, tau, stau, s);
    case 8: return run_gelqf<8>(batch, m, n, C, D, tau, stau, s);
    case 16: return run_gelqf<16>(batch, m, n, C, D, tau, stau, s);
    default: return run_gelqf<32>(batch, m, n, C, D, tau, stau, s);
  }
}

}  // namespace bf
