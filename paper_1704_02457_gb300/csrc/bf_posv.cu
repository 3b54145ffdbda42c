// Cholesky solves of SPD systems A X = B with a few right-hand sides:
//
//  potrs (FP64):  X = L^{-T} L^{-1} B with the factor from potrf_l.  The two
//    triangular solves are the right-hand-side forms of trsm (the trsv_lnn /
//    trsv_ltn routines of the paper's BLAS-2 list, Appendix A.3).
//
//  posv mixed:    the single-precision factor L32 of fl32(A) (k_chol_rows in
//    FP32, written to the caller's workspace) is used for FP32 triangular
//    solves inside an FP64 iterative refinement:
//        x = 0, r = b
//        repeat:  d = L32^{-T} L32^{-1} r   (FP32)
//                 x = x + d                 (FP64)
//                 r = b - A x               (FP64, A's lower triangle)
//        until ||R||_F / (||A||_F ||X||_F) <= tol   (all right-hand sides)
//    Each correction shrinks the residual by about cond(A) * 2^-24, so for
//    cond(A) <= 1e6 a handful of FP64 residuals replaces the FP64
//    factorization.
//
// One CTA per system.  The factor lives packed in shared memory (column l at
// cs(l), element (i, l) at cs(l) + i).  The FP64 solve gives one warp to one
// right-hand side (column-oriented forward and backward substitution in
// shared memory); the refinement's FP32 solves give one warp to four
// right-hand sides held in registers.  The FP64 residual gives every thread
// one row of A, read from L2 in panel-major order, for all right-hand sides
// at once.
#include <type_traits>

#include "bf_internal.cuh"

namespace bf {
namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ int col_start(int l, int n) { return (l * (2 * n - l + 1)) / 2 - l; }

template <typename T>
__device__ __forceinline__ void cp_async(T *dst, const T *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ double block_sum(double v, double *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; i++) s += red[i];
  return s;
}

// forward then backward substitution of one right-hand side v (length n) in
// shared memory against the packed factor L, by one warp: v <- L^{-T} L^{-1} v
template <typename T>
__device__ __forceinline__ void warp_solve(const T *L, const T *dinv, T *v, int n) {
  const int lane = threadIdx.x & 31;
  // L y = v: column j finishes y_j, then updates the rows below it
  for (int j = 0; j < n; j++) {
    const T yj = v[j] * dinv[j];
    __syncwarp();
    const int cs = col_start(j, n);
    for (int i = j + 1 + lane; i < n; i += 32) v[i] -= L[cs + i] * yj;
    if (lane == 0) v[j] = yj;
    __syncwarp();
  }
  // L^T x = y, column-oriented from the bottom up: x_j finishes, then the
  // rows above it take -L(j, i) x_j (L(j, i) = L^T(i, j) sits in packed
  // column i).  No reductions: a dot-product form would spend five shuffle
  // adds per column, each a full FP64 warp instruction.
  for (int j = n - 1; j >= 0; j--) {
    const T xj = v[j] * dinv[j];
    __syncwarp();
    for (int i = lane; i < j; i += 32) v[i] -= L[col_start(i, n) + j] * xj;
    if (lane == 0) v[j] = xj;
    __syncwarp();
  }
}

// The single-precision solves of the refinement, d = L32^{-T} L32^{-1} r for
// up to four right-hand sides k0..k0+3 by one warp, with the right-hand
// sides in registers: lane l holds rows l, l + 32, ... (R slots) of each.
// Column j's owner lane finishes y_j, one shuffle hands it to every lane,
// and each lane updates its own rows; the four right-hand sides interleave,
// so each step's shuffle latency is paid once for all of them.  Reads r from
// r64 and adds d to x64 (both FP64, length n per right-hand side).
template <int R>
__device__ __forceinline__ void warp_solve_refine(const float *L, const float *dinv, const double *r64,
                                                  double *x64, int n, int nrhs, int k0) {
  const int lane = threadIdx.x & 31;
  float v[R][4];
#pragma unroll
  for (int s = 0; s < R; s++)
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int i = s * 32 + lane;
      v[s][q] = (i < n && k0 + q < nrhs) ? (float)r64[(k0 + q) * n + i] : 0.0f;
    }
  // L y = r
#pragma unroll
  for (int s = 0; s < R; s++) {
    for (int l = 0; l < 32; l++) {
      const int j = s * 32 + l;
      if (j >= n) break;
      const float dj = dinv[j];
      const int cs = col_start(j, n);
      float y[4];
#pragma unroll
      for (int q = 0; q < 4; q++) y[q] = __shfl_sync(FULL, v[s][q], l) * dj;
      if (lane == l) {
#pragma unroll
        for (int q = 0; q < 4; q++) v[s][q] = y[q];
      }
#pragma unroll
      for (int t = s; t < R; t++) {
        const int i = t * 32 + lane;
        if (i > j && i < n) {
          const float lij = L[cs + i];
#pragma unroll
          for (int q = 0; q < 4; q++) v[t][q] = fmaf(-lij, y[q], v[t][q]);
        }
      }
    }
  }
  // L^T d = y, from the bottom up: L(j, i) = L^T(i, j) sits in packed column i
#pragma unroll
  for (int s = R - 1; s >= 0; s--) {
    for (int l = 31; l >= 0; l--) {
      const int j = s * 32 + l;
      if (j >= n) continue;
      const float dj = dinv[j];
      float xj[4];
#pragma unroll
      for (int q = 0; q < 4; q++) xj[q] = __shfl_sync(FULL, v[s][q], l) * dj;
      if (lane == l) {
#pragma unroll
        for (int q = 0; q < 4; q++) v[s][q] = xj[q];
      }
#pragma unroll
      for (int t = 0; t <= s; t++) {
        const int i = t * 32 + lane;
        if (i < j) {
          const float lji = L[col_start(i, n) + j];
#pragma unroll
          for (int q = 0; q < 4; q++) v[t][q] = fmaf(-lji, xj[q], v[t][q]);
        }
      }
    }
  }
#pragma unroll
  for (int s = 0; s < R; s++)
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int i = s * 32 + lane;
      if (i < n && k0 + q < nrhs) x64[(k0 + q) * n + i] += (double)v[s][q];
    }
}

// Column l of packed element e: column l starts at l(2n - l + 1)/2, so l is
// the smaller root of l^2 - (2n+1) l + 2e = 0, corrected for rounding.
__device__ __forceinline__ int packed_col(int e, int n) {
  const float q = 2.0f * n + 1.0f;
  int l = (int)((q - sqrtf(q * q - 8.0f * e)) * 0.5f);
  l = max(0, min(l, n - 1));
  while (l > 0 && col_start(l, n) + l > e) l--;
  while (l + 1 < n && col_start(l + 1, n) + l + 1 <= e) l++;
  return l;
}

// Loads the packed lower triangle of the panel-major factor into shared memory.
template <typename T>
__device__ __forceinline__ void load_factor(T *L, const T *pl, int cn, int i0, int j0, int n) {
  const int NE = n * (n + 1) / 2;
  for (int e = threadIdx.x; e < NE; e += blockDim.x) {
    const int l = packed_col(e, n);
    const int i = e - col_start(l, n);
    cp_async(&L[e], pl + pm_off(i0 + i, j0 + l, cn));
  }
}

// r = b - A x for NR right-hand sides (A's lower triangle, symmetric);
// accumulates ||r||^2 and ||x||^2 of this thread's rows.
template <int NR>
__device__ __forceinline__ void residual(int n, const double *pa, const Op &A, const double *pb,
                                         const Op &B, const double *x64, double *r64, double &rs,
                                         double &xs) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double acc[NR];
#pragma unroll
    for (int k = 0; k < NR; k++) acc[k] = 0.0;
    // one loop over j for every lane (A(i, j) from row i below the diagonal,
    // A(j, i) from column i above it): two loops of lane-dependent lengths
    // would run n + 31 masked FP64 iterations per warp instead of n
    const double *arow = pa + pm_off(A.i0 + i, A.j0, A.cn);
    for (int j = 0; j < n; j++) {
      const double a = (j <= i) ? arow[(long long)j * PS] : pa[pm_off(A.i0 + j, A.j0 + i, A.cn)];
#pragma unroll
      for (int k = 0; k < NR; k++) acc[k] = fma(a, x64[k * n + j], acc[k]);
    }
#pragma unroll
    for (int k = 0; k < NR; k++) {
      const double r = pb[pm_off(B.i0 + i, B.j0 + k, B.cn)] - acc[k];
      r64[k * n + i] = r;
      rs += r * r;
      xs += x64[k * n + i] * x64[k * n + i];
    }
  }
}

// Resident CTAs the refinement kernel is compiled for: 4 caps it at 64
// registers (no spills), so that shared memory (the FP32 factor, 42 KB at
// n = 128) rather than registers bounds it, at 5 CTAs per SM.  Measured at
// n = 128, 8192 systems, 4 right-hand sides: 4.16 ms at 116 registers (4
// CTAs), 3.83 ms at 64.
#ifndef BF_POSV_MINB
#define BF_POSV_MINB 4
#endif

template <bool MIXED>
__global__ void __launch_bounds__(256, MIXED ? BF_POSV_MINB : 1)
k_posv(int n, int nrhs, Op A, const float *l32, long long sl32, const int *info32, Op Lf, Op B,
       OpW X, double tol, int max_iter, int *iters, double *resid) {
  using TL = typename std::conditional<MIXED, float, double>::type;
  extern __shared__ double smem_d[];
  const int b = blockIdx.x;
  const int t = threadIdx.x, T = blockDim.x;
  const int NE = n * (n + 1) / 2;
  // shared memory: [x64 | r64 (MIXED)] [red] [L (TL)] [dinv (TL)] [v (TL, FP64 solve only)]
  double *x64 = smem_d;
  double *r64 = x64 + (MIXED ? nrhs * n : 0);
  double *red = r64 + (MIXED ? nrhs * n : 0);
  TL *L = (TL *)(red + 32);
  TL *dinv = L + ((NE + 3) & ~3);
  TL *v = dinv + ((n + 3) & ~3);

  if (MIXED && info32 && info32[b] != 0) {
    // the single-precision factorization failed: report and leave X untouched
    if (t == 0) {
      if (iters) iters[b] = -2;
      if (resid) resid[b] = -1.0;
    }
    return;
  }

  // factor into shared memory, right-hand sides alongside
  if (MIXED)
    load_factor<float>((float *)L, l32 + b * sl32, n, 0, 0, n);
  else
    load_factor<double>((double *)L, Lf.p + b * Lf.stride, Lf.cn, Lf.i0, Lf.j0, n);
  const double *pb = B.p + b * B.stride;
  for (int e = t; e < nrhs * n; e += T) {
    const int k = e / n, i = e - k * n;
    const double bv = pb[pm_off(B.i0 + i, B.j0 + k, B.cn)];
    if (MIXED) {
      r64[e] = bv;
      x64[e] = 0.0;
    } else {
      v[e] = (TL)bv;
    }
  }
  cp_async_wait_all();
  __syncthreads();
  for (int j = t; j < n; j += T) dinv[j] = (TL)1 / L[col_start(j, n) + j];
  __syncthreads();

  const int warp = t >> 5, nwarps = (T + 31) >> 5;
  if (!MIXED) {
    for (int k = warp; k < nrhs; k += nwarps) warp_solve<TL>(L, dinv, v + k * n, n);
    __syncthreads();
    double *px = X.p + b * X.stride;
    for (int e = t; e < nrhs * n; e += T) {
      const int k = e / n, i = e - k * n;
      px[pm_off(X.i0 + i, X.j0 + k, X.cn)] = (double)v[e];
    }
    return;
  }

  // ||A||_F from the lower triangle (off-diagonal entries count twice)
  const double *pa = A.p + b * A.stride;
  double sd = 0.0, so = 0.0;  // diagonal and off-diagonal sums of squares: one FMA per entry
  for (int e = t; e < NE; e += T) {
    const int l = packed_col(e, n);
    const int i = e - col_start(l, n);
    const double a = pa[pm_off(A.i0 + i, A.j0 + l, A.cn)];
    if (i == l)
      sd = fma(a, a, sd);
    else
      so = fma(a, a, so);
  }
  const double anrm = sqrt(block_sum(fma(2.0, so, sd), red));

  int it = 0;
  double rel = 0.0;
  bool done = false;
  for (; it < max_iter && !done; it++) {
    // x += A32^{-1} r in single precision, four right-hand sides per warp
    if constexpr (MIXED) {
      for (int k0 = warp * 4; k0 < nrhs; k0 += nwarps * 4) {
        switch ((n + 31) / 32) {
          case 1: warp_solve_refine<1>(L, dinv, r64, x64, n, nrhs, k0); break;
          case 2: warp_solve_refine<2>(L, dinv, r64, x64, n, nrhs, k0); break;
          case 3: warp_solve_refine<3>(L, dinv, r64, x64, n, nrhs, k0); break;
          case 4: warp_solve_refine<4>(L, dinv, r64, x64, n, nrhs, k0); break;
          case 5: warp_solve_refine<5>(L, dinv, r64, x64, n, nrhs, k0); break;
          case 6: warp_solve_refine<6>(L, dinv, r64, x64, n, nrhs, k0); break;
          case 7: warp_solve_refine<7>(L, dinv, r64, x64, n, nrhs, k0); break;
          default: warp_solve_refine<8>(L, dinv, r64, x64, n, nrhs, k0); break;
        }
      }
    }
    __syncthreads();
    // r = b - A x in FP64; thread i owns row i for every right-hand side
    double rs = 0.0, xs = 0.0;
    switch (nrhs) {
      case 1: residual<1>(n, pa, A, pb, B, x64, r64, rs, xs); break;
      case 2: residual<2>(n, pa, A, pb, B, x64, r64, rs, xs); break;
      case 3: residual<3>(n, pa, A, pb, B, x64, r64, rs, xs); break;
      case 4: residual<4>(n, pa, A, pb, B, x64, r64, rs, xs); break;
      case 5: residual<5>(n, pa, A, pb, B, x64, r64, rs, xs); break;
      case 6: residual<6>(n, pa, A, pb, B, x64, r64, rs, xs); break;
      case 7: residual<7>(n, pa, A, pb, B, x64, r64, rs, xs); break;
      default: residual<8>(n, pa, A, pb, B, x64, r64, rs, xs); break;
    }
    // both sums in one reduction; one thread forms the relative residual
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      rs += __shfl_xor_sync(FULL, rs, o);
      xs += __shfl_xor_sync(FULL, xs, o);
    }
    if ((t & 31) == 0) {
      red[warp] = rs;
      red[16 + warp] = xs;
    }
    __syncthreads();
    if (t == 0) {
      double rsum = 0.0, xsum = 0.0;
      for (int w = 0; w < nwarps; w++) {
        rsum += red[w];
        xsum += red[16 + w];
      }
      red[31] = sqrt(rsum) / (anrm * sqrt(xsum));
    }
    __syncthreads();
    rel = red[31];
    done = rel <= tol;  // the same value in every thread
  }
  double *px = X.p + b * X.stride;
  for (int e = t; e < nrhs * n; e += T) {
    const int k = e / n, i = e - k * n;
    px[pm_off(X.i0 + i, X.j0 + k, X.cn)] = x64[e];
  }
  if (t == 0) {
    if (iters) iters[b] = done ? it : -1;
    if (resid) resid[b] = rel;
  }
}

// Adjoint of X = A^{-1} B given A's factor L: Bbar = A^{-1} Xbar (the solve
// with the saved factor, one warp per right-hand side) and
// Abar = -(Bbar X^T + X Bbar^T) / 2, written in full.
__global__ void __launch_bounds__(256)
k_posv_adjoint(int n, int nrhs, Op Lf, Op Xs, Op Xb, OpW Bb, OpW Ab) {
  extern __shared__ double smem_d[];
  const int b = blockIdx.x;
  const int t = threadIdx.x, T = blockDim.x;
  const int NE = n * (n + 1) / 2;
  double *L = smem_d;
  double *dinv = L + ((NE + 1) & ~1);
  double *v = dinv + ((n + 1) & ~1);  // Xbar, then Bbar
  double *x = v + nrhs * n;
  load_factor<double>(L, Lf.p + b * Lf.stride, Lf.cn, Lf.i0, Lf.j0, n);
  const double *px = Xs.p + b * Xs.stride, *pxb = Xb.p + b * Xb.stride;
  for (int e = t; e < nrhs * n; e += T) {
    const int k = e / n, i = e - k * n;
    v[e] = pxb[pm_off(Xb.i0 + i, Xb.j0 + k, Xb.cn)];
    x[e] = px[pm_off(Xs.i0 + i, Xs.j0 + k, Xs.cn)];
  }
  cp_async_wait_all();
  __syncthreads();
  for (int j = t; j < n; j += T) dinv[j] = 1.0 / L[col_start(j, n) + j];
  __syncthreads();
  const int warp = t >> 5, nwarps = (T + 31) >> 5;
  for (int k = warp; k < nrhs; k += nwarps) warp_solve<double>(L, dinv, v + k * n, n);
  __syncthreads();
  double *pbb = Bb.p + b * Bb.stride;
  for (int e = t; e < nrhs * n; e += T) {
    const int k = e / n, i = e - k * n;
    pbb[pm_off(Bb.i0 + i, Bb.j0 + k, Bb.cn)] = v[e];
  }
  double *pab = Ab.p + b * Ab.stride;
  for (int e = t; e < n * n; e += T) {
    const int j = e / n, i = e - j * n;
    // (bbar_i x_j + x_i bbar_j) with separately rounded products and sums,
    // so that Abar(i, j) and Abar(j, i) are the same number bit for bit
    double s = 0.0;
    for (int k = 0; k < nrhs; k++)
      s = __dadd_rn(s, __dadd_rn(__dmul_rn(v[k * n + i], x[k * n + j]), __dmul_rn(x[k * n + i], v[k * n + j])));
    pab[pm_off(Ab.i0 + i, Ab.j0 + j, Ab.cn)] = -0.5 * s;
  }
}

size_t posv_smem(bool mixed, int n, int nrhs) {
  const size_t ne = (size_t)n * (n + 1) / 2;
  const size_t tl = mixed ? 4 : 8;
  size_t bytes = (mixed ? 2 * (size_t)nrhs * n * 8 : 0) + 32 * 8;
  // the FP64 solve works on a copy of the right-hand sides in shared memory;
  // the refinement keeps its single-precision ones in registers
  bytes += (((ne + 3) & ~(size_t)3) + (((size_t)n + 3) & ~(size_t)3) + (mixed ? 0 : (size_t)nrhs * n)) * tl;
  return bytes;
}

int posv_threads(int n, int nrhs) {
  const int t = max(32 * nrhs, (n + 31) & ~31);
  return min(256, max(32, t));
}

template <bool MIXED>
cudaError_t set_posv_smem_attr() {
  static std::atomic<unsigned long long> done{0};
  return smem_attr_once((const void *)k_posv<MIXED>, 200 * 1024, done);
}

}  // namespace

cudaError_t launch_potrs(int batch, int n, int nrhs, Op L, Op B, OpW X, cudaStream_t s) {
  const size_t smem = posv_smem(false, n, nrhs);
  if (smem > 200 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = set_posv_smem_attr<false>();
  if (e != cudaSuccess) return e;
  const Op none{nullptr, 0, 0, 0, 0};
  k_posv<false><<<batch, posv_threads(n, nrhs), smem, s>>>(n, nrhs, none, nullptr, 0, nullptr, L, B, X,
                                                           0.0, 0, nullptr, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_posv_adjoint(int batch, int n, int nrhs, Op L, Op X, Op Xbar, OpW Bbar, OpW Abar,
                                cudaStream_t s) {
  const size_t ne = (size_t)n * (n + 1) / 2;
  const size_t smem = (((ne + 1) & ~(size_t)1) + (((size_t)n + 1) & ~(size_t)1) + 2 * (size_t)nrhs * n) * 8;
  if (smem > 200 * 1024) return cudaErrorInvalidConfiguration;
  static std::atomic<unsigned long long> attr{0};
  cudaError_t e = smem_attr_once((const void *)k_posv_adjoint, 200 * 1024, attr);
  if (e != cudaSuccess) return e;
  k_posv_adjoint<<<batch, posv_threads(n, nrhs), smem, s>>>(n, nrhs, L, X, Xbar, Bbar, Abar);
  return cudaGetLastError();
}

cudaError_t launch_posv_mixed(int batch, int n, int nrhs, Op A, Op B, OpW X, double tol,
                              int max_iter, int *iters, double *resid, float *l32, int *info32,
                              bool aligned, cudaStream_t s) {
  const int pm = (n + PS - 1) / PS * PS;
  const OpWT<float> D{l32, (long long)pm * n, n, 0, 0};
  cudaError_t e = launch_chol_f32(batch, n, A, D, info32, aligned, s);
  if (e != cudaSuccess) return e;
  return launch_posv_refine(batch, n, nrhs, A, B, X, tol, max_iter, iters, resid, l32, info32, s);
}

cudaError_t launch_posv_refine(int batch, int n, int nrhs, Op A, Op B, OpW X, double tol, int max_iter, int *iters,
                               double *resid, const float *l32, const int *info32, cudaStream_t s) {
  const int pm = (n + PS - 1) / PS * PS;
  cudaError_t e;
  const size_t smem = posv_smem(true, n, nrhs);
  if (smem > 200 * 1024) return cudaErrorInvalidConfiguration;
  e = set_posv_smem_attr<true>();
  if (e != cudaSuccess) return e;
  const Op none{nullptr, 0, 0, 0, 0};
  k_posv<true><<<batch, posv_threads(n, nrhs), smem, s>>>(n, nrhs, A, l32, (long long)pm * n, info32, none,
                                                          B, X, tol, max_iter, iters, resid);
  return cudaGetLastError();
}

}  // namespace bf
