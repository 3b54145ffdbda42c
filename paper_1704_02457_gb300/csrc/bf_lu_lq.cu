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

// Pivot key of x: the bits of |x| as a signed integer (for non-negative
// doubles the IEEE order is the integer order), -1 for NaN, so that the
// pivot search compares on the integer pipes instead of issuing FP64
// compares, and NaN never wins.
__device__ __forceinline__ long long pivot_key(double x) {
  const long long a = __double_as_longlong(x) & 0x7fffffffffffffffLL;
  return a > 0x7ff0000000000000LL ? -1LL : a;
}

// The scalars of the reflector that annihilates x, from alpha and
// ss = ||x||^2 > 0: beta = -sign(alpha) sqrt(alpha^2 + ss), tau = (beta -
// alpha) / beta and scal = 1 / (alpha - beta), by one reciprocal square
// root and one reciprocal instead of a square root and two divisions (the
// sequential part of each row, which on GB300 costs a warp the same FP64
// issue time whatever its active lanes).  With s = alpha^2 + ss and
// r = 1/sqrt(s): beta = -sign(alpha) s r, tau = 1 + |alpha| r, and
// alpha - beta = sign(alpha) (|alpha| + s r).  The signs are applied on the
// bit patterns (copysign), not by FP64 products.  The reciprocal is the
// library's (rcp.approx and one third-order correction): a row whose
// |alpha| + ||(alpha, x)|| is subnormal gives NaN.
__device__ __forceinline__ void reflector_scalars(double alpha, double ss, double &beta, double &tau, double &scal) {
  const double s = fma(alpha, alpha, ss);
  const double r = rsqrt(s);
  const double rt = s * r;
  beta = copysign(rt, -alpha);
  tau = fma(fabs(alpha), r, 1.0);
  scal = copysign(recip3(fabs(alpha) + rt), alpha);
}

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
    const bool diag_nan = pivot_key(A_(j, j)) < 0;  // read before any lane can swap
    long long best = -1;
    int bi = j;  // stays the diagonal if nothing compares larger (e.g. NaN)
    for (int i = j + s; i < n; i += G) {
      const long long v = pivot_key(A_(i, j));
      if (v > best) {
        best = v;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
      const long long ov = __shfl_xor_sync(FULL, best, o);
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
    if (is_zero(piv)) {
      if (first_zero == 0) first_zero = j + 1;
    } else {
      const double r = recip3(piv);
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
    if (!is_zero(ss)) {
      double beta, scal;
      reflector_scalars(alpha, ss, beta, t, scal);
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

// Pivot arg-max over the CTA on integer keys (pivot_key), carrying the
// winner's signed value; ties go to the smaller row.  Every thread returns
// the same row.
__device__ __forceinline__ int cta_argmax_v(long long key, int idx, double v, double *out_v, long long *red_k,
                                            int *red_i, double *red_s) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long ok = __shfl_xor_sync(FULL, key, o);
    const int oi = __shfl_xor_sync(FULL, idx, o);
    const double ov = __shfl_xor_sync(FULL, v, o);
    if (ok > key || (ok == key && oi < idx)) {
      key = ok;
      idx = oi;
      v = ov;
    }
  }
  if (lane == 0) {
    red_k[wid] = key;
    red_i[wid] = idx;
    red_s[wid] = v;
  }
  __syncthreads();
  long long bk = red_k[0];
  double bv = red_s[0];
  int bi = red_i[0];
  for (int w = 1; w < nw; w++) {
    const long long ok = red_k[w];
    const int oi = red_i[w];
    if (ok > bk || (ok == bk && oi < bi)) {
      bk = ok;
      bi = oi;
      bv = red_s[w];
    }
  }
  *out_v = bv;
  return bi;
}

// getrf, one CTA per problem.  Per column j, three barriers:
//  (1) arg-max of |a(i, j)|, i >= j (NaN entries never win, a NaN diagonal
//      keeps its row); every thread learns the pivot row p and value;
//  (2) thread t swaps rows j and p in column t (t != j); warp 0 scales
//      column j below the diagonal by the pivot's reciprocal (row p takes
//      the old diagonal, read before barrier (1)).  An FP64 instruction costs
//      the same for 1 or 32 lanes, so the per-column scalar work stays on one
//      warp;
//  (3) the trailing update a(i, c) -= l(i) u(c), i, c > j, spread over all
//      threads element by element (column-major order), so the work does
//      not shrink onto fewer warps as the factorization proceeds.
__global__ void __launch_bounds__(512)
k_getrf_rows(int n, int ld, Op C, OpW D, int *ipiv, long long sipiv, int *info) {
  extern __shared__ double sm[];
  __shared__ long long red_k[16];
  __shared__ double red_s[16];
  __shared__ int red_i[16];
  const int b = blockIdx.x, t = threadIdx.x, T_ = blockDim.x;
  rows_load(sm, ld, n, n, C.p + b * C.stride, C);
  int first_zero = 0;
  for (int j = 0; j < n; j++) {
    const double x = (t >= j && t < n) ? sm[j * ld + t] : CUDART_NAN;
    const double djj = sm[j * ld + j];  // read before barrier (1): rewritten in phase (2)
    const long long key = pivot_key(x);
    double pv;
    const int p = cta_argmax_v(key, key >= 0 ? t : n, x, &pv, red_k, red_i, red_s);
    const bool keep = (p >= n) || pivot_key(djj) < 0;
    const int pr = keep ? j : p;
    const double piv = keep ? djj : pv;
    if (t == 0) ipiv[b * sipiv + j] = pr;
    if (is_zero(piv)) {
      if (first_zero == 0) first_zero = j + 1;
      // column j is zero at and below the diagonal: no swap, no update
      __syncthreads();
      continue;
    }
    if (pr != j && t < n && t != j) {
      const double y = sm[t * ld + j];
      sm[t * ld + j] = sm[t * ld + pr];
      sm[t * ld + pr] = y;
    }
    if (t < 32) {  // one warp forms the reciprocal and the multipliers (FP64 work is issued per warp)
      const double r = recip3(piv);
      for (int i = j + 1 + t; i < n; i += 32) sm[j * ld + i] = ((i == pr) ? djj : sm[j * ld + i]) * r;
      if (t == 0) sm[j * ld + j] = piv;
    }
    __syncthreads();
    const int R = n - j - 1;
    if (R > 0) {
      int c = j + 1 + t / R, i = j + 1 + t % R;
      const int dc = T_ / R, di = T_ % R;
      while (c < n) {
        sm[c * ld + i] = fma(-sm[j * ld + i], sm[c * ld + j], sm[c * ld + i]);
        c += dc;
        i += di;
        if (i >= n) {
          i -= R;
          c++;
        }
      }
    }
    __syncthreads();
  }
  rows_store(sm, ld, n, n, D.p + b * D.stride, D);
  if (info && t == 0) info[b] = first_zero;
}

// ---------------------------------------------------------------------------
// Blocked getrf for orders above the one-CTA kernels' shared memory: per
// block column of width w (32), a tall panel factorization, the panel's row
// swaps applied to the other columns, U12 = L11^{-1} A12 and the trailing
// update A22 -= L21 U12 by the gemm_nn kernel (the blocked right-looking
// form of the same algorithm: the same pivot rule, applied column by column
// inside the panel).
// ---------------------------------------------------------------------------

// The m x w panel at (j0, j0) of D (rows j0.., columns j0..j0+w-1), one CTA
// per problem, T >= m threads: the steps of k_getrf_rows on a tall panel.
// Pivot rows go to ipiv as global rows (j0 + local row).  A zero pivot is
// left in place (no swap, no update).  info: the first panel (j0 = 0) sets
// it, a later one only records a zero pivot where none came before (the
// panels of a problem run in stream order).
__global__ void __launch_bounds__(512)
k_getrf_panel(int m, int w, int ld, int j0, OpW D, int *ipiv, long long sipiv, int *info) {
  extern __shared__ double sm[];
  __shared__ long long red_k[16];
  __shared__ double red_s[16];
  __shared__ int red_i[16];
  const int b = blockIdx.x, t = threadIdx.x, T_ = blockDim.x;
  const Op P{D.p, D.stride, D.cn, D.i0 + j0, D.j0 + j0};
  rows_load(sm, ld, m, w, P.p + b * P.stride, P);
  int first_zero = 0;
  for (int j = 0; j < w; j++) {
    const double x = (t >= j && t < m) ? sm[j * ld + t] : CUDART_NAN;
    const double djj = sm[j * ld + j];
    const long long key = pivot_key(x);
    double pv;
    const int p = cta_argmax_v(key, key >= 0 ? t : m, x, &pv, red_k, red_i, red_s);
    const bool keep = (p >= m) || pivot_key(djj) < 0;
    const int pr = keep ? j : p;
    const double piv = keep ? djj : pv;
    if (t == 0) ipiv[b * sipiv + j0 + j] = j0 + pr;
    if (is_zero(piv)) {
      if (first_zero == 0) first_zero = j0 + j + 1;
      __syncthreads();
      continue;
    }
    if (pr != j && t < w && t != j) {
      const double y = sm[t * ld + j];
      sm[t * ld + j] = sm[t * ld + pr];
      sm[t * ld + pr] = y;
    }
    if (t < 32) {
      const double r = recip3(piv);
      for (int i = j + 1 + t; i < m; i += 32) sm[j * ld + i] = ((i == pr) ? djj : sm[j * ld + i]) * r;
      if (t == 0) sm[j * ld + j] = piv;
    }
    __syncthreads();
    const int R = m - j - 1;
    if (R > 0 && j + 1 < w) {
      int c = j + 1 + t / R, i = j + 1 + t % R;
      const int dc = T_ / R, di = T_ % R;
      while (c < w) {
        sm[c * ld + i] = fma(-sm[j * ld + i], sm[c * ld + j], sm[c * ld + i]);
        c += dc;
        i += di;
        if (i >= m) {
          i -= R;
          c++;
        }
      }
    }
    __syncthreads();
  }
  rows_store(sm, ld, m, w, D.p + b * D.stride, OpW{D.p, D.stride, D.cn, D.i0 + j0, D.j0 + j0});
  if (info && t == 0 && (j0 == 0 || (first_zero != 0 && info[b] == 0))) info[b] = first_zero;
}

// The panel's row interchanges (rows j0+s and ipiv[j0+s], s < w, in order)
// applied to the n - w columns outside the panel, then, right of the panel,
// U12 = L11^{-1} A12 (L11 unit lower, w x w) by forward substitution.
//
// The w interchanges compose to a permutation of at most 2w rows: row
// mv_to[k] receives the old row mv_from[k].  Warp 0 forms it in registers
// (lane q holds positions q and 32 + q; a row is found by a ballot) and keeps
// the rows that move; the CTA applies it to the columns in chunks: every
// thread reads its elements of a chunk, the CTA synchronizes, every thread
// writes them -- independent loads instead of a chain of dependent swaps per
// column.  Then the solve, through shared memory (below); a column of L11
// whose pivot was exactly zero is skipped, as the unblocked factorization
// skips its update.
constexpr int SWAP_T = 128;
constexpr int SWAP_R = 8;  // elements per thread and chunk

__global__ void __launch_bounds__(SWAP_T)
k_getrf_swap_solve(int n, int w, int j0, OpW D, const int *ipiv, long long sipiv) {
  extern __shared__ double Xs[];  // 32 x SWAP_T
  __shared__ double L11[32 * 33];
  __shared__ int mv_to[64], mv_from[64];
  __shared__ int nz[32];
  __shared__ int n_mv;
  const int b = blockIdx.x, t = threadIdx.x;
  double *pd = D.p + (long long)b * D.stride;
  auto at = [&](int r, int c) -> double & { return pd[pm_off(D.i0 + r, D.j0 + c, D.cn)]; };
  if (t < 32) {
    const int lane = t;
    const int pvl = lane < w ? ipiv[b * sipiv + j0 + lane] : -1;
    int trA = lane < w ? j0 + lane : -1, srcA = trA, trB = -1, srcB = -1;
    int k = w;
    for (int s2 = 0; s2 < w; s2++) {
      const int p = __shfl_sync(FULL, pvl, s2);
      if (p == j0 + s2) continue;
      const unsigned mA = __ballot_sync(FULL, trA == p), mB = __ballot_sync(FULL, trB == p);
      int pos;
      if (mA) {
        pos = __ffs(mA) - 1;
      } else if (mB) {
        pos = 32 + __ffs(mB) - 1;
      } else {
        pos = k++;
        if (pos < 32 && lane == pos) trA = srcA = p;
        if (pos >= 32 && lane == pos - 32) trB = srcB = p;
      }
      const int vs = __shfl_sync(FULL, srcA, s2);
      const int vp = pos < 32 ? __shfl_sync(FULL, srcA, pos) : __shfl_sync(FULL, srcB, pos - 32);
      if (lane == s2) srcA = vp;
      if (pos < 32 && lane == pos) srcA = vs;
      if (pos >= 32 && lane == pos - 32) srcB = vs;
    }
    // compact the rows that move (source differs from destination)
    const bool mvA = trA >= 0 && srcA != trA, mvB = trB >= 0 && srcB != trB;
    const unsigned bA = __ballot_sync(FULL, mvA), bB = __ballot_sync(FULL, mvB);
    const unsigned below = (1u << lane) - 1u;
    if (mvA) {
      const int q = __popc(bA & below);
      mv_to[q] = trA;
      mv_from[q] = srcA;
    }
    if (mvB) {
      const int q = __popc(bA) + __popc(bB & below);
      mv_to[q] = trB;
      mv_from[q] = srcB;
    }
    if (lane == 0) n_mv = __popc(bA) + __popc(bB);
    if (lane < w) nz[lane] = !is_zero(at(j0 + lane, j0 + lane));
  }
  for (int e = t; e < w * w; e += SWAP_T) {
    const int r = e / w, c = e % w;
    L11[r * 33 + c] = r > c ? at(j0 + r, j0 + c) : 0.0;
  }
  __syncthreads();
  // chunks of whole columns (every moved row of a column in the same chunk,
  // so that no chunk reads an element an earlier one has written); columns
  // fastest within a chunk
  const int cols = n - w, nm = n_mv;
  const int cpc = nm > 0 ? (SWAP_T * SWAP_R) / nm : cols;
  for (int u0 = 0; nm > 0 && u0 < cols; u0 += cpc) {
    const int cc = min(cpc, cols - u0), total = cc * nm;
    double v[SWAP_R];
#pragma unroll
    for (int i = 0; i < SWAP_R; i++) {
      const int e = i * SWAP_T + t;
      if (e < total) {
        const int k = e / cc, u = u0 + e - k * cc;
        v[i] = at(mv_from[k], u < j0 ? u : u + w);
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < SWAP_R; i++) {
      const int e = i * SWAP_T + t;
      if (e < total) {
        const int k = e / cc, u = u0 + e - k * cc;
        at(mv_to[k], u < j0 ? u : u + w) = v[i];
      }
    }
    __syncthreads();
  }
  // U12 = L11^{-1} A12 in chunks of SWAP_T columns staged in shared memory
  // (row r of the chunk at Xs[r * SWAP_T + u]): loaded and stored with
  // consecutive threads on consecutive columns, solved by a thread per
  // column, four rows at a time (one load of x(l) feeds four FMAs).
  for (int c0 = j0 + w; c0 < n; c0 += SWAP_T) {
    const int cc = min(SWAP_T, n - c0);
    for (int e = t; e < w * cc; e += SWAP_T) {
      const int r = e / cc, u = e - r * cc;
      Xs[r * SWAP_T + u] = at(j0 + r, c0 + u);
    }
    __syncthreads();
    if (t < cc) {
      for (int r0 = 0; r0 < w; r0 += 4) {
        double acc[4];
#pragma unroll
        for (int q = 0; q < 4; q++) acc[q] = r0 + q < w ? Xs[(r0 + q) * SWAP_T + t] : 0.0;
#pragma unroll 2
        for (int l = 0; l < r0; l++) {
          if (nz[l]) {
            const double xl = Xs[l * SWAP_T + t];
#pragma unroll
            for (int q = 0; q < 4; q++) acc[q] = fma(-L11[(r0 + q) * 33 + l], xl, acc[q]);
          }
        }
        // the 4 x 4 diagonal block (rows past w are never stored)
#pragma unroll
        for (int q = 1; q < 4; q++)
#pragma unroll
          for (int l = 0; l < q; l++)
            if (r0 + q < w && nz[r0 + l]) acc[q] = fma(-L11[(r0 + q) * 33 + r0 + l], acc[l], acc[q]);
#pragma unroll
        for (int q = 0; q < 4; q++)
          if (r0 + q < w) Xs[(r0 + q) * SWAP_T + t] = acc[q];
      }
    }
    __syncthreads();
    for (int e = t; e < (w - 1) * cc; e += SWAP_T) {
      const int r = 1 + e / cc, u = e - (r - 1) * cc;
      at(j0 + r, c0 + u) = Xs[r * SWAP_T + u];
    }
    __syncthreads();
  }
}

// copy of the m x n sub-matrices C into D (the blocked factorizations work
// in place): problems along grid y, each problem's elements in panel-major
// order along x, so that consecutive threads touch consecutive doubles
__global__ void k_copy_sub(int batch, int m, int n, Op C, OpW D) {
  const int per = ((m + PS - 1) / PS) * PS * n;
  for (int b = blockIdx.y; b < batch; b += gridDim.y) {
    const double *pc = C.p + (long long)b * C.stride;
    double *pd = D.p + (long long)b * D.stride;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < per; x += gridDim.x * blockDim.x) {
      const int r4 = x & (PS - 1), q = x / PS, c = q % n, r = (q / n) * PS + r4;
      if (r < m) pd[pm_off(D.i0 + r, D.j0 + c, D.cn)] = pc[pm_off(C.i0 + r, C.j0 + c, C.cn)];
    }
  }
}

bool same_op(const Op &C, const OpW &D) {
  return C.p == D.p && C.stride == D.stride && C.cn == D.cn && C.i0 == D.i0 && C.j0 == D.j0;
}

void copy_sub(int batch, int m, int n, Op C, OpW D, cudaStream_t s) {
  const int per = ((m + PS - 1) / PS) * PS * n;
  k_copy_sub<<<dim3((per + 255) / 256, std::min(batch, 65535)), 256, 0, s>>>(batch, m, n, C, D);
}

// gelqf, one CTA per problem.  Per row i, two barriers:
//  (1) warp 0 forms beta, tau and 1/(alpha - beta) from alpha and the norm
//      of a(i, i+1:n) (computed ahead, see (2)), scales the row into the
//      reflector x and writes beta and tau.  An FP64 instruction costs the
//      same for 1 or 32 lanes, so the per-row scalar work stays on one warp;
//  (2) the rows below, each by a group of S lanes (S a power of two with
//      rows * S filling the CTA, so the lanes stay busy as the rows run out):
//      w = a(r, i) + a(r, i+1:n) . x by a strided partial sum and a shuffle
//      reduction within the group, then a(r, i:n) -= tau w [1, x].  The group
//      of row i+1 then sums the squares of its new a(i+1, i+2:n): the next
//      step's norm.
__device__ __forceinline__ double warp_row_norm2(const double *sm, int ld, int r, int c0, int n) {
  const int lane = threadIdx.x & 31;
  double part = 0.0;
  for (int c = c0 + lane; c < n; c += 32) part = fma(sm[c * ld + r], sm[c * ld + r], part);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(FULL, part, o);
  return part;
}

__global__ void __launch_bounds__(512)
k_gelqf_rows(int m, int n, int ld, Op C, OpW D, double *tau, long long stau) {
  extern __shared__ double sm[];
  __shared__ double sc[2];  // tau, norm of the next row
  const int b = blockIdx.x, t = threadIdx.x, T_ = blockDim.x;
  rows_load(sm, ld, m, n, C.p + b * C.stride, C);
  const int k = min(m, n);
  if (t < 32) {
    const double ss0 = warp_row_norm2(sm, ld, 0, 1, n);
    if (t == 0) sc[1] = ss0;
  }
  __syncthreads();
  for (int i = 0; i < k; i++) {
    if (t < 32) {
      const double ss = sc[1];
      const double alpha = sm[i * ld + i];
      double tv = 0.0;
      __syncwarp();
      if (!is_zero(ss)) {
        double beta, scal;
        reflector_scalars(alpha, ss, beta, tv, scal);
        for (int c = i + 1 + t; c < n; c += 32) sm[c * ld + i] *= scal;
        if (t == 0) sm[i * ld + i] = beta;
      }
      if (t == 0) {
        tau[b * stau + i] = tv;
        sc[0] = tv;
      }
    }
    __syncthreads();
    const double tv = sc[0];
    const int R = m - i - 1;
    if (!is_zero(tv) && R > 0) {
      int S = 1;
      while (S < 32 && 2 * S * R <= T_) S *= 2;
      const int sub = t & (S - 1), groups = T_ / S;
      const int iters = (R + groups - 1) / groups;  // same trip count on every lane
      for (int it = 0; it < iters; it++) {
        const int r = i + 1 + t / S + it * groups;
        const bool ok = r < m;
        double w = (ok && sub == 0) ? sm[i * ld + r] : 0.0;
        if (ok)
          for (int c = i + 1 + sub; c < n; c += S) w = fma(sm[c * ld + r], sm[c * ld + i], w);
        for (int o = 1; o < S; o <<= 1) w += __shfl_xor_sync(FULL, w, o);
        double nx = 0.0;
        if (ok) {
          const double tw = tv * w;
          if (sub == 0) sm[i * ld + r] -= tw;
          if (it == 0 && t < 32) {  // the warp of row i+1 (group 0): also the next norm
            for (int c = i + 1 + sub; c < n; c += S) {
              const double y = fma(-tw, sm[c * ld + i], sm[c * ld + r]);
              sm[c * ld + r] = y;
              if (c >= i + 2) nx = fma(y, y, nx);
            }
          } else {  // an FP64 instruction costs a warp the same for any active lanes:
                    // the other warps skip the squares
            for (int c = i + 1 + sub; c < n; c += S) sm[c * ld + r] = fma(-tw, sm[c * ld + i], sm[c * ld + r]);
          }
        }
        if (r == i + 1) {  // the first group only; its S lanes share r
          const unsigned gmask = (S == 32) ? FULL : (((1u << S) - 1u) << ((t & 31) & ~(S - 1)));
          for (int o = 1; o < S; o <<= 1) nx += __shfl_xor_sync(gmask, nx, o);
          if (sub == 0) sc[1] = nx;
        }
      }
    } else if (R > 0 && t < 32) {  // H_i = I: the next row is unchanged
      const double ss1 = warp_row_norm2(sm, ld, i + 1, i + 2, n);
      if (t == 0) sc[1] = ss1;
    }
    __syncthreads();
  }
  rows_store(sm, ld, m, n, D.p + b * D.stride, D);
}

// ---------------------------------------------------------------------------
// Blocked gelqf for the sizes above the one-CTA kernels' shared memory: per
// block of ib (<= 32) rows, the panel (rows i..i+ib-1, columns i..n-1) is
// factorized by k_gelqf_rows, then its ib reflectors are applied to the rows
// below at once, as the block reflector of the compact WY form (rowwise):
//     H_i H_{i+1} ... H_{i+ib-1} = I - V^T T V,
// V the ib x (n-i) reflector rows (unit leading entry, zeros before it), T
// upper triangular with T(j, j) = tau_j and T(0:j, j) = -tau_j T(0:j, 0:j)
// (V(0:j, :) v_j^T).  The rows below become A2 - ((A2 V^T) T) V: the same
// products as applying the reflectors one by one, in another order.
// ---------------------------------------------------------------------------
constexpr int LQ_T = 256;    // threads of the apply kernel
constexpr int LQ_RB = 32;    // rows of A2 per step
constexpr int LQ_RPC = 128;  // rows of A2 per CTA

size_t lq_apply_smem(int nb, int nc) {
  const int ldv = nc | 1;
  return ((size_t)nb * ldv + (size_t)(2 * nb + LQ_RB) * (nb + 1)) * sizeof(double);
}

// One row's columns c, c + 8, ..., c + 8(K-1) of A2 -= W V (columns past nc
// read a valid V entry and are not stored).
template <int K>
__device__ __forceinline__ void lq_update_chunk(double *arow, const double *wrow, const double *Vs, int ldv, int ib,
                                                int c, int nc) {
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; k++) acc[k] = c + 8 * k < nc ? arow[(c + 8 * k) * PS] : 0.0;
  for (int s = 0; s < ib; s++) {
    const double w = wrow[s];
#pragma unroll
    for (int k = 0; k < K; k++) acc[k] = fma(-w, Vs[s * ldv + min(c + 8 * k, nc - 1)], acc[k]);
  }
#pragma unroll
  for (int k = 0; k < K; k++)
    if (c + 8 * k < nc) arow[(c + 8 * k) * PS] = acc[k];
}

// The apply step for panel i (NB = 16 or 32 rows per panel): CTA (b, y)
// takes rows i+ib + [y*LQ_RPC, (y+1)*LQ_RPC) of problem b.  Shared memory:
// V (NB rows, those past ib zero), G = V V^T (upper), T (upper, zero
// elsewhere) and a W block.  Every CTA of a problem forms G and T itself (no
// workspace; NB/(8 rows) of the update's FMAs).  Thread layouts are chosen so that the
// shared-memory reads of V within a warp fall in distinct banks (V's row
// stride is odd).
template <int NB>
__global__ void __launch_bounds__(LQ_T)
k_gelqf_apply(int m, int n, int i, int ib, OpW D, const double *tau, long long stau) {
  constexpr int NQ = NB / 8;    // W columns per thread
  constexpr int LDT = NB + 1;  // row stride of G, T and W
  extern __shared__ double sh[];
  const int nc = n - i, ldv = nc | 1;
  double *Vs = sh;
  double *Gm = Vs + NB * ldv;
  double *Tm = Gm + NB * LDT;
  double *Wt = Tm + NB * LDT;
  const int b = blockIdx.x, t = threadIdx.x;
  double *pd = D.p + (long long)b * D.stride;
  auto at = [&](int r, int c) -> double & { return pd[pm_off(D.i0 + r, D.j0 + c, D.cn)]; };
  for (int e = t; e < NB * nc; e += LQ_T) {
    const int s = e / nc, c = e - s * nc;
    Vs[s * ldv + c] = (s >= ib || c < s) ? 0.0 : (c == s ? 1.0 : at(i + s, i + c));
  }
  __syncthreads();
  // G(a, q) = v_a . v_q for a < q < ib, pairs numbered by q so that a warp's
  // dot products have similar lengths; v_q is zero before column q
  const int npair = ib * (ib - 1) / 2;
  for (int p = t; p < npair; p += LQ_T) {
    int q = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)p)) * 0.5f);
    while (q * (q - 1) / 2 > p) q--;
    while ((q + 1) * q / 2 <= p) q++;
    const int a = p - q * (q - 1) / 2;
    double g0 = 0.0, g1 = 0.0;
    int c = q;
    for (; c + 1 < nc; c += 2) {
      g0 = fma(Vs[a * ldv + c], Vs[q * ldv + c], g0);
      g1 = fma(Vs[a * ldv + c + 1], Vs[q * ldv + c + 1], g1);
    }
    if (c < nc) g0 = fma(Vs[a * ldv + c], Vs[q * ldv + c], g0);
    Gm[a * LDT + q] = g0 + g1;
  }
  __syncthreads();
  // T, column by column on warp 0; lane a only reads the entries T(a, q) it
  // wrote itself, so the columns need no synchronization between lanes
  if (t < NB) {
    const double *tb = tau + b * stau + i;
    for (int j = 0; j < NB; j++) {
      if (j >= ib) {  // past the panel's reflectors: T zero (G is not formed there)
        Tm[t * LDT + j] = 0.0;
        continue;
      }
      const double tj = tb[j];
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      int q = t;
      for (; q + 3 < j; q += 4) {
        s0 = fma(Tm[t * LDT + q], Gm[q * LDT + j], s0);
        s1 = fma(Tm[t * LDT + q + 1], Gm[(q + 1) * LDT + j], s1);
        s2 = fma(Tm[t * LDT + q + 2], Gm[(q + 2) * LDT + j], s2);
        s3 = fma(Tm[t * LDT + q + 3], Gm[(q + 3) * LDT + j], s3);
      }
      for (; q < j; q++) s0 = fma(Tm[t * LDT + q], Gm[q * LDT + j], s0);
      Tm[t * LDT + j] = t < j ? -tj * ((s0 + s1) + (s2 + s3)) : (t == j ? tj : 0.0);
    }
  }
  __syncthreads();
  const int m2 = m - i - ib;
  const int rbeg = blockIdx.y * LQ_RPC, rend = min(m2, rbeg + LQ_RPC);
  const int wr = t >> 3, ws = t & 7;  // W(wr, ws + 8q), q < NQ
  for (int r0 = rbeg; r0 < rend; r0 += LQ_RB) {
    const int rows = min(LQ_RB, rend - r0);
    const int rg = i + ib + r0;  // first row of the block in the matrix
    // W = A2 V^T: the eight threads of a row read its entries straight from
    // global memory (one sector serves them), eight at a time ahead of use
    double w4[NQ];
#pragma unroll
    for (int q = 0; q < NQ; q++) w4[q] = 0.0;
    if (wr < rows) {
      const double *arow = pd + pm_off(D.i0 + rg + wr, D.j0 + i, D.cn);  // column c at arow + c * PS
      int c = 0;
      for (; c + 8 <= nc; c += 8) {
        double a[8];
#pragma unroll
        for (int k = 0; k < 8; k++) a[k] = arow[(c + k) * PS];
#pragma unroll
        for (int k = 0; k < 8; k++)
#pragma unroll
          for (int q = 0; q < NQ; q++) w4[q] = fma(a[k], Vs[(ws + 8 * q) * ldv + c + k], w4[q]);
      }
      for (; c < nc; c++) {
        const double a = arow[c * PS];
#pragma unroll
        for (int q = 0; q < NQ; q++) w4[q] = fma(a, Vs[(ws + 8 * q) * ldv + c], w4[q]);
      }
    }
    __syncthreads();  // the previous step's update has read Wt
#pragma unroll
    for (int q = 0; q < NQ; q++) Wt[wr * LDT + ws + 8 * q] = w4[q];
    __syncthreads();
    // W <- W T (T upper: W T(:, s) sums W(:, 0..s))
    double u4[NQ];
#pragma unroll
    for (int q = 0; q < NQ; q++) u4[q] = 0.0;
    for (int q2 = 0; q2 < NB; q2++) {
      const double wq = Wt[wr * LDT + q2];
#pragma unroll
      for (int q = 0; q < NQ; q++) u4[q] = fma(wq, Tm[q2 * LDT + ws + 8 * q], u4[q]);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NQ; q++) Wt[wr * LDT + ws + 8 * q] = u4[q];
    __syncthreads();
    // A2 <- A2 - W V, thread (row ur, columns uc + 8k of each chunk of 64);
    // the last chunk runs only the column groups it has (a warp-uniform
    // count), so a narrow tail issues no FMAs on padding columns
    const int ur = t >> 3, uc = t & 7;
    if (ur < rows) {
      double *arow = pd + pm_off(D.i0 + rg + ur, D.j0 + i, D.cn);  // column c at arow + c * PS
      for (int c0 = 0; c0 < nc; c0 += 64) {
        switch (min(8, (nc - c0 + 7) >> 3)) {
          case 8: lq_update_chunk<8>(arow, Wt + ur * LDT, Vs, ldv, ib, c0 + uc, nc); break;
          case 7: lq_update_chunk<7>(arow, Wt + ur * LDT, Vs, ldv, ib, c0 + uc, nc); break;
          case 6: lq_update_chunk<6>(arow, Wt + ur * LDT, Vs, ldv, ib, c0 + uc, nc); break;
          case 5: lq_update_chunk<5>(arow, Wt + ur * LDT, Vs, ldv, ib, c0 + uc, nc); break;
          case 4: lq_update_chunk<4>(arow, Wt + ur * LDT, Vs, ldv, ib, c0 + uc, nc); break;
          case 3: lq_update_chunk<3>(arow, Wt + ur * LDT, Vs, ldv, ib, c0 + uc, nc); break;
          case 2: lq_update_chunk<2>(arow, Wt + ur * LDT, Vs, ldv, ib, c0 + uc, nc); break;
          default: lq_update_chunk<1>(arow, Wt + ur * LDT, Vs, ldv, ib, c0 + uc, nc); break;
        }
      }
    }
  }
}

// Lanes per problem of the one-warp kernels: the smallest G whose matrices
// for the warp's 32/G problems fit 20 KB (many resident warps per SM hide the
// latency of the per-column pivot and reciprocal); else one problem per warp.
int pick_g(size_t bytes_per_problem) {
  for (int g = 1; g <= 32; g *= 2)
    if (bytes_per_problem * (32 / g) <= 20 * 1024) return g;
  return 32;
}

// Rows from which the one-CTA-per-problem kernels are used (measured on
// square sweeps: the one-warp kernels win up to n = 32 for getrf, where the
// row kernel's per-column barriers dominate, and up to n = 64 for gelqf).
#ifndef BF_LU_ROWS_MIN
#define BF_LU_ROWS_MIN 48
#endif
#ifndef BF_LQ_ROWS_MIN
#define BF_LQ_ROWS_MIN 65
#endif
// Threads of the row kernels for the largest matrices (one CTA per SM fits
// by shared memory there, so the CTA itself must bring the warps).
#ifndef BF_LU_BIG_THREADS
#define BF_LU_BIG_THREADS 256
#endif
constexpr int LU_BIG_THREADS = BF_LU_BIG_THREADS;
// Orders from which the rule takes the blocked forms (measured on square
// sweeps: getrf blocked by 32 columns and gelqf blocked by 16 rows win from
// n = 96, the one-CTA forms at n = 64).
#ifndef BF_LQ_BLOCKED_MIN
#define BF_LQ_BLOCKED_MIN 96
#endif
#ifndef BF_LU_BLOCKED_MIN_N
#define BF_LU_BLOCKED_MIN_N 96
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

int getrf_layout_rule(int batch, int n) {
  (void)batch;
  if (n < BF_LU_ROWS_MIN) return LAYOUT_LU_WARP;
  return n < BF_LU_BLOCKED_MIN_N ? LAYOUT_LU_ROWS : LAYOUT_LU_BLOCKED;
}

bool getrf_layout_ok(int layout, int n) {
  switch (layout) {
    case LAYOUT_LU_WARP: case LAYOUT_LU_ROWS: return n <= LU_ONE_CTA_MAX_N;
    case LAYOUT_LU_BLOCKED: case LAYOUT_LU_BLOCKED16: return n <= GETRF_MAX_N;
    default: return false;
  }
}

namespace {

// Blocked getrf: for each block column j0 (width w = nb, 16 or 32, the last
// one narrower) the panel factorization, the panel's swaps on the other columns
// with U12 = L11^{-1} A12, and the trailing update A22 <- A22 - L21 U12 by
// the gemm_nn kernel; in place in D (C copied there first unless the two
// coincide).  Each launch covers the whole batch.
cudaError_t launch_getrf_blocked(int nb, int batch, int n, Op C, OpW D, int *ipiv, long long sipiv, int *info,
                                 cudaStream_t s) {
  if (!same_op(C, D)) copy_sub(batch, n, n, C, D, s);
  const bool aligned = (D.i0 % PS) == 0 && (D.stride % 2) == 0 && ((uintptr_t)D.p % 16) == 0;
  for (int j0 = 0; j0 < n; j0 += nb) {
    const int w = std::min(nb, n - j0), m = n - j0, ld = m | 1;
    const size_t smem = (size_t)ld * w * sizeof(double);
    cudaError_t e = set_smem((const void *)k_getrf_panel, smem);
    if (e != cudaSuccess) return e;
    k_getrf_panel<<<batch, std::max(64, (m + 31) / 32 * 32), smem, s>>>(m, w, ld, j0, D, ipiv, sipiv, info);
    if (n > w) {
      const size_t xs = (size_t)32 * SWAP_T * sizeof(double);
      e = set_smem((const void *)k_getrf_swap_solve, xs);
      if (e != cudaSuccess) return e;
      k_getrf_swap_solve<<<batch, SWAP_T, xs, s>>>(n, w, j0, D, ipiv, sipiv);
    }
    const int r = m - w;
    if (r > 0) {
      e = launch_gemm_nn(false, batch, r, r, w, -1.0, Op{D.p, D.stride, D.cn, D.i0 + j0 + w, D.j0 + j0},
                         Op{D.p, D.stride, D.cn, D.i0 + j0, D.j0 + j0 + w}, 1.0,
                         Op{D.p, D.stride, D.cn, D.i0 + j0 + w, D.j0 + j0 + w},
                         OpW{D.p, D.stride, D.cn, D.i0 + j0 + w, D.j0 + j0 + w}, aligned, s);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_getrf(int batch, int n, Op C, OpW D, int *ipiv, long long sipiv, int *info, cudaStream_t s) {
  const int forced = layout_forced(ROUTINE_GETRF, n, batch);
  const int lay = (forced > 0 && getrf_layout_ok(forced, n)) ? forced : getrf_layout_rule(batch, n);
  if (lay == LAYOUT_LU_BLOCKED) return launch_getrf_blocked(32, batch, n, C, D, ipiv, sipiv, info, s);
  if (lay == LAYOUT_LU_BLOCKED16) return launch_getrf_blocked(16, batch, n, C, D, ipiv, sipiv, info, s);
  if (lay == LAYOUT_LU_ROWS) {
    const int ld = n | 1;
    const size_t smem = (size_t)ld * n * sizeof(double);
    cudaError_t e = set_smem((const void *)k_getrf_rows, smem);
    if (e != cudaSuccess) return e;
    const int T = std::max(n > 96 ? LU_BIG_THREADS : (n > 64 ? 256 : 128), (n + 31) / 32 * 32);
    k_getrf_rows<<<batch, T, smem, s>>>(n, ld, C, D, ipiv, sipiv, info);
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

int gelqf_layout_rule(int batch, int m, int n) {
  (void)batch;
  if ((long long)m * n > GELQF_ONE_CTA_MAX_MN || (m >= BF_LQ_BLOCKED_MIN && n >= BF_LQ_BLOCKED_MIN))
    return LAYOUT_LQ_BLOCKED16;
  return m < BF_LQ_ROWS_MIN ? LAYOUT_LQ_WARP : LAYOUT_LQ_ROWS;
}

bool gelqf_layout_ok(int layout, int m, int n) {
  switch (layout) {
    case LAYOUT_LQ_WARP: case LAYOUT_LQ_ROWS: return (long long)m * n <= GELQF_ONE_CTA_MAX_MN;
    case LAYOUT_LQ_BLOCKED: case LAYOUT_LQ_BLOCKED16: return m <= GELQF_MAX_DIM && n <= GELQF_MAX_DIM;
    default: return false;
  }
}

namespace {

// Blocked gelqf: per block of nb (16 or 32) rows the panel by k_gelqf_rows, then
// the block reflector applied to the rows below by k_gelqf_apply; in place
// in D (C copied there first unless the two coincide).
cudaError_t launch_gelqf_blocked(int nb, int batch, int m, int n, Op C, OpW D, double *tau, long long stau,
                                 cudaStream_t s) {
  if (!same_op(C, D)) copy_sub(batch, m, n, C, D, s);
  const int k = std::min(m, n);
  for (int i = 0; i < k; i += nb) {
    const int ib = std::min(nb, k - i), nc = n - i, ld = ib | 1;
    const size_t smem = (size_t)ld * nc * sizeof(double);
    cudaError_t e = set_smem((const void *)k_gelqf_rows, smem);
    if (e != cudaSuccess) return e;
    const long long mn = (long long)ib * nc;
    k_gelqf_rows<<<batch, mn > 9216 ? LU_BIG_THREADS : (mn > 4096 ? 256 : 128), smem, s>>>(
        ib, nc, ld, Op{D.p, D.stride, D.cn, D.i0 + i, D.j0 + i}, OpW{D.p, D.stride, D.cn, D.i0 + i, D.j0 + i},
        tau + i, stau);
    const int m2 = m - i - ib;
    if (m2 > 0) {
      const size_t sa = lq_apply_smem(nb, nc);
      const dim3 grid(batch, (m2 + LQ_RPC - 1) / LQ_RPC);
      if (nb == 16) {
        e = set_smem((const void *)k_gelqf_apply<16>, sa);
        if (e != cudaSuccess) return e;
        k_gelqf_apply<16><<<grid, LQ_T, sa, s>>>(m, n, i, ib, D, tau, stau);
      } else {
        e = set_smem((const void *)k_gelqf_apply<32>, sa);
        if (e != cudaSuccess) return e;
        k_gelqf_apply<32><<<grid, LQ_T, sa, s>>>(m, n, i, ib, D, tau, stau);
      }
    }
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gelqf(int batch, int m, int n, Op C, OpW D, double *tau, long long stau, cudaStream_t s) {
  const int forced = layout_forced(ROUTINE_GELQF, n, batch);
  const int lay = (forced > 0 && gelqf_layout_ok(forced, m, n)) ? forced : gelqf_layout_rule(batch, m, n);
  if (lay == LAYOUT_LQ_BLOCKED) return launch_gelqf_blocked(32, batch, m, n, C, D, tau, stau, s);
  if (lay == LAYOUT_LQ_BLOCKED16) return launch_gelqf_blocked(16, batch, m, n, C, D, tau, stau, s);
  if (lay == LAYOUT_LQ_ROWS) {
    const int ld = m | 1;
    const size_t smem = (size_t)ld * n * sizeof(double);
    cudaError_t e = set_smem((const void *)k_gelqf_rows, smem);
    if (e != cudaSuccess) return e;
    k_gelqf_rows<<<batch, (size_t)m * n > 9216 ? LU_BIG_THREADS : ((size_t)m * n > 4096 ? 256 : 128), smem, s>>>(
        m, n, ld, C, D, tau, stau);
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
