// potrf_l and the fused syrk_potrf_ln, batched, FP64, panel-major operands.
//
// potrf_l (Sec. 5.2.2, Sec. 4.6):         lower(D) <- chol(C)
// syrk_potrf_ln (Sec. 4.7.2, Sec. 5.3):   lower(D) <- chol(C + A * B^T)
//
// The paper builds the factorization from kernels on register-resident
// blocks, keeps 1/L[j][j] for later solves (Sec. 4.7.1) and, for
// syrk_potrf, adds the A*B^T update inside the same kernel so that the sum is
// never stored and reloaded (Sec. 4.7.2).  Both ideas carry over; what
// changes on GB300 is where the lanes go.  A warp-wide FP64 instruction costs
// the same with 1 or 32 active lanes, and the per-column square root and
// reciprocal cost several FMAs each, so the sequential part of a small
// Cholesky must be shared by many problems at once.  Three kernels:
//
//  k_chol_tiny (n <= 8, when the batch gives one lane per problem at least
//    one warp per SM sub-partition): one lane per problem, the whole
//    triangle in registers, factored right-looking with compile-time indices.
//
//  k_chol_small (n <= 31): a warp holds Q = 32/G problems, G lanes per
//    problem.  The lower triangles live packed in shared memory, problem q's
//    element e at sm[e*Q' + q], Q' = Q + 1 for Q >= 16: the odd pitch puts
//    the elements that the load and store phases copy for one problem (lanes
//    along e) in distinct banks, as it does the G rows read at once in the
//    factorization.  The factorization runs column by column
//    (Cholesky-Crout); the pivot's rsqrt is one warp instruction for all Q
//    problems.  For syrk_potrf the A*B^T sum is added in 4x4 register blocks
//    straight into the shared-memory triangle before the factorization.
//
//  k_chol_rows4 / k_chol_rows2 / k_chol_rows (n <= 512): one thread per row,
//    blocks of BW columns held in registers, P problems per CTA, a warp
//    holding 32/P rows of each: P = 4 with BW = 8 for n = 32..96, P = 2 with
//    BW = 16 up to n = 256, P = 1 above.  With P*BW = 32 the diagonal block
//    of a block column is one full warp, which computes only the block's
//    lower triangle, spread evenly over its lanes.  For block column
//    [c0, c0+BW):
//      (a) acc = C[i][c0..]  (+ A[i][:] * B[c0..][:]^T for syrk_potrf)
//      (b) acc -= L[i][0:c0] * L[c0..][0:c0]^T            (gemm_nt downdate)
//      (c) the lanes of rows c0..c0+BW-1 factor the diagonal block in
//          registers with warp shuffles (potrf_l kernel on a register block)
//      (d) the rows below solve against it (trsm_rltn kernel)
//    The operand rows shared by a problem's threads, B[c0..][l..] and
//    L[c0..][l..], are staged 32 columns at a time in shared memory and read
//    as broadcasts.
//
// Non-SPD input: the first column j whose pivot is not > 0 (NaN included)
// sets info = j+1; the arithmetic continues on NaNs without branching, so the
// columns >= j are unspecified and no other problem is affected.
#include "bf_internal.cuh"

namespace bf {
namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ void tri_index(int t, int &tr, int &tc) {
  int r = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
  while (r * (r + 1) / 2 > t) r--;
  while ((r + 1) * (r + 2) / 2 <= t) r++;
  tr = r;
  tc = t - r * (r + 1) / 2;
}


// packed lower column-major: column l starts at cs(l); element (i, l) at cs(l) + i
__device__ __forceinline__ int col_start(int l, int n) { return (l * (2 * n - l + 1)) / 2 - l; }

// ---------------------------------------------------------------------------
// k_chol_small
// ---------------------------------------------------------------------------
#ifndef BF_SMALL_PAD
#define BF_SMALL_PAD 1
#endif
// The pad applies from 16 problems per warp (G <= 2), where the copies'
// conflicts were worst (potrf n = 16: 523 -> 579 GFLOP/s); with 8 or 4
// problems per warp the extra shared memory cost more resident warps than
// the conflicts (n = 24: 649 -> 631 padded).
#ifndef BF_SMALL_PAD_MINQ
#define BF_SMALL_PAD_MINQ 16
#endif
// problem pitch of the shared-memory triangles of k_chol_small
__host__ __device__ constexpr int small_pitch(int q) { return q + ((q >= BF_SMALL_PAD_MINQ) ? BF_SMALL_PAD : 0); }
template <int G, bool FUSED, bool ALIGNED>
__global__ void __launch_bounds__(32)
k_chol_small(int batch, int n, int k, Op A, Op B, Op C, OpW D, double *dinv, long long sdinv,
             int *info) {
  constexpr int Q = 32 / G;
  constexpr int QP = small_pitch(Q);
  extern __shared__ double sm[];
  const int lane = threadIdx.x;
  const int q = lane / G, s = lane % G;
  const int b0 = blockIdx.x * Q;
  const int b = b0 + q;
  const bool valid = b < batch;

  // ---- phase 1: lower triangle of C into shared memory (whole warp per
  // problem).  Asynchronous 8-byte copies: every lane issues all of its
  // copies for all Q problems before waiting once, so the global latency is
  // paid once per CTA instead of once per panel.
  for (int qq = 0; qq < Q; qq++) {
    const int bb = b0 + qq;
    if (bb >= batch) break;
    const double *pc = C.p + bb * C.stride;
    if (ALIGNED) {
      for (int p = 0; p * PS < n; p++) {
        const int ncol = min(n, p * PS + PS);
        const double *pp = pc + (long long)(C.i0 + p * PS) * C.cn + (long long)C.j0 * PS;
        for (int x = lane; x < ncol * PS; x += 32) {
          const int j = x / PS, i = p * PS + (x % PS);
          if (i < n && i >= j) cp_async8(&sm[(col_start(j, n) + i) * QP + qq], pp + x);
        }
      }
    } else {
      for (int x = lane; x < n * n; x += 32) {
        const int j = x / n, i = x - j * n;
        if (i >= j) cp_async8(&sm[(col_start(j, n) + i) * QP + qq], pc + pm_off(C.i0 + i, C.j0 + j, C.cn));
      }
    }
  }
  cp_async_wait_all();
  __syncwarp();

  // ---- syrk_potrf: add A*B^T in 4x4 register blocks of the lower block triangle
  if (FUSED && valid) {
    const double *pa = A.p + b * A.stride;
    const double *pb = B.p + b * B.stride;
    const int TR = (n + 3) / 4;
    const int ntiles = TR * (TR + 1) / 2;
    for (int t = s; t < ntiles; t += G) {
      int tr, tc;
      tri_index(t, tr, tc);
      const int i0 = tr * 4, j0 = tc * 4;
      double acc[4][4];
#pragma unroll
      for (int r = 0; r < 4; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) acc[r][c] = 0.0;
      if (ALIGNED) {
        const double *ap = pa + (long long)(A.i0 + i0) * A.cn + (long long)A.j0 * PS;
        const double *bp = pb + (long long)(B.i0 + j0) * B.cn + (long long)B.j0 * PS;
#pragma unroll 4
        for (int l = 0; l < k; l++) {
          const double2 a01 = __ldg((const double2 *)(ap + l * PS));
          const double2 a23 = __ldg((const double2 *)(ap + l * PS + 2));
          const double2 b01 = __ldg((const double2 *)(bp + l * PS));
          const double2 b23 = __ldg((const double2 *)(bp + l * PS + 2));
          const double av[4] = {a01.x, a01.y, a23.x, a23.y};
          const double bv[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
          for (int r = 0; r < 4; r++)
#pragma unroll
            for (int c = 0; c < 4; c++) acc[r][c] = fma(av[r], bv[c], acc[r][c]);
        }
      } else {
        const double *ar[4], *br[4];
#pragma unroll
        for (int r = 0; r < 4; r++) {
          ar[r] = pa + pm_off(A.i0 + min(i0 + r, n - 1), A.j0, A.cn);
          br[r] = pb + pm_off(B.i0 + min(j0 + r, n - 1), B.j0, B.cn);
        }
        for (int l = 0; l < k; l++) {
          double av[4], bv[4];
#pragma unroll
          for (int r = 0; r < 4; r++) {
            av[r] = __ldg(ar[r] + l * PS);
            bv[r] = __ldg(br[r] + l * PS);
          }
#pragma unroll
          for (int r = 0; r < 4; r++)
#pragma unroll
            for (int c = 0; c < 4; c++) acc[r][c] = fma(av[r], bv[c], acc[r][c]);
        }
      }
#pragma unroll
      for (int r = 0; r < 4; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) {
          const int i = i0 + r, j = j0 + c;
          if (i < n && i >= j) sm[(col_start(j, n) + i) * QP + q] += acc[r][c];
        }
    }
  }
  __syncwarp();

  // ---- phase 2: Cholesky-Crout, column by column; row i belongs to sub-lane i % G
  int first_bad = 0;
  for (int j = 0; j < n; j++) {
    const int cj = col_start(j, n);
    const int istart = j + ((s - (j % G)) + G) % G;
    double dval = 0.0;
    int i = istart;
    // four rows at a time share the loads of row j
    for (; i + 3 * G < n; i += 4 * G) {
      double a0 = sm[(cj + i) * QP + q], a1 = sm[(cj + i + G) * QP + q];
      double a2 = sm[(cj + i + 2 * G) * QP + q], a3 = sm[(cj + i + 3 * G) * QP + q];
      int cl = 0;
      for (int l = 0; l < j; l++) {
        const double ljl = sm[(cl + j) * QP + q];
        a0 = fma(-sm[(cl + i) * QP + q], ljl, a0);
        a1 = fma(-sm[(cl + i + G) * QP + q], ljl, a1);
        a2 = fma(-sm[(cl + i + 2 * G) * QP + q], ljl, a2);
        a3 = fma(-sm[(cl + i + 3 * G) * QP + q], ljl, a3);
        cl += n - l - 1;
      }
      if (i == j) dval = a0;
      sm[(cj + i) * QP + q] = a0;
      sm[(cj + i + G) * QP + q] = a1;
      sm[(cj + i + 2 * G) * QP + q] = a2;
      sm[(cj + i + 3 * G) * QP + q] = a3;
    }
    for (; i < n; i += G) {
      double a0 = sm[(cj + i) * QP + q];
      int cl = 0;
      for (int l = 0; l < j; l++) {
        a0 = fma(-sm[(cl + i) * QP + q], sm[(cl + j) * QP + q], a0);
        cl += n - l - 1;
      }
      if (i == j) dval = a0;
      sm[(cj + i) * QP + q] = a0;
    }
    // pivot of problem q comes from its sub-lane that owns row j
    const double d = (G == 1) ? dval : __shfl_sync(FULL, dval, q * G + (j % G));
    const double r = rsqrt(d);
    if (first_bad == 0 && not_positive(d)) first_bad = j + 1;
    // the pivot's own entry holds d, so one product serves every row (no
    // divergent second FP64 instruction for the pivot row)
    for (int ii = istart; ii < n; ii += G) sm[(cj + ii) * QP + q] *= r;
    if (dinv && valid && s == (j % G)) dinv[b * sdinv + j] = r;
    __syncwarp();
  }

  // ---- phase 3: lower triangle back to D (whole warp per problem)
  for (int qq = 0; qq < Q; qq++) {
    const int bb = b0 + qq;
    if (bb >= batch) break;
    double *pd = D.p + bb * D.stride;
    if (ALIGNED) {
      for (int p = 0; p * PS < n; p++) {
        const int ncol = min(n, p * PS + PS);
        double *pp = pd + (long long)(D.i0 + p * PS) * D.cn + (long long)D.j0 * PS;
        for (int x = lane; x < ncol * PS; x += 32) {
          const int j = x / PS, i = p * PS + (x % PS);
          if (i < n && i >= j) pp[x] = sm[(col_start(j, n) + i) * QP + qq];
        }
      }
    } else {
      for (int x = lane; x < n * n; x += 32) {
        const int j = x / n, i = x - j * n;
        if (i >= j) pd[pm_off(D.i0 + i, D.j0 + j, D.cn)] = sm[(col_start(j, n) + i) * QP + qq];
      }
    }
  }
  if (info && valid && s == 0) info[b] = first_bad;
}

// ---------------------------------------------------------------------------
// k_chol_tiny (n <= 8): one lane per problem, the whole triangle in registers
// ---------------------------------------------------------------------------
// With 32 problems per warp every FP64 instruction does useful work for 32
// problems, the pivot's rsqrt included, and there is no shared memory to
// stage through: each lane reads its own problem's lower triangle (pairs of
// rows of a column are one 16-byte load when the operands are aligned),
// factors it right-looking with compile-time indices, and writes the lower
// triangle back.

// element (i, j) of an operand whose top row is a panel top (i0 % PS == 0)
__device__ __forceinline__ long long tiny_off(int i, int j, int cn) {
  return (long long)(i & ~(PS - 1)) * cn + (long long)j * PS + (i & (PS - 1));
}

template <int N, bool ALIGNED>
__device__ __forceinline__ void tiny_load_lower(double (&c)[N][N], const double *p, const Op &o) {
  if (ALIGNED) {
    const double *base = p + (long long)o.i0 * o.cn + (long long)o.j0 * PS;
#pragma unroll
    for (int j = 0; j < N; j++)
#pragma unroll
      for (int i = j; i < N; i++) {
        if ((i & 1) == 0 && i + 1 < N) {
          const double2 v = __ldg((const double2 *)(base + tiny_off(i, j, o.cn)));
          c[i][j] = v.x;
          c[i + 1][j] = v.y;
        } else if (!((i & 1) == 1 && i - 1 >= j)) {
          c[i][j] = __ldg(base + tiny_off(i, j, o.cn));
        }
      }
  } else {
#pragma unroll
    for (int j = 0; j < N; j++)
#pragma unroll
      for (int i = j; i < N; i++) c[i][j] = __ldg(p + pm_off(o.i0 + i, o.j0 + j, o.cn));
  }
}

// row l-column of an N x k operand: v[i] = X(i, l)
template <int N, bool ALIGNED>
__device__ __forceinline__ void tiny_load_col(double (&v)[N], const double *p, const Op &o, int l) {
  if (ALIGNED) {
    const double *base = p + (long long)o.i0 * o.cn + (long long)(o.j0 + l) * PS;
#pragma unroll
    for (int i = 0; i < N; i++) {
      if ((i & 1) == 0 && i + 1 < N) {
        const double2 x = __ldg((const double2 *)(base + tiny_off(i, 0, o.cn)));
        v[i] = x.x;
        v[i + 1] = x.y;
      } else if ((i & 1) == 0) {
        v[i] = __ldg(base + tiny_off(i, 0, o.cn));
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; i++) v[i] = __ldg(p + pm_off(o.i0 + i, o.j0 + l, o.cn));
  }
}

template <int N, bool FUSED, bool ALIGNED>
__global__ void __launch_bounds__(128)
k_chol_tiny(int batch, int k, Op A, Op B, Op C, OpW D, double *dinv, long long sdinv, int *info) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  double c[N][N];
  tiny_load_lower<N, ALIGNED>(c, C.p + (long long)b * C.stride, C);
  if (FUSED) {
    const double *pa = A.p + (long long)b * A.stride, *pb = B.p + (long long)b * B.stride;
#pragma unroll 2
    for (int l = 0; l < k; l++) {
      double av[N], bv[N];
      tiny_load_col<N, ALIGNED>(av, pa, A, l);
      tiny_load_col<N, ALIGNED>(bv, pb, B, l);
#pragma unroll
      for (int j = 0; j < N; j++)
#pragma unroll
        for (int i = j; i < N; i++) c[i][j] = fma(av[i], bv[j], c[i][j]);
    }
  }
  int bad = 0;
  double *dv = dinv ? dinv + (long long)b * sdinv : nullptr;
#pragma unroll
  for (int j = 0; j < N; j++) {
    const double d = c[j][j];
    const double r = rsqrt(d);
    if (bad == 0 && not_positive(d)) bad = j + 1;
    c[j][j] = d * r;
    if (dv) dv[j] = r;
#pragma unroll
    for (int i = j + 1; i < N; i++) c[i][j] *= r;
#pragma unroll
    for (int jj = j + 1; jj < N; jj++)
#pragma unroll
      for (int i = jj; i < N; i++) c[i][jj] = fma(-c[i][j], c[jj][j], c[i][jj]);
  }
  double *pd = D.p + (long long)b * D.stride;
  if (ALIGNED) {
    double *base = pd + (long long)D.i0 * D.cn + (long long)D.j0 * PS;
#pragma unroll
    for (int j = 0; j < N; j++)
#pragma unroll
      for (int i = j; i < N; i++) {
        if ((i & 1) == 0 && i + 1 < N) {
          *(double2 *)(base + tiny_off(i, j, D.cn)) = make_double2(c[i][j], c[i + 1][j]);
        } else if (!((i & 1) == 1 && i - 1 >= j)) {
          base[tiny_off(i, j, D.cn)] = c[i][j];
        }
      }
  } else {
#pragma unroll
    for (int j = 0; j < N; j++)
#pragma unroll
      for (int i = j; i < N; i++) pd[pm_off(D.i0 + i, D.j0 + j, D.cn)] = c[i][j];
  }
  if (info) info[b] = bad;
}

// ---------------------------------------------------------------------------
// k_chol_rows
// ---------------------------------------------------------------------------
constexpr int KC = 32;  // columns per staged chunk

// Compute type of the row kernel: double for the library routines, float
// for the single-precision factor of the mixed-precision solver.
template <typename T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }

template <typename T, int BW, int P>
struct __align__(16) RowsSmem {
  T stage[P][KC][BW + 2];  // stage[p][ll][jj]: row c0+jj, column l0+ll of problem p's shared
                           // operand (even pitch: pairs (jj, jj+1) are one vector load)
  T Ls[P][BW][BW + 1];     // diagonal block of L: Ls[p][jj][j]
  T rinv[P][BW];
  int bad[P];
};

// Two problems per CTA (RowMap<2>) up to these orders.  The CTA of 2n
// threads must leave room for two CTAs per SM, or the FP64 pipes idle while
// one warp factors a diagonal block: at n = 256 that caps registers at 64.
// Measured at n = 256: potrf 910 -> 1000 GFLOP/s; syrk_potrf 969 -> 938
// before the diagonal warp's triangle split, 968 -> 988 with it.
#ifndef BF_ROWS_P2_MAX_N
#define BF_ROWS_P2_MAX_N 256
#endif
#ifndef BF_ROWS_SPLIT
#define BF_ROWS_SPLIT 1  // balanced triangle split of the diagonal warp's k-loops
#endif
// The split in the descriptor-array kernel's one-problem CTAs, in the blocks
// whose diagonal half-warp has an idle partner (c0 % 32 == 16).  Not in
// k_chol_rows: there the extra registers (70 -> 118) cost a resident CTA,
// measured 1019 -> 984 GFLOP/s at syrk_potrf n = 256 (the tail launch).
#ifndef BF_ROWS_SPLIT_P1
#define BF_ROWS_SPLIT_P1 1
#endif
#ifndef BF_ROWS_P2_FP32
#define BF_ROWS_P2_FP32 0
#endif
#ifndef BF_ROWS_P2_MAX_N_FUSED
#define BF_ROWS_P2_MAX_N_FUSED 256
#endif

// 64 < n <= 128: the two-problem kernel built for 4 CTAs of 256 threads per
// SM (64 registers) rather than 2 of 384 (78-80 registers), so that more
// CTAs keep the FP64 pipe fed while one factors a diagonal block.  Measured:
// potrf n = 96 968 -> 998, n = 128 1018 -> 1061; syrk_potrf n = 128
// 1101 -> 1118 GFLOP/s; at n = 48 and 64 it was 0.5-1% slower.
// Resident CTAs per SM that each build of the two-problem kernel is
// compiled for (its register bound: 65536 / (threads x CTAs)).  More CTAs
// keep the FP64 pipe fed while one factors a diagonal block; fewer registers
// slow the k-loops.  Measured (GFLOP/s):
//   n <= 64,  128 threads: 6 CTAs (80 registers); 8 (64) was 0.5-1% slower
//   n <= 128, 256 threads: 4 (64) against 3 (80): potrf n = 96 968 -> 998,
//                          n = 128 1018 -> 1061; syrk_potrf n = 128 1101 -> 1118
//   n <= 192, 384 threads: 3 (56, some spills) against 2 (78-80): potrf
//                          n = 144 911 -> 1052, n = 192 1041 -> 1103;
//                          syrk_potrf n = 144 1041 -> 1129, n = 192 1125 -> 1157
//   n <= 256, 512 threads: 2 (64)
// Orders factored four problems per CTA (k_chol_rows4), per routine, in
// builds of 256 threads x 4 CTAs per SM (n <= 64) and 384 x 3 (n <= 96).
// Measured against the small kernel below and the two-problem kernel above
// (GFLOP/s, potrf / syrk_potrf):
//   n = 32: 626 -> 730 / 849 -> 1024     n = 48: 709 -> 896 / 1013 -> 1097
//   n = 40: 593 -> 821 / 892 -> 1065     n = 64: 853 -> 979 / 1088 -> 1136
//   n = 72: 713 -> 1009 / 899 -> 1112    n = 88: 789 -> 1022 / 941 -> 1097
//   n = 96: 1001 -> 1058 / 1144 -> 1152
// At n = 112 it ties and at n = 128 the two-problem kernel is 4% faster (at
// 512 threads, 2 CTAs per SM); below 32 the small kernel is faster (n = 28:
// 596 against 490, n = 16: 578 against 371).
#ifndef BF_ROWS_P4_MIN_N
#define BF_ROWS_P4_MIN_N 32
#endif
#ifndef BF_ROWS_P4_MAX_N
#define BF_ROWS_P4_MAX_N 96
#endif
#ifndef BF_ROWS_P4_MIN_N_FUSED
#define BF_ROWS_P4_MIN_N_FUSED 32
#endif
#ifndef BF_ROWS_P4_MAX_N_FUSED
#define BF_ROWS_P4_MAX_N_FUSED 96
#endif
#ifndef BF_ROWS_P4_MINB256
#define BF_ROWS_P4_MINB256 4
#endif
#ifndef BF_ROWS_P4_MINB384
#define BF_ROWS_P4_MINB384 3
#endif
#ifndef BF_ROWS_P2_MINB128
#define BF_ROWS_P2_MINB128 6
#endif
#ifndef BF_ROWS_P2_MINB256
#define BF_ROWS_P2_MINB256 4
#endif
#ifndef BF_ROWS_P2_MINB384
#define BF_ROWS_P2_MINB384 3
#endif

#ifndef BF_ROWS_KUNROLL
#define BF_ROWS_KUNROLL 4
#endif
constexpr int ROWS_KUNROLL = BF_ROWS_KUNROLL;  // unroll of the syrk k-loop

// Thread -> (problem, row) map of the row kernel.  A warp holds RPW = 32/P
// consecutive rows of each of the CTA's P problems: lanes [p*RPW, (p+1)*RPW)
// are rows g*RPW .. g*RPW + RPW-1 of problem p, g the warp index.  With P = 2
// and 16-column blocks the rows of a block's diagonal block fill one whole
// warp (16 lanes per problem), so the diagonal factorization and the rows
// below it never issue with idle lanes.
template <int P>
struct RowMap {
  static constexpr int RPW = 32 / P;
  int lane, p, i;
  __device__ __forceinline__ RowMap() {
    lane = threadIdx.x & 31;
    p = lane / RPW;
    i = (threadIdx.x >> 5) * RPW + (lane % RPW);
  }
};

// Balanced split of a BW x BW lower triangle over BW lanes, H = BW/2: lane s
// takes row s up to column min(s, H), and lanes s <= H - 2 also take row
// BW-1-s from column H+1 on.  Slot m (0..H) of lane s is entry (row, col);
// lanes below H use slots 0..H-1, the others 0..H.  For BW = 16 that is at
// most 9 entries a lane for the triangle's 136 (8.5 on average); for BW = 8,
// 5 for 36.
template <int BW>
__device__ __forceinline__ void split_slot(int s, int m, int &row, int &col, bool &valid) {
  constexpr int H = BW / 2;
  if (s >= H || m <= s) {
    row = s;
    col = m;
    valid = m <= s;
  } else {
    row = BW - 1 - s;
    col = H + m - s;
    valid = m <= H - 1;
  }
}

// One block column [c0, c0 + BW) of the factorization.  W is the number of
// accumulators (the block's width rounded up to a multiple of 8).  The
// diagonal block's rows c0..c0+BW-1 of problem p are lanes
// p*RPW + c0%RPW + (0..BW-1) of warp c0/RPW (BW divides RPW and c0 is a
// multiple of BW).
template <int W, int BW, int P, bool FUSED, bool ALIGNED, typename T, bool S1>
__device__ __forceinline__ void rows_block(RowsSmem<T, BW, P> &S, const RowMap<P> &rm, int c0, int n, int k,
                                           int b0, int batch, bool me_valid, const double *pa, const double *pc,
                                           T *pd, Op A, Op B, Op C, OpWT<T> D, T *dinv, long long sdinv) {
  using T2 = typename Vec2<T>::type;
  constexpr int RPW = RowMap<P>::RPW;
  const int t = threadIdx.x;
  const int T_ = blockDim.x;
  const int i = rm.i, p = rm.p;
  const int w = min(BW, n - c0);
  const bool active = me_valid && (i < n) && (i >= c0);
  T acc[W];
  // Two problems per CTA, full 16-column block: the warp of the diagonal
  // block (16 rows of each problem) computes only the block's lower triangle
  // in (a') and (b), spread over its lanes by split_slot: at most 9 FMAs per
  // step a lane instead of 16.  Its rows are gathered back before (c).
  // With one problem per CTA the diagonal block fills half a warp; the split
  // applies when the other half holds rows above the block (c0 % 32 == 16),
  // which then idle, and only the diagonal half scatters its slots.
  constexpr int H = BW / 2, NSLOT = H + 1;
  constexpr bool SPLIT = BF_ROWS_SPLIT && (P * BW == 32 || (P == 1 && BW == 16 && S1)) && W == BW && BW >= 8;
  const bool dwarp = SPLIT && ((t >> 5) == c0 / RPW) && (P > 1 || c0 % 32 == 16);  // warp-uniform
  const bool dhalf = P > 1 || (rm.lane >> 4) == 1;  // a lane of the diagonal block (in a split warp)
  const int sb = rm.lane & (BW - 1);                    // row within the diagonal block

  // (a) C[i][c0 + jj] for the lower part of the block column.  The diagonal
  // warp keeps its 9 triangle slots in acc[0..8] until it gathers its rows,
  // and adds C then.
#pragma unroll
  for (int jj = 0; jj < W; jj++) {
    const int col = c0 + jj;
    acc[jj] = (!dwarp && active && jj < w && i >= col) ? (T)pc[pm_off(C.i0 + i, C.j0 + col, C.cn)] : (T)0;
  }

  // (a') syrk_potrf: += A[i][:] * B[c0..c0+w)[:]^T, B rows staged per chunk
  if (FUSED) {
    const double *arow = pa + pm_off(A.i0 + min(i, n - 1), A.j0, A.cn);
    for (int l0 = 0; l0 < k; l0 += KC) {
      const int kc = min(KC, k - l0);
      __syncthreads();
      for (int x = t; x < P * BW * KC; x += T_) {
        const int px = x / (BW * KC), xr = x - px * (BW * KC);
        const int r4 = xr % PS, ll = (xr / PS) % KC, pnl = xr / (PS * KC);
        const int jj = pnl * PS + r4;
        S.stage[px][ll][jj] =
            (b0 + px < batch && jj < w && ll < kc)
                ? (T)__ldg(B.p + (long long)(b0 + px) * B.stride + pm_off(B.i0 + c0 + jj, B.j0 + l0 + ll, B.cn))
                : (T)0;
      }
      __syncthreads();
      if (dwarp) {
        const int ro = BW - 1 - sb, smax = min(sb, H);  // slots m <= smax are on the lane's own row
        const bool own_ok = me_valid && sb < w, oth_ok = me_valid && sb <= H - 2 && ro < w;
        const double *arow_o = pa + pm_off(A.i0 + min(c0 + ro, n - 1), A.j0, A.cn);
        const int obase = max(0, H - sb);  // other-row slot m reads column H + m - sb
        for (int ll = 0; ll < kc; ll++) {
          const T xo = own_ok ? (T)__ldg(arow + (long long)(l0 + ll) * PS) : (T)0;
          const T xt = oth_ok ? (T)__ldg(arow_o + (long long)(l0 + ll) * PS) : (T)0;
          const T *st = S.stage[p][ll];
#pragma unroll
          for (int m = 0; m < NSLOT; m++) {
            const bool own = m <= smax;
            acc[m] = fma_t(own ? xo : xt, own ? st[m] : st[min(obase + m, BW - 1)], acc[m]);
          }
        }
      } else if (active) {
#pragma unroll ROWS_KUNROLL
        for (int ll = 0; ll < kc; ll++) {
          const T x = (T)__ldg(arow + (long long)(l0 + ll) * PS);
#pragma unroll
          for (int jj = 0; jj < W; jj += 2) {
            const T2 bv = *(const T2 *)&S.stage[p][ll][jj];
            acc[jj] = fma_t(x, bv.x, acc[jj]);
            if (jj + 1 < W) acc[jj + 1] = fma_t(x, bv.y, acc[jj + 1]);
          }
        }
      }
    }
  }

  // (b) downdate with the columns of L already computed: -= L[i][0:c0] L[c0..][0:c0]^T
  {
    const T *lrow = pd + pm_off(D.i0 + min(i, n - 1), D.j0, D.cn);
    for (int l0 = 0; l0 < c0; l0 += KC) {
      const int kc = min(KC, c0 - l0);
      __syncthreads();
      for (int x = t; x < P * BW * KC; x += T_) {
        const int px = x / (BW * KC), xr = x - px * (BW * KC);
        const int r4 = xr % PS, ll = (xr / PS) % KC, pnl = xr / (PS * KC);
        const int jj = pnl * PS + r4;
        S.stage[px][ll][jj] =
            (b0 + px < batch && jj < w && ll < kc)
                ? D.p[(long long)(b0 + px) * D.stride + pm_off(D.i0 + c0 + jj, D.j0 + l0 + ll, D.cn)]
                : (T)0;
      }
      __syncthreads();
      if (dwarp) {
        const int smax = min(sb, H), obase = max(0, H - sb);
        for (int ll = 0; ll < kc; ll++) {
          const T *st = S.stage[p][ll];
          const T xo = st[sb], xt = st[BW - 1 - sb];
#pragma unroll
          for (int m = 0; m < NSLOT; m++) {
            const bool own = m <= smax;
            acc[m] = fma_t(-(own ? xo : xt), own ? st[m] : st[min(obase + m, BW - 1)], acc[m]);
          }
        }
      } else if (active) {
#pragma unroll 2
        for (int ll = 0; ll < kc; ll++) {
          const T x = lrow[(long long)(l0 + ll) * PS];
#pragma unroll
          for (int jj = 0; jj < W; jj += 2) {
            const T2 lv = *(const T2 *)&S.stage[p][ll][jj];
            acc[jj] = fma_t(-x, lv.x, acc[jj]);
            if (jj + 1 < W) acc[jj + 1] = fma_t(-x, lv.y, acc[jj + 1]);
          }
        }
      }
    }
  }

  // the diagonal warp: slots to shared memory, then each lane its row, plus C
  if (dwarp) {
#pragma unroll
    for (int m = 0; m < NSLOT; m++) {
      int row, col;
      bool ok;
      split_slot<BW>(sb, m, row, col, ok);
      if (ok && dhalf) S.Ls[p][row][col] = acc[m];
    }
    __syncwarp();
#pragma unroll
    for (int jj = 0; jj < W; jj++) {
      const bool lower = jj <= sb;
      const T cv = (me_valid && dhalf && sb < w && jj < w && lower) ? (T)pc[pm_off(C.i0 + i, C.j0 + c0 + jj, C.cn)]
                                                                      : (T)0;
      acc[jj] = cv + (lower ? S.Ls[p][sb][jj] : (T)0);
    }
    __syncwarp();
  }

  // (c) diagonal block: its rows are lanes base..base+BW-1 of one warp, which
  // factor it in registers with shuffles among themselves
  const int base = p * RPW + (c0 % RPW);
  const int dl = rm.lane - base;
  if ((t >> 5) == c0 / RPW && dl >= 0 && dl < BW) {
    const unsigned dmask = (BW * P == 32) ? FULL : (((1u << BW) - 1u) << base);
    int bad = 0;  // every diagonal lane sees every pivot and tracks the first bad one
    // all W columns: padding columns (j >= w) hold zeros and only feed other
    // padding columns, which are never stored
#pragma unroll
    for (int j = 0; j < W; j++) {
      const T d = __shfl_sync(dmask, acc[j], base + j);
      const T r = rsqrt_t(d);
      if (j < w && bad == 0 && not_positive(d)) bad = c0 + j + 1;
      // lane j's own acc[j] is d: one product for every lane gives its
      // L_jj = d r and the others' entries, with no divergent FP64 branch
      acc[j] *= r;
      if (dl == j) S.rinv[p][j] = r;
#pragma unroll
      for (int jj = j + 1; jj < W; jj++) {
        const T v = __shfl_sync(dmask, acc[j], base + jj);
        acc[jj] = fma_t(-acc[j], v, acc[jj]);
      }
    }
#pragma unroll
    for (int jj = 0; jj < W; jj++) S.Ls[p][dl][jj] = acc[jj];
    if (dl == 0 && bad != 0 && S.bad[p] == 0) S.bad[p] = bad;
  }
  __syncthreads();

  // (d) rows below the diagonal block: substitution against it
  if (active && i >= c0 + BW) {
#pragma unroll
    for (int j = 0; j < W; j++) {
      acc[j] *= S.rinv[p][j];
#pragma unroll
      for (int jj = j + 1; jj < W; jj++) acc[jj] = fma_t(-acc[j], S.Ls[p][jj][j], acc[jj]);
    }
  }

  // (e) store the block column
  if (active) {
    T *drow = pd + pm_off(D.i0 + i, D.j0, D.cn);
#pragma unroll
    for (int jj = 0; jj < W; jj++) {
      const int col = c0 + jj;
      if (jj < w && i >= col) drow[(long long)col * PS] = acc[jj];
    }
  }
  if (t < P * BW) {
    const int px = t / BW, j = t - px * BW;
    if (dinv && b0 + px < batch && j < w) dinv[(long long)(b0 + px) * sdinv + c0 + j] = S.rinv[px][j];
  }
  __syncthreads();
}

// CTA = P problems of the batch (problems blockIdx.x*P + p), threads laid out
// by RowMap<P>.  Problems past the end of the batch (last CTA) run along
// without touching memory.
template <int BW, int P, bool FUSED, bool ALIGNED, typename T, bool S1 = false>
__device__ __forceinline__ void chol_rows_body(int b0, int batch, int n, int k, Op A, Op B, Op C, OpWT<T> D,
                                               T *dinv, long long sdinv, int *info) {
  __shared__ RowsSmem<T, BW, P> S;
  const RowMap<P> rm;
  const bool me_valid = b0 + rm.p < batch;
  const long long bme = me_valid ? b0 + rm.p : b0;  // lanes of a missing problem alias the first
  const double *pa = FUSED ? A.p + bme * A.stride : nullptr;
  const double *pc = C.p + bme * C.stride;
  T *pd = D.p + bme * D.stride;
  if (threadIdx.x < P) S.bad[threadIdx.x] = 0;
  __syncthreads();
  for (int c0 = 0; c0 < n; c0 += BW) {
    if constexpr (BW == 4) {
      rows_block<4, 4, P, FUSED, ALIGNED, T, S1>(S, rm, c0, n, k, b0, batch, me_valid, pa, pc, pd, A, B, C, D,
                                                 dinv, sdinv);
    } else if constexpr (BW == 8) {
      rows_block<8, 8, P, FUSED, ALIGNED, T, S1>(S, rm, c0, n, k, b0, batch, me_valid, pa, pc, pd, A, B, C, D,
                                                 dinv, sdinv);
    } else {
      const int w8 = (min(BW, n - c0) + 7) & ~7;
      if (w8 == 8)
        rows_block<8, BW, P, FUSED, ALIGNED, T, S1>(S, rm, c0, n, k, b0, batch, me_valid, pa, pc, pd, A, B, C, D,
                                                    dinv, sdinv);
      else
        rows_block<16, BW, P, FUSED, ALIGNED, T, S1>(S, rm, c0, n, k, b0, batch, me_valid, pa, pc, pd, A, B, C, D,
                                                     dinv, sdinv);
    }
  }
  if (info && threadIdx.x < P && b0 + (int)threadIdx.x < batch) info[b0 + threadIdx.x] = S.bad[threadIdx.x];
}

// One problem per CTA, up to 512 rows.
template <int BW, bool FUSED, bool ALIGNED, typename T>
__global__ void __launch_bounds__(512)
k_chol_rows(int batch, int n, int k, Op A, Op B, Op C, OpWT<T> D, T *dinv, long long sdinv, int *info) {
  chol_rows_body<BW, 1, FUSED, ALIGNED, T>(blockIdx.x, batch, n, k, A, B, C, D, dinv, sdinv, info);
}

// Two problems per CTA, up to MAXT/2 rows; registers bounded so that MINB
// CTAs of MAXT threads fit an SM.
template <int BW, bool FUSED, bool ALIGNED, typename T, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB)
k_chol_rows2(int batch, int n, int k, Op A, Op B, Op C, OpWT<T> D, T *dinv, long long sdinv, int *info) {
  chol_rows_body<BW, 2, FUSED, ALIGNED, T>(blockIdx.x * 2, batch, n, k, A, B, C, D, dinv, sdinv, info);
}

// Four problems per CTA with 8-column blocks: a warp holds 8 rows of each
// of four problems, so each rsqrt and shuffle step of a diagonal block's
// factorization serves four problems instead of two.  Up to MAXT/4 rows.
template <bool FUSED, bool ALIGNED, typename T, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB)
k_chol_rows4(int batch, int n, int k, Op A, Op B, Op C, OpWT<T> D, T *dinv, long long sdinv, int *info) {
  chol_rows_body<8, 4, FUSED, ALIGNED, T>(blockIdx.x * 4, batch, n, k, A, B, C, D, dinv, sdinv, info);
}

// Eight problems per CTA with 4-column blocks: a warp holds 4 rows of each
// of eight problems, so the diagonal block's rsqrt, pivot test and scaling
// serve eight problems per warp instruction, at one block column (and its
// barriers) per four columns.  Up to MAXT/8 rows.
template <bool FUSED, bool ALIGNED, typename T, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB)
k_chol_rows8(int batch, int n, int k, Op A, Op B, Op C, OpWT<T> D, T *dinv, long long sdinv, int *info) {
  chol_rows_body<4, 8, FUSED, ALIGNED, T>(blockIdx.x * 8, batch, n, k, A, B, C, D, dinv, sdinv, info);
}

// Descriptor-array form: CTA b factors problem b of its own order (rows past
// it idle), after checking the problem's record.  AFTER_SYRK: the second
// launch of syrk_potrf in two launches (the syrk kernel has formed
// C + A B^T in D): the record is checked with the fused routine's rules, as
// the syrk launch checked it, and D is factored in place.
// With `order`, CTA q takes record order[q], and only when its order m lies
// in (lo, hi] (or, with report_bad, when its sizes are out of range): the
// one-problem class of the ordered form.
template <int BW, bool FUSED, bool AFTER_SYRK = false>
__global__ void __launch_bounds__(512)
k_chol_rows_v(int batch, const bf_dsize *size, const bf_dsub *A, const bf_dsub *B, const bf_dsub *C,
              const bf_dsub *D, int want_dinv, int *info, int max_m, int *status, const int *order = nullptr,
              int lo = -1, int hi = CHOL_MAX_N, int report_bad = 1) {
  constexpr bool REC = FUSED || AFTER_SYRK;  // the record has the fused operands
  if ((int)blockIdx.x >= batch) return;
  const int b = order ? order[blockIdx.x] : (int)blockIdx.x;
  if (b < 0 || b >= batch) return;
  const int m = size[b].m, k = REC ? size[b].k : 0;
  const bool sized = m >= 0 && k >= 0 && m <= max_m;
  if (sized ? !(m > lo && m <= hi) : report_bad == 0) return;  // another class's record
  int err = 0;
  if (!sized)
    err = -1;
  else if (m > 0) {
    if (REC && k > 0 && !dsub_ok(A[b], m, k))
      err = -2;
    else if (REC && k > 0 && !dsub_ok(B[b], m, k))
      err = -3;
    else if (!dsub_ok(C[b], m, m))
      err = REC ? -4 : -2;
    else if (!dsub_ok(D[b], m, m))
      err = REC ? -5 : -3;
  }
  if (threadIdx.x == 0 && status) status[b] = err;
  if (err != 0) return;
  if (m == 0) {
    if (threadIdx.x == 0 && info) info[b] = 0;
    return;
  }
  const Op c = AFTER_SYRK ? dsub_op(D[b]) : dsub_op(C[b]);
  const Op a = (FUSED && k > 0) ? dsub_op(A[b]) : c;  // k == 0: A and B are never read
  const Op bb = (FUSED && k > 0) ? dsub_op(B[b]) : c;
  const OpW d = dsub_opw(D[b]);
  // the inverse-diagonal array holds min(m, n) entries of its matrix
  const bf_dmat &dm = D[b].mat;
  double *dv = (want_dinv && dm.dA && D[b].j + m <= min(dm.m, dm.n)) ? dm.dA + D[b].j : nullptr;
  chol_rows_body<BW, 1, FUSED, false, double, BF_ROWS_SPLIT_P1 != 0>(0, 1, m, k, a, bb, c, d, dv, 0,
                                                                    info ? info + b : nullptr);
}

// ---------------------------------------------------------------------------
// Descriptor-array Cholesky with P problems per CTA, the records taken in a
// given order -- best by decreasing size, so that the problems sharing a CTA
// have similar orders.  Each problem keeps its own sizes and operands; the
// CTA runs its block columns to the largest order among its problems, and a
// problem's rows idle once it is done.  The steps are those of rows_block,
// with the diagonal warp's triangle split (the warp holds BW = 32/P rows of
// each problem's diagonal block).  On GB300 an FP64 warp instruction costs
// the same with 1 or 32 active lanes, and one problem per CTA leaves a
// problem's last warp partly empty; with P problems of similar order per
// CTA a warp carries 32/P rows of each.
// ---------------------------------------------------------------------------

// One problem of a CTA (n = 0: an empty slot).
struct VProb {
  const double *a, *b, *c;
  double *d, *dinv;
  int ai, aj, acn, bi, bj, bcn, ci, cj, ccn, di, dj, dcn;
  int n, k;
};

template <int W, int BW, int P, bool FUSED>
__device__ __forceinline__ void rows_block_vp(RowsSmem<double, BW, P> &S, const VProb *V, const RowMap<P> &rm,
                                              int c0, int kmax) {
  constexpr int RPW = RowMap<P>::RPW;
  const int t = threadIdx.x, T_ = blockDim.x;
  const int i = rm.i, p = rm.p;
  const VProb &me = V[p];
  const int n = me.n;
  const int w = min(BW, n - c0);
  const bool active = i < n && i >= c0;
  const int ir = min(i, max(n - 1, 0));  // a row to address (read only when active)
  double acc[W];
  // The warp of the diagonal blocks (BW rows of each of the P problems, a
  // full warp) computes only the blocks' lower triangles in (a') and (b),
  // spread over its lanes by split_slot, and gathers its rows before (c), as
  // the strided kernels do.
  constexpr int H = BW / 2, NSLOT = H + 1;
  constexpr bool SPLIT = BF_ROWS_SPLIT && W == BW && BW >= 8;
  const bool dwarp = SPLIT && (t >> 5) == c0 / RPW;  // warp-uniform
  const int sb = rm.lane & (BW - 1);                 // row within the diagonal block

  // (a) C[i][c0 + jj] on and below the diagonal (the diagonal warp adds C
  // when it gathers its rows)
#pragma unroll
  for (int jj = 0; jj < W; jj++) {
    const int col = c0 + jj;
    acc[jj] = (!dwarp && active && jj < w && i >= col) ? me.c[pm_off(me.ci + i, me.cj + col, me.ccn)] : 0.0;
  }

  // (a') syrk_potrf: += A[i][:] B[c0..c0+w)[:]^T, B rows of every problem staged per chunk
  if (FUSED) {
    const double *arow = me.a + pm_off(me.ai + ir, me.aj, me.acn);
    for (int l0 = 0; l0 < kmax; l0 += KC) {
      const int kc = min(KC, kmax - l0);
      __syncthreads();
      for (int x = t; x < P * BW * KC; x += T_) {
        const int px = x / (BW * KC), xr = x - px * (BW * KC);
        const int r4 = xr % PS, ll = (xr / PS) % KC, pnl = xr / (PS * KC);
        const int jj = pnl * PS + r4;
        const VProb &q = V[px];
        S.stage[px][ll][jj] = (jj < q.n - c0 && ll < kc && ll < q.k - l0)
                                  ? __ldg(q.b + pm_off(q.bi + c0 + jj, q.bj + l0 + ll, q.bcn))
                                  : 0.0;
      }
      __syncthreads();
      const int kme = min(kc, me.k - l0);
      if (dwarp) {
        const int ro = BW - 1 - sb, smax = min(sb, H);  // slots m <= smax are on the lane's own row
        const bool own_ok = sb < w, oth_ok = sb <= H - 2 && ro < w;
        const double *arow_o = me.a + pm_off(me.ai + min(c0 + ro, max(n - 1, 0)), me.aj, me.acn);
        const int obase = max(0, H - sb);  // other-row slot m reads column H + m - sb
        for (int ll = 0; ll < kme; ll++) {
          const double xo = own_ok ? __ldg(arow + (long long)(l0 + ll) * PS) : 0.0;
          const double xt = oth_ok ? __ldg(arow_o + (long long)(l0 + ll) * PS) : 0.0;
          const double *st = S.stage[p][ll];
#pragma unroll
          for (int m = 0; m < NSLOT; m++) {
            const bool own = m <= smax;
            acc[m] = fma(own ? xo : xt, own ? st[m] : st[min(obase + m, BW - 1)], acc[m]);
          }
        }
      } else if (active) {
        for (int ll = 0; ll < kme; ll++) {
          const double x = __ldg(arow + (long long)(l0 + ll) * PS);
#pragma unroll
          for (int jj = 0; jj < W; jj += 2) {
            const double2 bv = *(const double2 *)&S.stage[p][ll][jj];
            acc[jj] = fma(x, bv.x, acc[jj]);
            if (jj + 1 < W) acc[jj + 1] = fma(x, bv.y, acc[jj + 1]);
          }
        }
      }
    }
  }

  // (b) downdate with the columns of L already computed
  {
    const double *lrow = me.d + pm_off(me.di + ir, me.dj, me.dcn);
    for (int l0 = 0; l0 < c0; l0 += KC) {
      const int kc = min(KC, c0 - l0);
      __syncthreads();
      for (int x = t; x < P * BW * KC; x += T_) {
        const int px = x / (BW * KC), xr = x - px * (BW * KC);
        const int r4 = xr % PS, ll = (xr / PS) % KC, pnl = xr / (PS * KC);
        const int jj = pnl * PS + r4;
        const VProb &q = V[px];
        S.stage[px][ll][jj] =
            (jj < q.n - c0 && ll < kc) ? q.d[pm_off(q.di + c0 + jj, q.dj + l0 + ll, q.dcn)] : 0.0;
      }
      __syncthreads();
      if (dwarp) {
        const int smax = min(sb, H), obase = max(0, H - sb);
        for (int ll = 0; ll < kc; ll++) {
          const double *st = S.stage[p][ll];
          const double xo = st[sb], xt = st[BW - 1 - sb];
#pragma unroll
          for (int m = 0; m < NSLOT; m++) {
            const bool own = m <= smax;
            acc[m] = fma(-(own ? xo : xt), own ? st[m] : st[min(obase + m, BW - 1)], acc[m]);
          }
        }
      } else if (active) {
#pragma unroll 2
        for (int ll = 0; ll < kc; ll++) {
          const double x = lrow[(long long)(l0 + ll) * PS];
#pragma unroll
          for (int jj = 0; jj < W; jj += 2) {
            const double2 lv = *(const double2 *)&S.stage[p][ll][jj];
            acc[jj] = fma(-x, lv.x, acc[jj]);
            if (jj + 1 < W) acc[jj + 1] = fma(-x, lv.y, acc[jj + 1]);
          }
        }
      }
    }
  }

  // the diagonal warp: slots to shared memory, then each lane its row, plus C
  if (dwarp) {
#pragma unroll
    for (int m = 0; m < NSLOT; m++) {
      int row, col;
      bool ok;
      split_slot<BW>(sb, m, row, col, ok);
      if (ok) S.Ls[p][row][col] = acc[m];
    }
    __syncwarp();
#pragma unroll
    for (int jj = 0; jj < W; jj++) {
      const bool lower = jj <= sb;
      const double cv =
          (sb < w && jj < w && lower) ? me.c[pm_off(me.ci + c0 + sb, me.cj + c0 + jj, me.ccn)] : 0.0;
      acc[jj] = cv + (lower ? S.Ls[p][sb][jj] : 0.0);
    }
    __syncwarp();
  }

  // (c) diagonal blocks: problem p's rows c0..c0+BW-1 are lanes
  // p*RPW + (0..BW-1) of warp c0/RPW (BW == RPW), factored in registers
  const int base = p * RPW + (c0 % RPW);
  const int dl = rm.lane - base;
  if ((t >> 5) == c0 / RPW && dl >= 0 && dl < BW) {
    int bad = 0;
#pragma unroll
    for (int j = 0; j < W; j++) {
      const double d = __shfl_sync(0xffffffffu, acc[j], base + j);
      const double r = rsqrt(d);
      if (j < w && bad == 0 && not_positive(d)) bad = c0 + j + 1;
      // lane j's own acc[j] is d: one product for every lane gives its
      // L_jj = d r and the others' entries, with no divergent FP64 branch
      acc[j] *= r;
      if (dl == j) S.rinv[p][j] = r;
#pragma unroll
      for (int jj = j + 1; jj < W; jj++) {
        const double v = __shfl_sync(0xffffffffu, acc[j], base + jj);
        acc[jj] = fma(-acc[j], v, acc[jj]);
      }
    }
#pragma unroll
    for (int jj = 0; jj < W; jj++) S.Ls[p][dl][jj] = acc[jj];
    if (dl == 0 && bad != 0 && S.bad[p] == 0) S.bad[p] = bad;
  }
  __syncthreads();

  // (d) rows below the diagonal block
  if (active && i >= c0 + BW) {
#pragma unroll
    for (int j = 0; j < W; j++) {
      acc[j] *= S.rinv[p][j];
#pragma unroll
      for (int jj = j + 1; jj < W; jj++) acc[jj] = fma(-acc[j], S.Ls[p][jj][j], acc[jj]);
    }
  }

  // (e) store the block column, and 1/L_jj
  if (active) {
    double *drow = me.d + pm_off(me.di + i, me.dj, me.dcn);
#pragma unroll
    for (int jj = 0; jj < W; jj++) {
      const int col = c0 + jj;
      if (jj < w && i >= col) drow[(long long)col * PS] = acc[jj];
    }
  }
  if (t < P * BW) {
    const int px = t / BW, j = t - px * BW;
    const VProb &q = V[px];
    if (q.dinv && j < q.n - c0) q.dinv[c0 + j] = S.rinv[px][j];
  }
  __syncthreads();
}

// CTA b takes the records at positions P*b .. P*b + P-1 of `order` (NULL:
// the records themselves), and of those the ones whose order m lies in
// (lo, hi]; the launch with report_bad set also reports the records whose
// sizes are out of range.  Records are checked as in k_chol_rows_v.
template <int P, int BW, bool FUSED, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB)
k_chol_rows_vp(int batch, const int *order, const bf_dsize *size, const bf_dsub *A, const bf_dsub *B,
               const bf_dsub *C, const bf_dsub *D, int want_dinv, int *info, int max_m, int *status, int lo,
               int hi, int report_bad) {
  static_assert(BW == 32 / P, "a warp holds one diagonal block of each problem");
  __shared__ RowsSmem<double, BW, P> S;
  __shared__ VProb V[P];
  __shared__ int rec[P];
  const RowMap<P> rm;
  const int t = threadIdx.x;
  if (t < P) {
    const long long pos = (long long)blockIdx.x * P + t;
    VProb v{};
    int r = -1;
    if (pos < batch) {
      r = order ? order[pos] : (int)pos;
      if (r < 0 || r >= batch) r = -1;
    }
    int use = -1;
    if (r >= 0) {
      const int m = size[r].m, k = FUSED ? size[r].k : 0;
      const bool sized = m >= 0 && m <= max_m && k >= 0;
      if (sized ? (m > lo && m <= hi) : report_bad != 0) {
        int err = sized ? 0 : -1;
        if (err == 0 && m > 0) {
          if (FUSED && k > 0 && !dsub_ok(A[r], m, k))
            err = -2;
          else if (FUSED && k > 0 && !dsub_ok(B[r], m, k))
            err = -3;
          else if (!dsub_ok(C[r], m, m))
            err = FUSED ? -4 : -2;
          else if (!dsub_ok(D[r], m, m))
            err = FUSED ? -5 : -3;
        }
        if (status) status[r] = err;
        if (err == 0 && m == 0 && info) info[r] = 0;
        if (err == 0 && m > 0) {
          const bf_dsub &c = C[r], &d = D[r];
          const bf_dsub &a = (FUSED && k > 0) ? A[r] : c;  // k == 0: A and B are never read
          const bf_dsub &bb = (FUSED && k > 0) ? B[r] : c;
          v.a = a.mat.pA; v.ai = a.i; v.aj = a.j; v.acn = a.mat.cn;
          v.b = bb.mat.pA; v.bi = bb.i; v.bj = bb.j; v.bcn = bb.mat.cn;
          v.c = c.mat.pA; v.ci = c.i; v.cj = c.j; v.ccn = c.mat.cn;
          v.d = d.mat.pA; v.di = d.i; v.dj = d.j; v.dcn = d.mat.cn;
          // the inverse-diagonal array holds min(m, n) entries of its matrix
          v.dinv = (want_dinv && d.mat.dA && d.j + m <= min(d.mat.m, d.mat.n)) ? d.mat.dA + d.j : nullptr;
          v.n = m;
          v.k = k;
          use = r;
        }
      }
    }
    V[t] = v;
    rec[t] = use;
    S.bad[t] = 0;
  }
  __syncthreads();
  int nmax = 0, kmax = 0;
#pragma unroll
  for (int q = 0; q < P; q++) {
    nmax = max(nmax, V[q].n);
    kmax = max(kmax, V[q].k);
  }
  if (nmax == 0) return;  // CTA-uniform
  for (int c0 = 0; c0 < nmax; c0 += BW) {
    if constexpr (BW == 8) {
      rows_block_vp<8, 8, P, FUSED>(S, V, rm, c0, kmax);
    } else {
      if (min(BW, nmax - c0) <= 8)
        rows_block_vp<8, BW, P, FUSED>(S, V, rm, c0, kmax);
      else
        rows_block_vp<16, BW, P, FUSED>(S, V, rm, c0, kmax);
    }
  }
  if (info && t < P && rec[t] >= 0) info[rec[t]] = S.bad[t];
}

// Counting sort of the records by decreasing order m, on one CTA: a
// histogram over the keys, the running offsets from the largest key down,
// then every record takes the next slot of its key (atomically, so records
// of equal order land in any order).  Out-of-range sizes sort first.
constexpr int ORDER_T = 1024;

__global__ void __launch_bounds__(ORDER_T) k_vbatched_order(int batch, const bf_dsize *size, int max_m, int *order) {
  __shared__ int cnt[CHOL_MAX_N + 2];
  const int nkey = max_m + 2;  // key m for 0 <= m <= max_m, max_m + 1 for out of range
  for (int x = threadIdx.x; x < nkey; x += ORDER_T) cnt[x] = 0;
  __syncthreads();
  for (int b = threadIdx.x; b < batch; b += ORDER_T) {
    const int m = size[b].m;
    atomicAdd(&cnt[(m < 0 || m > max_m) ? max_m + 1 : m], 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // exclusive offsets, largest key first (at most 514 keys)
    int run = 0;
    for (int x = nkey - 1; x >= 0; x--) {
      const int c = cnt[x];
      cnt[x] = run;
      run += c;
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < batch; b += ORDER_T) {
    const int m = size[b].m;
    order[atomicAdd(&cnt[(m < 0 || m > max_m) ? max_m + 1 : m], 1)] = b;
  }
}

// Block width of k_chol_rows: 16-column blocks halve the work the diagonal
// block's warp spends above the diagonal and the registers per thread.
constexpr int ROWS_BW = 16;


// MAXT, MINB: the launch bounds of the two-problem kernel (MAXT = 0: one
// problem per CTA)
template <int MAXT, int MINB, bool FUSED, bool ALIGNED, typename T>
cudaError_t launch_rows_p(int batch, int n, int k, Op A, Op B, Op C, OpWT<T> D, T *dinv, long long sdinv,
                          int *info, cudaStream_t s) {
  constexpr int P = MAXT ? 2 : 1;
  constexpr int RPW = 32 / P;
  const int threads = ((n + RPW - 1) / RPW) * 32;
  const unsigned blocks = (unsigned)((batch + P - 1) / P);
  if constexpr (P == 1)
    k_chol_rows<ROWS_BW, FUSED, ALIGNED, T><<<blocks, threads, 0, s>>>(batch, n, k, A, B, C, D, dinv, sdinv, info);
  else
    k_chol_rows2<ROWS_BW, FUSED, ALIGNED, T, MAXT, MINB>
        <<<blocks, threads, 0, s>>>(batch, n, k, A, B, C, D, dinv, sdinv, info);
  return cudaGetLastError();
}

template <int MAXT, int MINB, bool FUSED, typename T>
cudaError_t launch_rows4(bool aligned, int batch, int n, int k, Op A, Op B, Op C, OpWT<T> D, T *dinv,
                         long long sdinv, int *info, cudaStream_t s) {
  const int threads = ((n + 7) / 8) * 32;
  const unsigned blocks = (unsigned)((batch + 3) / 4);
  if (aligned)
    k_chol_rows4<FUSED, true, T, MAXT, MINB><<<blocks, threads, 0, s>>>(batch, n, k, A, B, C, D, dinv, sdinv, info);
  else
    k_chol_rows4<FUSED, false, T, MAXT, MINB><<<blocks, threads, 0, s>>>(batch, n, k, A, B, C, D, dinv, sdinv, info);
  return cudaGetLastError();
}

template <int MAXT, int MINB, bool FUSED, typename T>
cudaError_t launch_rows8_t(bool aligned, int batch, int n, int k, Op A, Op B, Op C, OpWT<T> D, T *dinv,
                           long long sdinv, int *info, cudaStream_t s) {
  const int threads = ((n + 3) / 4) * 32;
  const unsigned blocks = (unsigned)((batch + 7) / 8);
  if (aligned)
    k_chol_rows8<FUSED, true, T, MAXT, MINB><<<blocks, threads, 0, s>>>(batch, n, k, A, B, C, D, dinv, sdinv, info);
  else
    k_chol_rows8<FUSED, false, T, MAXT, MINB><<<blocks, threads, 0, s>>>(batch, n, k, A, B, C, D, dinv, sdinv, info);
  return cudaGetLastError();
}

// The eight-problem kernel (orders up to 64), built per CTA size for 64
// registers a thread.
template <bool FUSED>
cudaError_t launch_rows8(bool aligned, int batch, int n, int k, Op A, Op B, Op C, OpW D, double *dinv,
                         long long sdinv, int *info, cudaStream_t s) {
  if (n <= 32) return launch_rows8_t<256, 4, FUSED, double>(aligned, batch, n, k, A, B, C, D, dinv, sdinv, info, s);
  if (n <= 48) return launch_rows8_t<384, 3, FUSED, double>(aligned, batch, n, k, A, B, C, D, dinv, sdinv, info, s);
  return launch_rows8_t<512, 2, FUSED, double>(aligned, batch, n, k, A, B, C, D, dinv, sdinv, info, s);
}

template <int MAXT, int MINB, bool FUSED, typename T>
cudaError_t launch_rows_a(bool aligned, int batch, int n, int k, Op A, Op B, Op C, OpWT<T> D, T *dinv,
                          long long sdinv, int *info, cudaStream_t s) {
  return aligned ? launch_rows_p<MAXT, MINB, FUSED, true, T>(batch, n, k, A, B, C, D, dinv, sdinv, info, s)
                 : launch_rows_p<MAXT, MINB, FUSED, false, T>(batch, n, k, A, B, C, D, dinv, sdinv, info, s);
}

// Tail balance of the two-problem kernel at n > 192 (512-thread CTAs, two
// resident per SM).  A CTA carries two whole problems, so when the last wave
// holds more pairs than there are SMs, but leaves many slots empty, some SMs
// run two pairs through it while the others idle (n = k = 256, batch 1024:
// 512 pairs over 304 slots, SMs active 86% of the launch).  Then the pairs of
// the full waves go to k_chol_rows2 and the rest of the problems to the
// one-problem kernel, whose smaller CTAs spread them evenly: 989.5 -> 1018.3
// GFLOP/s there.  Not applied when the last wave has at most one pair per SM
// (each then runs alone at nearly the speed of two: potrf n = 256, batch
// 2048, measured 1068 unsplit vs 1018 split), nor for n <= 192, where the
// one-problem kernel is 10-30% slower per problem than the pair kernel.
// The split is applied when the last wave is at most this fraction full (in
// percent).
#ifndef BF_ROWS_TAIL_FILL
#define BF_ROWS_TAIL_FILL 80
#endif

template <typename T>
inline OpWT<T> shift_op(OpWT<T> o, long long b) {
  if (o.p) o.p += b * o.stride;
  return o;
}
inline Op shift_op(Op o, long long b) {
  if (o.p) o.p += b * o.stride;
  return o;
}

template <int MAXT, int MINB, bool FUSED, typename T>
cudaError_t launch_rows_pairs(bool aligned, int batch, int n, int k, Op A, Op B, Op C, OpWT<T> D, T *dinv,
                              long long sdinv, int *info, cudaStream_t s) {
  int pairs_cut = 0;  // pairs that go to the two-problem kernel when the tail is split
  if (BF_ROWS_TAIL_FILL > 0 && MAXT > 384 && n > 192) {
    static std::atomic<int> occ[64 * 17];
    const int threads = ((n + 15) / 16) * 32;
    const void *fn = aligned ? (const void *)k_chol_rows2<ROWS_BW, FUSED, true, T, MAXT, MINB>
                             : (const void *)k_chol_rows2<ROWS_BW, FUSED, false, T, MAXT, MINB>;
    const int sms = device_sm_count();
    const long long slots = (long long)resident_ctas(fn, threads, occ) * sms;
    const long long pairs = (batch + 1) / 2;
    if (slots > 0 && pairs > slots) {
      const long long full = pairs / slots, rest = pairs - full * slots;
      if (rest > sms && rest * 100 <= slots * BF_ROWS_TAIL_FILL) pairs_cut = (int)(full * slots);
    }
  }
  if (pairs_cut == 0)
    return launch_rows_a<MAXT, MINB, FUSED, T>(aligned, batch, n, k, A, B, C, D, dinv, sdinv, info, s);
  const int head = 2 * pairs_cut;
  cudaError_t e = launch_rows_a<MAXT, MINB, FUSED, T>(aligned, head, n, k, A, B, C, D, dinv, sdinv, info, s);
  if (e != cudaSuccess) return e;
  return launch_rows_a<0, 1, FUSED, T>(aligned, batch - head, n, k, shift_op(A, head), shift_op(B, head),
                                    shift_op(C, head), shift_op(D, head), dinv ? dinv + head * sdinv : nullptr,
                                    sdinv, info ? info + head : nullptr, s);
}

// Problems per CTA of the double-precision row kernel at order n: four
// where the 8-column layout wins, two up to the pair kernel's largest order,
// else one; then halved while the launch would have fewer CTAs than SMs, so
// that a small batch spreads over the GPU (latency over per-SM throughput).
// The fused routine also takes four per CTA at orders from
// BF_ROWS_P4_FUSED_MIN_N8 that are multiples of 8 (full last block):
// syrk_potrf n = 24, 832 -> 922 GFLOP/s; at n = 28 the small kernel is
// faster (895 against 746).
#ifndef BF_ROWS_P4_FUSED_MIN_N8
#define BF_ROWS_P4_FUSED_MIN_N8 24
#endif

template <bool FUSED>
int rows_problems_per_cta(int n, int batch) {
  constexpr int p2_max = FUSED ? BF_ROWS_P2_MAX_N_FUSED : BF_ROWS_P2_MAX_N;
  constexpr int p4_min = FUSED ? BF_ROWS_P4_MIN_N_FUSED : BF_ROWS_P4_MIN_N;
  constexpr int p4_max = FUSED ? BF_ROWS_P4_MAX_N_FUSED : BF_ROWS_P4_MAX_N;
  const bool p4 = (n >= p4_min && n <= p4_max) ||
                  (FUSED && n >= BF_ROWS_P4_FUSED_MIN_N8 && n % 8 == 0 && n <= p4_max);
  int p = p4 ? 4 : (n <= p2_max ? 2 : 1);
  const long long sms = device_sm_count();
  while (p > 1 && ((long long)batch + p - 1) / p < sms) p /= 2;
  return p;
}

template <bool FUSED, typename T>
cudaError_t launch_rows(bool aligned, int batch, int n, int k, Op A, Op B, Op C, OpWT<T> D, T *dinv,
                        long long sdinv, int *info, cudaStream_t s) {
  if constexpr (sizeof(T) == 8 || BF_ROWS_P2_FP32) {  // by default the FP32 factor keeps one problem per CTA
    const int p = rows_problems_per_cta<FUSED>(n, batch);
    if (p == 4 && n <= 64)
      return launch_rows4<256, BF_ROWS_P4_MINB256, FUSED, T>(aligned, batch, n, k, A, B, C, D, dinv, sdinv, info,
                                                            s);
    if (p == 4 && n <= 96)
      return launch_rows4<384, BF_ROWS_P4_MINB384, FUSED, T>(aligned, batch, n, k, A, B, C, D, dinv, sdinv, info,
                                                            s);
    if (p == 4)
      return launch_rows4<512, 2, FUSED, T>(aligned, batch, n, k, A, B, C, D, dinv, sdinv, info, s);
    if (p == 2 && n <= 64)
      return launch_rows_pairs<128, BF_ROWS_P2_MINB128, FUSED, T>(aligned, batch, n, k, A, B, C, D, dinv, sdinv,
                                                                  info, s);
    if (p == 2 && n <= 128)
      return launch_rows_pairs<256, BF_ROWS_P2_MINB256, FUSED, T>(aligned, batch, n, k, A, B, C, D, dinv, sdinv,
                                                                  info, s);
    if (p == 2 && n <= 192)
      return launch_rows_pairs<384, BF_ROWS_P2_MINB384, FUSED, T>(aligned, batch, n, k, A, B, C, D, dinv, sdinv,
                                                                  info, s);
    if (p == 2)
      return launch_rows_pairs<512, 2, FUSED, T>(aligned, batch, n, k, A, B, C, D, dinv, sdinv, info, s);
  }
  return launch_rows_a<0, 1, FUSED, T>(aligned, batch, n, k, A, B, C, D, dinv, sdinv, info, s);
}

// Lanes per problem of k_chol_small: the smallest G (at most 16) whose
// shared-memory triangles for the 32/G problems of a warp fit the budget, so
// that enough single-warp CTAs are resident on each SM.  Measured: more
// resident warps pay for a larger G (the pivot's rsqrt shared by fewer
// problems); a lane that walks a whole problem through shared memory is
// latency-bound (potrf n = 24 at G = 1: 244 GFLOP/s, at G = 4: 650).  26 KB
// gives G = 2, 4, 8 at n = 16, 24, 32 (budgets of 40 and 80 KB were slower
// there) and G = 8 rather than 16 at n = 33..40 (n = 40: potrf 550 -> 593,
// syrk_potrf 806 -> 894 GFLOP/s).
// Fewest lanes per problem of k_chol_small.  One lane per problem serves
// orders up to 8 in registers (k_chol_tiny); walking a whole problem
// through shared memory it is latency-bound: n = 12 measured 476 GFLOP/s at
// G = 1 and 517 at G = 2.
#ifndef BF_SMALL_MIN_G
#define BF_SMALL_MIN_G 2
#endif
#ifndef BF_SMALL_SMEM_BUDGET_KB
#define BF_SMALL_SMEM_BUDGET_KB 26
#endif
constexpr long long SMALL_SMEM_BUDGET = BF_SMALL_SMEM_BUDGET_KB * 1024;

// Largest order factored by k_chol_small; the four-problem row kernel takes
// over above (see BF_ROWS_P4_MIN_N).
#ifndef BF_CHOL_SMALL_MAX_N
#define BF_CHOL_SMALL_MAX_N 31
#endif
int pick_small_g(int n) {
  const long long ne = (long long)n * (n + 1) / 2;
  for (int g = BF_SMALL_MIN_G; g <= 16; g *= 2)
    if (ne * (32 / g) * 8 <= SMALL_SMEM_BUDGET) return g;
  return (ne * 2 * 8 <= 48 * 1024) ? 16 : 0;
}

template <int G, bool FUSED>
cudaError_t launch_small_g(bool aligned, int batch, int n, int k, Op A, Op B, Op C, OpW D,
                           double *dinv, long long sdinv, int *info, cudaStream_t s) {
  constexpr int Q = 32 / G;
  const size_t smem = (size_t)n * (n + 1) / 2 * small_pitch(Q) * sizeof(double);
  const unsigned blocks = (unsigned)((batch + Q - 1) / Q);
  if (smem > 48 * 1024) {
    static std::atomic<unsigned long long> attr_a{0}, attr_u{0};
    const void *fn = aligned ? (const void *)k_chol_small<G, FUSED, true> : (const void *)k_chol_small<G, FUSED, false>;
    cudaError_t e = smem_attr_once(fn, 200 * 1024, aligned ? attr_a : attr_u);
    if (e != cudaSuccess) return e;
  }
  if (aligned)
    k_chol_small<G, FUSED, true><<<blocks, 32, smem, s>>>(batch, n, k, A, B, C, D, dinv, sdinv, info);
  else
    k_chol_small<G, FUSED, false><<<blocks, 32, smem, s>>>(batch, n, k, A, B, C, D, dinv, sdinv, info);
  return cudaGetLastError();
}

// Largest order factored by k_chol_tiny (one lane per problem, registers).
#ifndef BF_CHOL_TINY_MAX_N
#define BF_CHOL_TINY_MAX_N 8
#endif

template <int N, bool FUSED>
cudaError_t launch_tiny_n(bool aligned, int batch, int k, Op A, Op B, Op C, OpW D, double *dinv, long long sdinv,
                          int *info, cudaStream_t s) {
  const unsigned blocks = (unsigned)((batch + 127) / 128);
  if (aligned)
    k_chol_tiny<N, FUSED, true><<<blocks, 128, 0, s>>>(batch, k, A, B, C, D, dinv, sdinv, info);
  else
    k_chol_tiny<N, FUSED, false><<<blocks, 128, 0, s>>>(batch, k, A, B, C, D, dinv, sdinv, info);
  return cudaGetLastError();
}

template <bool FUSED>
cudaError_t launch_tiny(bool aligned, int batch, int n, int k, Op A, Op B, Op C, OpW D, double *dinv,
                        long long sdinv, int *info, cudaStream_t s) {
  switch (n) {
    case 1: return launch_tiny_n<1, FUSED>(aligned, batch, k, A, B, C, D, dinv, sdinv, info, s);
    case 2: return launch_tiny_n<2, FUSED>(aligned, batch, k, A, B, C, D, dinv, sdinv, info, s);
    case 3: return launch_tiny_n<3, FUSED>(aligned, batch, k, A, B, C, D, dinv, sdinv, info, s);
    case 4: return launch_tiny_n<4, FUSED>(aligned, batch, k, A, B, C, D, dinv, sdinv, info, s);
    case 5: return launch_tiny_n<5, FUSED>(aligned, batch, k, A, B, C, D, dinv, sdinv, info, s);
    case 6: return launch_tiny_n<6, FUSED>(aligned, batch, k, A, B, C, D, dinv, sdinv, info, s);
    case 7: return launch_tiny_n<7, FUSED>(aligned, batch, k, A, B, C, D, dinv, sdinv, info, s);
    default: return launch_tiny_n<8, FUSED>(aligned, batch, k, A, B, C, D, dinv, sdinv, info, s);
  }
}

// The built-in choice of layout for potrf / syrk_potrf (the LAYOUT_CHOL_*
// candidates of bf_internal.cuh).
// Orders from which a batch of at least two problems per SM is factored in
// two diagonal blocks (potrf, trsm, syrk, potrf), and from which the fused
// routine forms its sum with the syrk kernel first.  Measured on the sweep's
// batches (GFLOP/s, row kernels -> blocked): potrf n = 128 1066 -> 1092,
// n = 192 1104 -> 1134, n = 256 1068 -> 1118; syrk_potrf n = 128 1123 ->
// 1176, n = 256 1018 -> 1189 (the fused row kernel re-reads A for every
// block column); syrk first: syrk_potrf n = 48 1103 -> 1121, n = 96 1154 ->
// 1183.  The FP64 pipe bounds these orders, so the store and reload of the
// sum that fusion saves (Sec. 4.7.2) costs less than the fused kernel's
// re-reads and barriers.
#ifndef BF_CHOL_BLOCKED_MIN_N
#define BF_CHOL_BLOCKED_MIN_N 128
#endif
#ifndef BF_CHOL_SPLIT_MIN_N
#define BF_CHOL_SPLIT_MIN_N 48
#endif

// Orders factored eight problems per CTA in 4-column blocks (k_chol_rows8),
// for batches that give every SM at least four such CTAs.  Measured on the
// sweep's batches against the previous choice (ms): potrf n = 24 1.723 ->
// 1.512 (small kernel, G = 4), n = 32 1.965 -> 1.744, n = 48 2.416 -> 2.360
// (four-problem row kernel); n = 16 ties, n = 64 4% slower.  syrk_potrf
// n = 24 2.379 -> 2.297; at n = 32 and 48 the syrk-first form stays faster.
#ifndef BF_ROWS8_MIN_N
#define BF_ROWS8_MIN_N 21
#endif
#ifndef BF_ROWS8_MAX_N
#define BF_ROWS8_MAX_N 56
#endif
#ifndef BF_ROWS8_MAX_N_FUSED
#define BF_ROWS8_MAX_N_FUSED 28
#endif

template <bool FUSED>
int chol_rule(int batch, int n) {
  // few problems of a small order: one problem per CTA over an SM's four
  // sub-partitions (the latency kernel)
  if (n <= BF_CHOL_LAT_MAX_N && (long long)batch <= (long long)BF_CHOL_LAT_MAX_BATCH_PER_SM * device_sm_count())
    return LAYOUT_CHOL_LAT;
  if (n >= BF_ROWS8_MIN_N && n <= (FUSED ? BF_ROWS8_MAX_N_FUSED : BF_ROWS8_MAX_N) &&
      (long long)batch >= 32LL * device_sm_count())
    return LAYOUT_CHOL_ROWS8;
  const bool full = (long long)batch >= 2LL * device_sm_count();
  if (full && n >= BF_CHOL_BLOCKED_MIN_N) return LAYOUT_CHOL_BLOCKED;
  if (FUSED && full && n >= BF_CHOL_SPLIT_MIN_N) return LAYOUT_CHOL_SPLIT;
  bool small = n <= BF_CHOL_SMALL_MAX_N;
  // the fused routine's four-problem orders below it, for batches that give
  // four-problem CTAs at least one per SM sub-partition
  if (small && rows_problems_per_cta<FUSED>(n, batch) == 4 && (long long)batch >= 16LL * device_sm_count())
    small = false;
  // enough problems for one lane each to give every SM sub-partition a
  // warp: the register kernel
  if (small && n <= BF_CHOL_TINY_MAX_N && (long long)batch >= 32LL * 4 * device_sm_count())
    return LAYOUT_CHOL_TINY;
  int g = small ? pick_small_g(n) : 0;
  // Small batches: more lanes per problem until the launch has a warp for
  // every SM sub-partition (4 per SM), up to one problem per warp.  The
  // budget's G is chosen for throughput; with few problems it would leave
  // most of the GPU idle and each warp a long serial chain of FP64 work.
  if (g)
    while (g < 32 && (long long)batch * g < 32LL * 4 * device_sm_count()) g *= 2;
  switch (g) {
    case 2: return LAYOUT_CHOL_SMALL_G2;
    case 4: return LAYOUT_CHOL_SMALL_G4;
    case 8: return LAYOUT_CHOL_SMALL_G8;
    case 16: return LAYOUT_CHOL_SMALL_G16;
    case 32: return LAYOUT_CHOL_SMALL_G32;
    default: return LAYOUT_CHOL_ROWS;
  }
}

// info of a factorization whose pieces were launched separately: the first
// column whose diagonal entry of L is not > 0.  Every kernel here forms
// L_jj = d * rsqrt(d), which is NaN when the pivot d is not > 0 (NaN
// included), and a positive number otherwise, so this is the first failing
// pivot.
__global__ void k_info_from_diag(int batch, int n, OpW D, int *info) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  const double *pd = D.p + (long long)b * D.stride;
  int bad = 0;
  for (int j = 0; j < n && bad == 0; j++)
    if (!(pd[pm_off(D.i0 + j, D.j0 + j, D.cn)] > 0.0)) bad = j + 1;
  info[b] = bad;
}

inline Op as_op(const OpW &d) { return Op{d.p, d.stride, d.cn, d.i0, d.j0}; }

// Blocked potrf of D (in place; the first half read from C): with h = n/2
// rounded down to a panel top,
//   L11 = chol(C11);  L21 = C21 L11^{-T};  D22 = C22 - L21 L21^T;  L22 = chol(D22)
// with the merged trsm and the syrk kernel, each diagonal block factored in
// the layout the rule picks for its own order and the batch (blocked again
// from order 128, eight problems per CTA at 21..56).  info is rebuilt from
// the diagonal at the end.
cudaError_t launch_chol_blocked(bool aligned, int batch, int n, Op C, OpW D, double *dinv, long long sdinv, int *info,
                                cudaStream_t s);

// potrf of a diagonal block of the blocked form, in the layout the rule picks
// for its own order and the batch (the blocked form again for a large
// block); info is left to the caller, which rebuilds it from the diagonal.
cudaError_t launch_potrf_block(bool aligned, int batch, int h, Op C, OpW D, double *dinv, long long sdinv,
                               cudaStream_t s) {
  const Op none{nullptr, 0, 0, 0, 0};
  switch (chol_rule<false>(batch, h)) {
    case LAYOUT_CHOL_BLOCKED: return launch_chol_blocked(aligned, batch, h, C, D, dinv, sdinv, nullptr, s);
    case LAYOUT_CHOL_ROWS8: return launch_rows8<false>(aligned, batch, h, 0, none, none, C, D, dinv, sdinv, nullptr, s);
    case LAYOUT_CHOL_LAT: return launch_chol_lat(false, batch, h, 0, none, none, C, D, dinv, sdinv, nullptr, s);
    default: return launch_rows<false, double>(aligned, batch, h, 0, none, none, C, D, dinv, sdinv, nullptr, s);
  }
}

cudaError_t launch_chol_blocked(bool aligned, int batch, int n, Op C, OpW D, double *dinv, long long sdinv, int *info,
                                cudaStream_t s) {
  const int h = (n / 2) & ~(PS - 1);
  cudaError_t e = launch_potrf_block(aligned, batch, h, C, D, dinv, sdinv, s);
  if (e != cudaSuccess) return e;
  const Op L11{D.p, D.stride, D.cn, D.i0, D.j0};
  const Op C21{C.p, C.stride, C.cn, C.i0 + h, C.j0};
  const OpW D21{D.p, D.stride, D.cn, D.i0 + h, D.j0};
  e = launch_trsm_rltn(batch, n - h, h, 1.0, L11, dinv, sdinv, C21, D21, s);
  if (e != cudaSuccess) return e;
  const Op L21 = as_op(D21);
  const Op C22{C.p, C.stride, C.cn, C.i0 + h, C.j0 + h};
  const OpW D22{D.p, D.stride, D.cn, D.i0 + h, D.j0 + h};
  e = launch_gemm_nt(true, batch, n - h, n - h, h, -1.0, L21, L21, 1.0, C22, D22, aligned, s);
  if (e != cudaSuccess) return e;
  e = launch_potrf_block(aligned, batch, n - h, as_op(D22), D22, dinv ? dinv + h : nullptr, sdinv, s);
  if (e != cudaSuccess || !info) return e;
  k_info_from_diag<<<(batch + 127) / 128, 128, 0, s>>>(batch, n, D, info);
  return cudaGetLastError();
}

template <bool FUSED>
cudaError_t launch_chol_t(bool aligned, int batch, int n, int k, Op A, Op B, Op C, OpW D,
                          double *dinv, long long sdinv, int *info, cudaStream_t s) {
  int lay = layout_forced(FUSED ? ROUTINE_SYRK_POTRF : ROUTINE_POTRF, n, batch);
  if (lay <= 0) lay = chol_rule<FUSED>(batch, n);
  if (lay == LAYOUT_CHOL_SPLIT || lay == LAYOUT_CHOL_BLOCKED) {
    // the fused routine's sum formed by the syrk kernel into D first
    if (FUSED) {
      cudaError_t e = launch_gemm_nt(true, batch, n, n, k, 1.0, A, B, 1.0, C, D, aligned, s);
      if (e != cudaSuccess) return e;
      C = as_op(D);
    }
    if (lay == LAYOUT_CHOL_BLOCKED) return launch_chol_blocked(aligned, batch, n, C, D, dinv, sdinv, info, s);
    const Op none{nullptr, 0, 0, 0, 0};
    return launch_rows<false, double>(aligned, batch, n, 0, none, none, C, D, dinv, sdinv, info, s);
  }
  switch (lay) {
    case LAYOUT_CHOL_TINY: return launch_tiny<FUSED>(aligned, batch, n, k, A, B, C, D, dinv, sdinv, info, s);
    case LAYOUT_CHOL_SMALL_G2: return launch_small_g<2, FUSED>(aligned, batch, n, k, A, B, C, D, dinv, sdinv, info, s);
    case LAYOUT_CHOL_SMALL_G4: return launch_small_g<4, FUSED>(aligned, batch, n, k, A, B, C, D, dinv, sdinv, info, s);
    case LAYOUT_CHOL_SMALL_G8: return launch_small_g<8, FUSED>(aligned, batch, n, k, A, B, C, D, dinv, sdinv, info, s);
    case LAYOUT_CHOL_SMALL_G16:
      return launch_small_g<16, FUSED>(aligned, batch, n, k, A, B, C, D, dinv, sdinv, info, s);
    case LAYOUT_CHOL_SMALL_G32:
      return launch_small_g<32, FUSED>(aligned, batch, n, k, A, B, C, D, dinv, sdinv, info, s);
    case LAYOUT_CHOL_LAT: return launch_chol_lat(FUSED, batch, n, k, A, B, C, D, dinv, sdinv, info, s);
    case LAYOUT_CHOL_ROWS8: return launch_rows8<FUSED>(aligned, batch, n, k, A, B, C, D, dinv, sdinv, info, s);
    default: return launch_rows<FUSED, double>(aligned, batch, n, k, A, B, C, D, dinv, sdinv, info, s);
  }
}

}  // namespace

int chol_layout_rule(bool fused, int batch, int n) {
  return fused ? chol_rule<true>(batch, n) : chol_rule<false>(batch, n);
}

bool chol_layout_ok(int layout, int n) {
  switch (layout) {
    case LAYOUT_CHOL_TINY: return n <= BF_CHOL_TINY_MAX_N;
    case LAYOUT_CHOL_SMALL_G2: case LAYOUT_CHOL_SMALL_G4: case LAYOUT_CHOL_SMALL_G8:
    case LAYOUT_CHOL_SMALL_G16: case LAYOUT_CHOL_SMALL_G32: {
      // the triangles of the warp's problems must fit the kernel's shared memory
      const int g = 2 << (layout - LAYOUT_CHOL_SMALL_G2);
      return n <= BF_CHOL_SMALL_MAX_N && (long long)n * (n + 1) / 2 * small_pitch(32 / g) * 8 <= 200 * 1024;
    }
    case LAYOUT_CHOL_ROWS: return n <= CHOL_MAX_N;
    case LAYOUT_CHOL_LAT: return n <= BF_CHOL_LAT_MAX_N;
    case LAYOUT_CHOL_SPLIT: return n <= CHOL_MAX_N;
    case LAYOUT_CHOL_BLOCKED: return n >= 32 && n <= CHOL_MAX_N;
    case LAYOUT_CHOL_ROWS8: return n <= 64;
    default: return false;
  }
}

cudaError_t launch_chol(bool fused, int batch, int n, int k, Op A, Op B, Op C, OpW D,
                        double *dinv, long long sdinv, int *info, bool aligned, cudaStream_t s) {
  return fused ? launch_chol_t<true>(aligned, batch, n, k, A, B, C, D, dinv, sdinv, info, s)
               : launch_chol_t<false>(aligned, batch, n, k, A, B, C, D, dinv, sdinv, info, s);
}

// The descriptor-array syrk_potrf can form the sum with the syrk kernel
// first (the strided form's split layout) when the layout entry of
// (syrk_potrf, max_m, batch) asks for it.  By default it stays fused: on
// 4096 problems of order U{8..128} the two launches measured 588 against
// 623 GFLOP/s (632 against 724 with the records sorted by decreasing order),
// the descriptor-array syrk reaching only 646-672 GFLOP/s on those sizes.
#ifndef BF_CHOL_V_SPLIT_MIN_N
#define BF_CHOL_V_SPLIT_MIN_N (1 << 30)
#endif

cudaError_t launch_chol_v(bool fused, int batch, const bf_dsize *size, const bf_dsub *A, const bf_dsub *B,
                          const bf_dsub *C, const bf_dsub *D, bool want_dinv, int *info, int max_m, int *status,
                          cudaStream_t s) {
  const int threads = ((max_m + 31) / 32) * 32;
  if (threads > 512 || threads == 0) return cudaErrorInvalidConfiguration;
  // the layout entry of (syrk_potrf, max_m, batch) may force either form
  const int lay = fused ? layout_forced(ROUTINE_SYRK_POTRF, max_m, batch) : 0;
  const bool two = lay > 0 ? (lay == LAYOUT_CHOL_SPLIT || lay == LAYOUT_CHOL_BLOCKED) : max_m >= BF_CHOL_V_SPLIT_MIN_N;
  if (fused && two) {
    // C + A B^T by the syrk kernel into D (its records checked there, no
    // status written), then D factored in place by a launch that checks the
    // same records with the same rules and reports status
    cudaError_t e = launch_gemm_nt_v(true, batch, size, 1.0, A, B, 1.0, C, D, max_m, max_m, nullptr, s);
    if (e != cudaSuccess) return e;
    k_chol_rows_v<ROWS_BW, false, true>
        <<<batch, threads, 0, s>>>(batch, size, A, B, C, D, want_dinv, info, max_m, status);
    return cudaGetLastError();
  }
  if (fused)
    k_chol_rows_v<ROWS_BW, true><<<batch, threads, 0, s>>>(batch, size, A, B, C, D, want_dinv, info, max_m, status);
  else
    k_chol_rows_v<ROWS_BW, false><<<batch, threads, 0, s>>>(batch, size, A, B, C, D, want_dinv, info, max_m, status);
  return cudaGetLastError();
}

// Problems per SM below which the ordered form keeps one problem per CTA
// (the records still in the given order): two per CTA halve the CTAs, and
// a small batch then leaves SMs short of warps.  Measured on orders
// U{8..128}, sorted records, GFLOP/s one per CTA / two per CTA: 1024
// problems 499 / 465, 1536 696 / 617, 2048 710 / 712, 3072 718 / 937, 4096
// 723 / 936.
// Four problems per CTA (8 rows of each per warp: a problem's last warp
// wastes at most 7 rows' lanes instead of 15) also for max_m up to 128, at
// 512 threads and 64 registers, from 24 problems per SM.  Measured on
// orders U{8..128}, sorted, GFLOP/s two / four per CTA: 2048 problems
// 712 / 632, 3072 937 / 926, 4096 936 / 994.
#ifndef BF_CHOL_VP_P4_MAX_M
#define BF_CHOL_VP_P4_MAX_M 128
#endif
#ifndef BF_CHOL_VP_P4_MIN_BATCH_PER_SM
#define BF_CHOL_VP_P4_MIN_BATCH_PER_SM 24
#endif
#ifndef BF_CHOL_VP_MIN_BATCH_PER_SM
#define BF_CHOL_VP_MIN_BATCH_PER_SM 12
#endif

// The ordered descriptor-array form: one launch for the orders up to 256
// (four problems per CTA with 8-column blocks when max_m <= 64, or <= 128 in
// large batches, else two with 16-column blocks), and one problem per CTA
// above 256 (a second launch over the whole array; each CTA skips the
// records of the other class).  The first launch also reports the records
// whose sizes are out of range.
cudaError_t launch_chol_vp(bool fused, int batch, const int *order, const bf_dsize *size, const bf_dsub *A,
                           const bf_dsub *B, const bf_dsub *C, const bf_dsub *D, bool want_dinv, int *info,
                           int max_m, int *status, cudaStream_t s) {
  const int wd = want_dinv ? 1 : 0;
  if ((long long)batch < (long long)BF_CHOL_VP_MIN_BATCH_PER_SM * device_sm_count()) {
    // too few problems to pair: one per CTA, in the given order
    const int threads = ((max_m + 31) / 32) * 32;
    if (fused)
      k_chol_rows_v<ROWS_BW, true><<<batch, threads, 0, s>>>(batch, size, A, B, C, D, wd, info, max_m, status,
                                                              order, -1, CHOL_MAX_N, 1);
    else
      k_chol_rows_v<ROWS_BW, false><<<batch, threads, 0, s>>>(batch, size, A, B, C, D, wd, info, max_m, status,
                                                               order, -1, CHOL_MAX_N, 1);
    return cudaGetLastError();
  }
  const unsigned g4 = (unsigned)((batch + 3) / 4), g2 = (unsigned)((batch + 1) / 2);
#define BF_VP(P_, BW_, MAXT_, MINB_, grid, threads, lo, hi, bad)                                                \
  do {                                                                                                         \
    if (fused)                                                                                                 \
      k_chol_rows_vp<P_, BW_, true, MAXT_, MINB_><<<grid, threads, 0, s>>>(batch, order, size, A, B, C, D, wd,  \
                                                                          info, max_m, status, lo, hi, bad);    \
    else                                                                                                       \
      k_chol_rows_vp<P_, BW_, false, MAXT_, MINB_><<<grid, threads, 0, s>>>(batch, order, size, A, B, C, D, wd, \
                                                                           info, max_m, status, lo, hi, bad);   \
  } while (0)
  // One launch for all orders up to 256, so that the small problems' CTAs
  // (latency-bound: few FP64 instructions each) run beside the large ones
  // instead of after them: four problems per CTA when max_m <= 64 (or <= 128
  // from BF_CHOL_VP_P4_MIN_BATCH_PER_SM problems per SM), else two.
  // Register bounds: 64 a thread.  On 4096 problems of order U{8..128} the
  // two-problem build measured 724 (128 registers, two CTAs per SM), 822
  // (85, three), 935 (64, four; a few spills) and 905 GFLOP/s (51, five).
  if (max_m <= 32) {
    BF_VP(4, 8, 128, 8, g4, 128, -1, 256, 1);
  } else if (max_m <= 64) {
    BF_VP(4, 8, 256, 4, g4, 256, -1, 256, 1);
  } else if (max_m <= BF_CHOL_VP_P4_MAX_M &&
             (long long)batch >= (long long)BF_CHOL_VP_P4_MIN_BATCH_PER_SM * device_sm_count()) {
    BF_VP(4, 8, 512, 2, g4, ((max_m + 7) / 8) * 32, -1, 256, 1);
  } else {
    const int threads = ((std::min(max_m, 256) + 15) / 16) * 32;
    if (threads <= 256)
      BF_VP(2, 16, 256, 4, g2, threads, -1, 256, 1);
    else
      BF_VP(2, 16, 512, 2, g2, threads, -1, 256, 1);
  }
#undef BF_VP
  if (max_m > 256) {
    const int threads = ((max_m + 31) / 32) * 32;
    if (fused)
      k_chol_rows_v<ROWS_BW, true><<<batch, threads, 0, s>>>(batch, size, A, B, C, D, wd, info, max_m, status,
                                                              order, 256, CHOL_MAX_N, 0);
    else
      k_chol_rows_v<ROWS_BW, false><<<batch, threads, 0, s>>>(batch, size, A, B, C, D, wd, info, max_m, status,
                                                               order, 256, CHOL_MAX_N, 0);
  }
  return cudaGetLastError();
}

cudaError_t launch_vbatched_order(int batch, const bf_dsize *size, int max_m, int *order, cudaStream_t s) {
  k_vbatched_order<<<1, ORDER_T, 0, s>>>(batch, size, max_m, order);
  return cudaGetLastError();
}

cudaError_t launch_chol_f32(int batch, int n, Op C, OpWT<float> D, int *info, bool aligned,
                            cudaStream_t s) {
  const Op none{nullptr, 0, 0, 0, 0};
  return launch_rows<false, float>(aligned, batch, n, 0, none, none, C, D, nullptr, 0, info, s);
}

}  // namespace bf
