// gemm_nt and syrk_ln, batched, FP64, panel-major operands.
//
// gemm_nt (Appendix A.2.1; Sec. 5.2.2):  D <- alpha * A * B^T + beta * C
// syrk_ln (Sec. 5.2.2):                  lower(D) <- alpha * A * B^T + beta * C
//
// Design.  On GB300 the FP64 pipe executes two FMA lanes per SM and clock, so
// a warp-wide DFMA occupies the SM's FP64 units for 16 cycles whatever its
// active mask, while loads, integer work and FP32 run on pipes that are an
// order of magnitude wider.  The kernel therefore spends every FP64 lane on
// useful work: each thread owns one 4x4 register block of one problem's D
// (rows i0..i0+3 sit in one panel of height 4, Sec. 4.1 register blocking),
// and threads are numbered over (problem, block) so that warps stay full
// across problem boundaries.  Operand columns of the register block are one
// 32-byte panel column each (Sec. 4.3.3: 'NT' reads both A and B along their
// panels), fetched with two 16-byte loads through L1; the 16 FMAs per column
// pair hide them.  syrk_ln numbers only the blocks of the lower block
// triangle, grouping the diagonal blocks in warps of their own that skip the
// FMAs above the diagonal.
#include "bf_internal.cuh"

namespace bf {
namespace {

// t -> (tr, tc) with tr >= tc and t = tr*(tr+1)/2 + tc.
__device__ __forceinline__ void tri_index(int t, int &tr, int &tc) {
  int r = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
  while (r * (r + 1) / 2 > t) r--;
  while ((r + 1) * (r + 2) / 2 <= t) r++;
  tr = r;
  tc = t - r * (r + 1) / 2;
}

// One 4x4 register block (rows i0.., columns j0..) of problem b.  DIAG: a
// diagonal block of syrk, whose FMAs above the diagonal are skipped.  KS > 1
// (small batches): the block is shared by KS adjacent lanes, lane ks taking
// the columns l = ks, ks + KS, ...; the partial blocks are summed with
// shuffles and lane 0 of the group writes D.
template <bool SYRK, bool DIAG, bool ALIGNED, int KS>
__device__ __forceinline__ void gemm_tile(int b, int tr, int tc, int ks, int m, int n, int k, double alpha,
                                          const Op &A, const Op &B, double beta, const Op &C,
                                          const OpW &D) {
  const int i0 = tr * 4, j0 = tc * 4;
  const double *pa = A.p + b * A.stride;
  const double *pb = B.p + b * B.stride;
  const double *pc = C.p ? C.p + b * C.stride : nullptr;
  double *pd = D.p + b * D.stride;

  const bool full = (i0 + 4 <= m) && (j0 + 4 <= n) && (!SYRK || tr != tc);
  const bool a1 = (alpha == 1.0);
  double acc[4][4];

  // alpha == 1: start from beta*C so that the epilogue costs no FP64 work.
  if (a1 && beta != 0.0 && ks == 0) {
    if (ALIGNED && full) {
      const double *cp = pc + (long long)(C.i0 + i0) * C.cn + (long long)(C.j0 + j0) * PS;
#pragma unroll
      for (int c = 0; c < 4; c++) {
        double2 lo = *(const double2 *)(cp + c * PS);
        double2 hi = *(const double2 *)(cp + c * PS + 2);
        acc[0][c] = lo.x; acc[1][c] = lo.y; acc[2][c] = hi.x; acc[3][c] = hi.y;
      }
    } else {
#pragma unroll
      for (int r = 0; r < 4; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) {
          const int i = i0 + r, j = j0 + c;
          acc[r][c] = (i < m && j < n && (!SYRK || i >= j)) ? pc[pm_off(C.i0 + i, C.j0 + j, C.cn)] : 0.0;
        }
    }
    if (beta != 1.0) {
#pragma unroll
      for (int r = 0; r < 4; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) acc[r][c] *= beta;
    }
  } else {
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
      for (int c = 0; c < 4; c++) acc[r][c] = 0.0;
  }

  if (ALIGNED) {
    // rows i0..i0+3 of A (and j0..j0+3 of B) are one panel: column l is 4
    // consecutive doubles.  Rows past m inside the last panel exist in memory
    // (storage is padded to whole panels); their results are never stored.
    const double *ap = pa + (long long)(A.i0 + i0) * A.cn + (long long)A.j0 * PS;
    const double *bp = pb + (long long)(B.i0 + j0) * B.cn + (long long)B.j0 * PS;
#pragma unroll 4
    for (int l = ks; l < k; l += KS) {
      const double2 a01 = __ldg((const double2 *)(ap + l * PS));
      const double2 a23 = __ldg((const double2 *)(ap + l * PS + 2));
      const double2 b01 = __ldg((const double2 *)(bp + l * PS));
      const double2 b23 = __ldg((const double2 *)(bp + l * PS + 2));
      const double av[4] = {a01.x, a01.y, a23.x, a23.y};
      const double bv[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
      for (int r = 0; r < 4; r++)
#pragma unroll
        for (int c = 0; c < 4; c++)
          if (!DIAG || c <= r) acc[r][c] = fma(av[r], bv[c], acc[r][c]);
    }
  } else {
    // generic variant (Sec. 4.4.2): sub-matrix rows not aligned to a panel top
    const double *ar[4], *br[4];
#pragma unroll
    for (int r = 0; r < 4; r++) {
      const int ii = min(i0 + r, m - 1), jj = min(j0 + r, n - 1);
      ar[r] = pa + pm_off(A.i0 + ii, A.j0, A.cn);
      br[r] = pb + pm_off(B.i0 + jj, B.j0, B.cn);
    }
#pragma unroll 2
    for (int l = ks; l < k; l += KS) {
      double av[4], bv[4];
#pragma unroll
      for (int r = 0; r < 4; r++) {
        av[r] = __ldg(ar[r] + l * PS);
        bv[r] = __ldg(br[r] + l * PS);
      }
#pragma unroll
      for (int r = 0; r < 4; r++)
#pragma unroll
        for (int c = 0; c < 4; c++)
          if (!DIAG || c <= r) acc[r][c] = fma(av[r], bv[c], acc[r][c]);
    }
  }

  if (KS > 1) {
    const int lane = threadIdx.x & 31;
    const unsigned gmask = ((1u << KS) - 1u) << (lane & ~(KS - 1));
#pragma unroll
    for (int o = 1; o < KS; o <<= 1)
#pragma unroll
      for (int r = 0; r < 4; r++)
#pragma unroll
        for (int c = 0; c < 4; c++)
          if (!DIAG || c <= r) acc[r][c] += __shfl_xor_sync(gmask, acc[r][c], o);
    if (ks != 0) return;
  }

  // epilogue
  if (ALIGNED && full) {
    double *dp = pd + (long long)(D.i0 + i0) * D.cn + (long long)(D.j0 + j0) * PS;
    const double *cp = (!a1 && beta != 0.0)
                           ? pc + (long long)(C.i0 + i0) * C.cn + (long long)(C.j0 + j0) * PS
                           : nullptr;
#pragma unroll
    for (int c = 0; c < 4; c++) {
      double v[4];
#pragma unroll
      for (int r = 0; r < 4; r++) v[r] = acc[r][c];
      if (!a1) {
        if (cp) {
          const double2 lo = *(const double2 *)(cp + c * PS);
          const double2 hi = *(const double2 *)(cp + c * PS + 2);
          v[0] = fma(alpha, v[0], beta * lo.x);
          v[1] = fma(alpha, v[1], beta * lo.y);
          v[2] = fma(alpha, v[2], beta * hi.x);
          v[3] = fma(alpha, v[3], beta * hi.y);
        } else {
#pragma unroll
          for (int r = 0; r < 4; r++) v[r] *= alpha;
        }
      }
      *(double2 *)(dp + c * PS) = make_double2(v[0], v[1]);
      *(double2 *)(dp + c * PS + 2) = make_double2(v[2], v[3]);
    }
  } else {
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
      for (int c = 0; c < 4; c++) {
        const int i = i0 + r, j = j0 + c;
        if (i < m && j < n && (!SYRK || i >= j)) {
          double v = acc[r][c];
          if (!a1) {
            v *= alpha;
            if (beta != 0.0) v = fma(beta, pc[pm_off(C.i0 + i, C.j0 + j, C.cn)], v);
          }
          pd[pm_off(D.i0 + i, D.j0 + j, D.cn)] = v;
        }
      }
  }
}

// gemm_nt: thread t -> (problem, block), blocks of a problem row-major.
// syrk_ln: the strictly-lower blocks of all problems come first, then the
// diagonal blocks of all problems, so that each warp does one kind of block
// and the diagonal ones save their upper-half FMAs.
template <bool SYRK, bool ALIGNED, int KS>
__global__ void __launch_bounds__(128)
k_gemm_nt(int batch, int m, int n, int k, double alpha, Op A, Op B, double beta, Op C, OpW D,
          int tiles_c, int tiles_pp) {
  const long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / KS;
  const int ks = (int)(threadIdx.x % KS);  // the KS lanes of a block are adjacent
  if (!SYRK) {
    if (t >= (long long)batch * tiles_pp) return;
    const int b = (int)(t / tiles_pp);
    const int tt = (int)(t - (long long)b * tiles_pp);
    const int tr = tt / tiles_c;
    gemm_tile<false, false, ALIGNED, KS>(b, tr, tt - tr * tiles_c, ks, m, n, k, alpha, A, B, beta, C, D);
  } else {
    const int TR = tiles_c;                 // block rows (= block columns)
    const int OD = TR * (TR - 1) / 2;       // strictly-lower blocks per problem
    const long long nod = (long long)batch * OD;
    if (t < nod) {
      const int b = (int)(t / OD);
      int r, c;
      tri_index((int)(t - (long long)b * OD), r, c);
      gemm_tile<true, false, ALIGNED, KS>(b, r + 1, c, ks, m, n, k, alpha, A, B, beta, C, D);
    } else if (t < nod + (long long)batch * TR) {
      const long long u = t - nod;
      const int b = (int)(u / TR);
      const int d = (int)(u - (long long)b * TR);
      gemm_tile<true, true, ALIGNED, KS>(b, d, d, ks, m, n, k, alpha, A, B, beta, C, D);
    }
  }
}

// Descriptor-array form: CTA = (problem, chunk of 128 register blocks).  The
// problem's record is checked first; all threads of the CTA see the same
// result, so an invalid or finished problem leaves the CTA as a whole.
template <bool SYRK>
__global__ void __launch_bounds__(128)
k_gemm_nt_v(int batch, const bf_dsize *size, double alpha, const bf_dsub *A, const bf_dsub *B, double beta,
            const bf_dsub *C, const bf_dsub *D, int chunks, int max_m, int max_n, int *status) {
  const int b = blockIdx.x / chunks, chunk = blockIdx.x - b * chunks;
  if (b >= batch) return;
  const bf_dsize sz = size[b];
  const int m = sz.m, n = SYRK ? sz.m : sz.n, k = sz.k;
  int err = 0;
  if (m < 0 || n < 0 || k < 0 || m > max_m || n > max_n)
    err = -1;
  else if (m > 0 && n > 0) {
    if (k > 0 && !dsub_ok(A[b], m, k))
      err = -2;
    else if (k > 0 && !dsub_ok(B[b], n, k))
      err = -3;
    else if (beta != 0.0 && !dsub_ok(C[b], m, n))
      err = -4;
    else if (!dsub_ok(D[b], m, n))
      err = -5;
  }
  if (chunk == 0 && threadIdx.x == 0 && status) status[b] = err;
  if (err != 0 || m == 0 || n == 0) return;
  const int tr = (m + 3) / 4, tcn = (n + 3) / 4;
  const int tiles = SYRK ? tr * (tr + 1) / 2 : tr * tcn;
  const int tile = chunk * blockDim.x + threadIdx.x;
  if (tile >= tiles) return;
  const OpW d = dsub_opw(D[b]);
  const Op dr{d.p, 0, d.cn, d.i0, d.j0};
  const Op a = k > 0 ? dsub_op(A[b]) : dr;  // k == 0: A and B are never read
  const Op bb = k > 0 ? dsub_op(B[b]) : dr;
  const Op c = beta != 0.0 ? dsub_op(C[b]) : Op{nullptr, 0, 0, 0, 0};
  const bool aligned = (a.i0 % PS) == 0 && (bb.i0 % PS) == 0 && (!c.p || (c.i0 % PS) == 0) && (d.i0 % PS) == 0 &&
                       !((unsigned long long)a.p & 15ull) && !((unsigned long long)bb.p & 15ull) &&
                       (!c.p || !((unsigned long long)c.p & 15ull)) && !((unsigned long long)d.p & 15ull);
  int r, cc;
  if (SYRK) {
    tri_index(tile, r, cc);
  } else {
    r = tile / tcn;
    cc = tile - r * tcn;
  }
  if (SYRK && r == cc) {
    if (aligned)
      gemm_tile<true, true, true, 1>(0, r, cc, 0, m, n, k, alpha, a, bb, beta, c, d);
    else
      gemm_tile<true, true, false, 1>(0, r, cc, 0, m, n, k, alpha, a, bb, beta, c, d);
  } else {
    if (aligned)
      gemm_tile<SYRK, false, true, 1>(0, r, cc, 0, m, n, k, alpha, a, bb, beta, c, d);
    else
      gemm_tile<SYRK, false, false, 1>(0, r, cc, 0, m, n, k, alpha, a, bb, beta, c, d);
  }
}

template <int KS>
cudaError_t launch_gemm_ks(bool syrk, bool aligned, long long total, int batch, int m, int n, int k, double alpha,
                           Op A, Op B, double beta, Op C, OpW D, int tcn, int tiles_pp, cudaStream_t s) {
  const int threads = 128;
  const long long blocks = (total * KS + threads - 1) / threads;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const unsigned g = (unsigned)blocks;
  if (syrk) {
    if (aligned)
      k_gemm_nt<true, true, KS><<<g, threads, 0, s>>>(batch, m, n, k, alpha, A, B, beta, C, D, tcn, tiles_pp);
    else
      k_gemm_nt<true, false, KS><<<g, threads, 0, s>>>(batch, m, n, k, alpha, A, B, beta, C, D, tcn, tiles_pp);
  } else {
    if (aligned)
      k_gemm_nt<false, true, KS><<<g, threads, 0, s>>>(batch, m, n, k, alpha, A, B, beta, C, D, tcn, tiles_pp);
    else
      k_gemm_nt<false, false, KS><<<g, threads, 0, s>>>(batch, m, n, k, alpha, A, B, beta, C, D, tcn, tiles_pp);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gemm_nt_v(bool syrk, int batch, const bf_dsize *size, double alpha, const bf_dsub *A,
                             const bf_dsub *B, double beta, const bf_dsub *C, const bf_dsub *D, int max_m,
                             int max_n, int *status, cudaStream_t s) {
  const int tr = (max_m + 3) / 4, tcn = ((syrk ? max_m : max_n) + 3) / 4;
  const long long tiles = syrk ? (long long)tr * (tr + 1) / 2 : (long long)tr * tcn;
  const int chunks = (int)max(1LL, (tiles + 127) / 128);
  const long long blocks = (long long)batch * chunks;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  if (syrk)
    k_gemm_nt_v<true><<<(unsigned)blocks, 128, 0, s>>>(batch, size, alpha, A, B, beta, C, D, chunks, max_m,
                                                       max_m, status);
  else
    k_gemm_nt_v<false><<<(unsigned)blocks, 128, 0, s>>>(batch, size, alpha, A, B, beta, C, D, chunks, max_m,
                                                        max_n, status);
  return cudaGetLastError();
}

int gemm_layout_rule(bool syrk, int batch, int m, int n, int k) {
  const int tr = (m + 3) / 4, tcn = (n + 3) / 4;
  const long long total = (long long)batch * (syrk ? tr * (tr + 1) / 2 : tr * tcn);
  if (total < 2LL * 4 * 32 * device_sm_count()) return (k >= 16) ? LAYOUT_GEMM_KS4 : (k >= 8 ? LAYOUT_GEMM_KS2 : LAYOUT_GEMM_KS1);
  return LAYOUT_GEMM_KS1;
}

cudaError_t launch_gemm_nt(bool syrk, int batch, int m, int n, int k, double alpha, Op A, Op B,
                           double beta, Op C, OpW D, bool aligned, cudaStream_t s) {
  const int tr = (m + 3) / 4, tcn = (n + 3) / 4;
  const int tiles_pp = syrk ? tr * (tr + 1) / 2 : tr * tcn;  // syrk: tcn == tr
  const long long total = (long long)batch * tiles_pp;
  // Small batches (fewer than two blocks per lane of every SM sub-partition's
  // warp slot): split k over 2 or 4 lanes per block, so the launch spreads
  // over the SMs instead of leaving each warp a long serial k-loop.
  int lay = layout_forced(syrk ? ROUTINE_SYRK_LN : ROUTINE_GEMM_NT, m, batch);
  if (lay <= 0) lay = gemm_layout_rule(syrk, batch, m, n, k);
  const int ks = lay == LAYOUT_GEMM_KS4 ? 4 : (lay == LAYOUT_GEMM_KS2 ? 2 : 1);
  if (ks == 4) return launch_gemm_ks<4>(syrk, aligned, total, batch, m, n, k, alpha, A, B, beta, C, D, tcn, tiles_pp, s);
  if (ks == 2) return launch_gemm_ks<2>(syrk, aligned, total, batch, m, n, k, alpha, A, B, beta, C, D, tcn, tiles_pp, s);
  return launch_gemm_ks<1>(syrk, aligned, total, batch, m, n, k, alpha, A, B, beta, C, D, tcn, tiles_pp, s);
}

}  // namespace bf
