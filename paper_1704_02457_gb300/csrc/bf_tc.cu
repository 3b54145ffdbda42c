// Trailing update of a blocked Cholesky factorization on the tensor cores
// (tcgen05), for the mixed-precision solver:
//
//     lower(D) <- C - L21 * L21^T
//
// L21 is the m x k panel below a diagonal block (k <= 32, m <= 128), C and D
// the m x m trailing block, all FP64 panel-major.  The paper's routines come
// in separate single- and double-precision versions (Appendix A.3); this
// update is the place where a mixed-precision factorization can drop to a
// tensor-core format, while the diagonal blocks and panels stay FP64.  The
// product runs in one of three precisions:
//   BF16:   L21 rounded to bfloat16, products accumulated in FP32
//           (tcgen05.mma kind::f16);
//   TF32:   L21 rounded to TF32, FP32 accumulation (kind::tf32);
//   3xTF32: L21 = H + R, H = tf32(L21), R = tf32(L21 - H); the product is
//           H H^T + H R^T + R H^T (three passes, kind::tf32), which keeps
//           about FP32 accuracy (the R R^T term is below it).
//
// One CTA of four warps per problem:
//   - one thread starts TMA bulk copies (cp.async.bulk) of the panel's m/4
//     panels of 4 rows x k columns -- each a contiguous run of 32 k bytes in
//     the panel-major format (Sec. 4.3.3) -- into shared memory, completing
//     on an mbarrier;
//   - the threads convert the FP64 panel into the operand format, in the
//     K-major, non-swizzled layout of 8-row x 16-byte core matrices that the
//     tensor core reads through a shared-memory matrix descriptor;
//   - one thread issues the MMAs (M = 128 rows, N = m rounded up to 16, K =
//     16 for BF16, 8 for TF32 per instruction) into an FP32 accumulator in
//     tensor memory (TMEM), and commits them to a second mbarrier;
//   - each warp reads its 32 accumulator rows back (tcgen05.ld) and writes
//     D = C - acc on the lower triangle, in FP64.
// Both operands of the MMA are the same shared-memory tile (B = A = L21), so
// the product is L21 L21^T.  Every wait on an mbarrier is bounded: on a
// timeout the CTA records -3 in err[b], waits (bounded) for its own work in
// flight, releases its TMEM and returns.
#include <cuda_bf16.h>
#include <stdint.h>

#include "bf_internal.cuh"

namespace bf {
namespace {

constexpr int TC_T = 128;       // threads: 4 warps, one per 32 TMEM lanes
constexpr int TC_M = 128;       // MMA rows
constexpr int TC_KMAX = 32;     // panel width
// shared memory: two operand tiles (TF32 fills one: 128 x 32 x 4 bytes), the
// FP64 panel, then the barriers: 64 KB, three CTAs per SM
constexpr int TC_TILE = 16 * 1024;
constexpr int TC_STAGE = TC_M * TC_KMAX * 8;
constexpr int TC_SMEM = 2 * TC_TILE + TC_STAGE + 64;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of a K-major, non-swizzled operand: start
// address, byte distance between core matrices adjacent along K (leading
// byte offset) and along M/N (stride byte offset), all in units of 16 bytes,
// the fixed version bits 46..48 = 0b001, no base offset, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor: FP32 accumulator (bits 4..5 = 1), A and B formats
// (bits 7..9, 10..12: 1 = BF16, 2 = TF32), both K-major, N / 8 in bits
// 17..22, M / 16 in bits 24..28.
__device__ __forceinline__ uint32_t idesc(uint32_t fmt, int M, int N) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Bounded wait for the phase of parity `parity` to complete.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < (1 << 22); it++) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Conversions by integer arithmetic on the bit patterns, so that they keep
// off the FP64 pipe (on GB300 a conversion from or to FP64 occupies it like
// an FMA).  Outside the normal FP32 range, and for zero, the hardware
// conversion is used.
//
// x rounded to nearest even with KEEP mantissa bits (7: BF16, 10: TF32, 23:
// FP32), returned as FP32 bits (exact: the low 23 - KEEP bits are zero).
template <int KEEP>
__device__ __forceinline__ uint32_t round_to_f32_bits(double x) {
  constexpr int CUT = 52 - KEEP;
  unsigned long long u = (unsigned long long)__double_as_longlong(x);
  u += ((1ull << (CUT - 1)) - 1ull) + ((u >> CUT) & 1ull);  // ties to even; a carry moves into the exponent
  u &= ~((1ull << CUT) - 1ull);
  const int e = (int)((u >> 52) & 0x7FF) - 896;  // FP32 biased exponent
  if (e >= 1 && e <= 254)
    return (uint32_t)((u >> 63) << 31) | ((uint32_t)e << 23) | (uint32_t)((u >> 29) & 0x7FFFFFu);
  // zero, subnormal, overflow or non-finite: the hardware's rounding
  const float f = (float)x;
  if (KEEP == 23) return __float_as_uint(f);
  if (KEEP == 7) return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(f)) << 16;
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(f));
  return r;
}

// FP32 bits -> the same value in FP64 (exact).
__device__ __forceinline__ double f32_bits_to_double(uint32_t f) {
  const uint32_t e = (f >> 23) & 0xFFu;
  if (e == 0u || e == 255u) return (double)__uint_as_float(f);
  const unsigned long long u = ((unsigned long long)(f >> 31) << 63) | ((unsigned long long)(e + 896u) << 52) |
                               ((unsigned long long)(f & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)u);
}

// Byte offset of element (r, k) in a K-major, non-swizzled tile of TC_M rows:
// core matrices of 8 rows x 16 bytes, the 16 row groups of one 16-byte
// column chunk contiguous (stride 128 bytes), chunks 2048 bytes apart.
template <int ES>
__device__ __forceinline__ uint32_t tile_off(int r, int k) {
  constexpr int PER = 16 / ES;  // elements per 16-byte chunk
  return (uint32_t)(((k / PER) * (TC_M / 8) + r / 8) * 128 + (r % 8) * 16 + (k % PER) * ES);
}
constexpr uint32_t TC_LBO = (TC_M / 8) * 128;  // next chunk along K
constexpr uint32_t TC_SBO = 128;               // next 8-row group

// W (FP64) -> L32 (FP32), lower triangle, one CTA per problem; info32 = the
// first failure of the blocked factorization: the column of the first
// failing pivot (block c's info plus c * nb), or -3 for a timed-out update.
__global__ void __launch_bounds__(256)
k_factor_to_f32(int n, int nblk, int nb, const double *W, long long sw, float *l32, long long sl, const int *infos,
                int batch, int *info32) {
  const int b = blockIdx.x;
  const double *w = W + (long long)b * sw;
  float *l = l32 + (long long)b * sl;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int j = e / n, i = e - j * n;
    if (i >= j) l[pm_off(i, j, n)] = __uint_as_float(round_to_f32_bits<23>(w[pm_off(i, j, n)]));
  }
  if (threadIdx.x == 0) {
    int r = 0;
    for (int c = 0; c < nblk && r == 0; c++) {
      const int v = infos[(long long)c * batch + b];
      r = v < 0 ? v : (v > 0 ? c * nb + v : 0);
    }
    info32[b] = r;
  }
}

// PREC: 0 BF16, 1 TF32, 2 3xTF32
template <int PREC>
__global__ void __launch_bounds__(TC_T)
k_syrk_tc(int m, int k, Op L, Op C, OpW D, int *err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char *tile_h = smem;
  unsigned char *tile_r = smem + TC_TILE;
  double *stage = (double *)(smem + 2 * TC_TILE);
  uint64_t *bars = (uint64_t *)(smem + 2 * TC_TILE + TC_STAGE);
  uint32_t *tmem_slot = (uint32_t *)(bars + 2);
  const int b = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t bar_tma = smem_u32(&bars[0]), bar_mma = smem_u32(&bars[1]);
  const int N = (m + 15) & ~15;
  const int ncols = N <= 32 ? 32 : (N <= 64 ? 64 : 128);  // TMEM columns: a power of two >= 32
  const int panels = (m + PS - 1) / PS;

  if (tid == 0) {
    mbar_init(bar_tma, 1);
    mbar_init(bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  // the panel: m/4 runs of 4 rows x k columns (contiguous, 32 k bytes each)
  if (tid == 0) {
    const uint32_t bytes = (uint32_t)panels * 32u * (uint32_t)k;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_tma), "r"(bytes) : "memory");
    const double *src = L.p + (long long)b * L.stride + pm_off(L.i0, L.j0, L.cn);
    for (int p = 0; p < panels; p++)
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              smem_u32(stage + p * PS * k)),
          "l"(src + (long long)p * PS * L.cn), "r"(32u * (uint32_t)k), "r"(bar_tma)
          : "memory");
  }
  bool ok = mbar_wait(bar_tma, 0);
  if (__syncthreads_or(!ok)) {
    if (tid == 0 && err) err[b] = -3;
    mbar_wait(bar_tma, 0);
    goto release;
  }

  // FP64 panel -> operand tiles (rows >= m and columns >= k are zero)
  for (int e = tid; e < TC_M * TC_KMAX; e += TC_T) {
    const int r = e / TC_KMAX, kk = e % TC_KMAX;
    const bool in = r < m && kk < k;
    const double x = in ? stage[(r / PS) * PS * k + kk * PS + (r % PS)] : 0.0;
    if (PREC == 0) {
      *(unsigned short *)(tile_h + tile_off<2>(r, kk)) = in ? (unsigned short)(round_to_f32_bits<7>(x) >> 16) : 0;
    } else {
      const uint32_t h = in ? round_to_f32_bits<10>(x) : 0u;
      *(uint32_t *)(tile_h + tile_off<4>(r, kk)) = h;
      if (PREC == 2)
        *(uint32_t *)(tile_r + tile_off<4>(r, kk)) = in ? round_to_f32_bits<10>(x - f32_bits_to_double(h)) : 0u;
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();

  if (tid == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    constexpr int KI = PREC == 0 ? 16 : 8;        // K of one instruction
    constexpr int CH = PREC == 0 ? 8 : 4;         // elements of a 16-byte chunk
    const uint32_t id = idesc(PREC == 0 ? 1u : 2u, TC_M, N);
    const uint32_t th = smem_u32(tile_h), tr = smem_u32(tile_r);
    int issued = 0;
    const int passes = PREC == 2 ? 3 : 1;
    for (int pass = 0; pass < passes; pass++) {
      // 3xTF32: H H^T, H R^T, R H^T
      const uint32_t ta = pass == 2 ? tr : th;
      const uint32_t tb = pass == 1 ? tr : th;
      for (int k0 = 0; k0 < TC_KMAX; k0 += KI) {
        if (k0 >= k) break;
        const uint32_t off = (uint32_t)(k0 / CH) * TC_LBO;
        const uint64_t da = sdesc(ta + off, TC_LBO, TC_SBO), db = sdesc(tb + off, TC_LBO, TC_SBO);
        const uint32_t acc = issued > 0 ? 1u : 0u;
        if (PREC == 0)
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
              "l"(da), "l"(db), "r"(id), "r"(acc)
              : "memory");
        else
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
              "l"(da), "l"(db), "r"(id), "r"(acc)
              : "memory");
        issued++;
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_mma)
                 : "memory");
  }
  {
    // D = C - acc on the lower triangle: warp w holds rows 32 w .. 32 w + 31;
    // a chunk's C loads go out before its accumulator is read (the first
    // before the wait for the MMAs)
    const int i = 32 * warp + lane;
    const double *crow = C.p + (long long)b * C.stride + pm_off(C.i0 + (i < m ? i : 0), C.j0, C.cn);
    double *drow = D.p + (long long)b * D.stride + pm_off(D.i0 + (i < m ? i : 0), D.j0, D.cn);
    double cv[32];
#pragma unroll
    for (int jj = 0; jj < 32; jj++) cv[jj] = (i < m && jj <= i) ? crow[PS * jj] : 0.0;
    ok = mbar_wait(bar_mma, 0);
    if (__syncthreads_or(!ok)) {
      if (tid == 0 && err) err[b] = -3;
      mbar_wait(bar_mma, 0);
      goto release;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    for (int c0 = 0; c0 < N; c0 += 32) {
      if (c0 > 0) {
#pragma unroll
        for (int jj = 0; jj < 32; jj++) cv[jj] = (i < m && c0 + jj <= i) ? crow[PS * (c0 + jj)] : 0.0;
      }
      uint32_t v[32];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
          "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
            "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
            "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
          : "r"(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (i < m && c0 <= i) {
#pragma unroll
        for (int jj = 0; jj < 32; jj++)
          if (c0 + jj <= i) drow[PS * (c0 + jj)] = cv[jj] - f32_bits_to_double(v[jj]);
      }
    }
  }

release:
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

}  // namespace

bool syrk_tc_ok(int m, int k, const Op &L) {
  // the runs of the bulk copies start 16-byte aligned: rows from a panel top
  // (a run then starts 32 (i0 cn + 4 j0 + 4 p cn) bytes into the problem),
  // problems an even number of doubles apart, 16-byte aligned storage
  if (m < 1 || m > TC_M || k < 1 || k > TC_KMAX) return false;
  if ((L.i0 % PS) != 0 || (L.stride % 2) != 0) return false;
  return ((uintptr_t)L.p % 16) == 0;
}

cudaError_t launch_syrk_tc(int prec, int batch, int m, int k, Op L, Op C, OpW D, int *err, cudaStream_t s) {
  if (!syrk_tc_ok(m, k, L) || prec < 0 || prec > 2) return cudaErrorInvalidValue;
  static std::atomic<unsigned long long> a0{0}, a1{0}, a2{0};
  const void *fn = prec == 0 ? (const void *)k_syrk_tc<0> : (prec == 1 ? (const void *)k_syrk_tc<1> : (const void *)k_syrk_tc<2>);
  cudaError_t e = smem_attr_once(fn, TC_SMEM, prec == 0 ? a0 : (prec == 1 ? a1 : a2));
  if (e != cudaSuccess) return e;
  if (prec == 0)
    k_syrk_tc<0><<<batch, TC_T, TC_SMEM, s>>>(m, k, L, C, D, err);
  else if (prec == 1)
    k_syrk_tc<1><<<batch, TC_T, TC_SMEM, s>>>(m, k, L, C, D, err);
  else
    k_syrk_tc<2><<<batch, TC_T, TC_SMEM, s>>>(m, k, L, C, D, err);
  return cudaGetLastError();
}

// The blocked mixed-precision factorization and refinement: for each block
// column of width nb, FP64 potrf of the diagonal block and FP64 trsm of the
// panel below (the library's own kernels, on the FP64 working copy W), then
// the trailing update on the tensor cores in precision `prec`.  The first
// block column reads A, later ones W.  The factor, rounded to FP32, then
// drives the FP32 solves of the FP64 iterative refinement.
cudaError_t launch_posv_mixed_tc(int prec, int batch, int n, int nrhs, Op A, Op B, OpW X, double tol, int max_iter,
                                 int *iters, double *resid, double *W, double *dinv, float *l32, int *infos,
                                 int *info32, cudaStream_t s) {
  constexpr int NB = TC_KMAX;
  const int pm = (n + PS - 1) / PS * PS;
  const long long sw = (long long)pm * n;
  const int nblk = (n + NB - 1) / NB;
  const Op none{nullptr, 0, 0, 0, 0};
  cudaError_t e = cudaSuccess;
  for (int c = 0; c < nblk; c++) {
    const int j0 = c * NB, w = min(NB, n - j0), m = n - j0 - w;
    const Op src = c == 0 ? A : Op{W, sw, n, 0, 0};
    const Op sdiag{src.p, src.stride, src.cn, src.i0 + j0, src.j0 + j0};
    const OpW wdiag{W, sw, n, j0, j0};
    const Op wdiag_r{W, sw, n, j0, j0};
    const bool aligned = c > 0 || ((A.i0 % PS) == 0 && (A.stride % 2) == 0 && ((uintptr_t)A.p % 16) == 0);
    e = launch_chol(false, batch, w, 0, none, none, sdiag, wdiag, dinv + j0, n, infos + (long long)c * batch,
                    aligned, s);
    if (e != cudaSuccess || m == 0) break;
    const Op spanel{src.p, src.stride, src.cn, src.i0 + j0 + w, src.j0 + j0};
    e = launch_trsm_rltn(batch, m, w, 1.0, wdiag_r, dinv + j0, n, spanel, OpW{W, sw, n, j0 + w, j0}, s);
    if (e != cudaSuccess) break;
    const Op strail{src.p, src.stride, src.cn, src.i0 + j0 + w, src.j0 + j0 + w};
    e = launch_syrk_tc(prec, batch, m, w, Op{W, sw, n, j0 + w, j0}, strail, OpW{W, sw, n, j0 + w, j0 + w},
                       infos + (long long)c * batch, s);
    if (e != cudaSuccess) break;
  }
  if (e != cudaSuccess) return e;
  k_factor_to_f32<<<batch, 256, 0, s>>>(n, nblk, NB, W, sw, l32, sw, infos, batch, info32);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_posv_refine(batch, n, nrhs, A, B, X, tol, max_iter, iters, resid, l32, info32, s);
}

}  // namespace bf
