// Internal declarations shared by the CUDA translation units of the library.
//
// Panel-major addressing (Sec. 4.3.3 of the paper): with panel height PS (a
// power of two) and panel length cn, element (r, c) of a matrix lies at
//   (r - r % PS) * cn + c * PS + r % PS.
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include "bfgpu.h"

namespace bf {

constexpr int PS = BF_PS;
static_assert((PS & (PS - 1)) == 0, "panel height must be a power of two");

// A read-only operand of a batched call: storage of problem 0, distance in
// doubles between consecutive problems, panel length and the sub-matrix
// offset of the operand.
struct Op {
  const double *p;
  long long stride;
  int cn;
  int i0, j0;
};

// A written operand (of element type T; OpW for the FP64 routines).
template <typename T>
struct OpWT {
  T *p;
  long long stride;
  int cn;
  int i0, j0;
};
using OpW = OpWT<double>;

__host__ __device__ __forceinline__ long long pm_off(int r, int c, int cn) {
  return (long long)(r & ~(PS - 1)) * cn + (long long)c * PS + (r & (PS - 1));
}

// ---- launchers (each returns the cudaError_t of its launch) ---------------

cudaError_t launch_gemm_nt(bool syrk, int batch, int m, int n, int k, double alpha, Op A, Op B,
                           double beta, Op C, OpW D, bool aligned, cudaStream_t s);

// gemm_nn (trmm = false: D = alpha A X + beta C, X k x n) and trmm_rlnn
// (trmm = true: D = alpha A X with X = L lower n x n, k = n, C unused).
cudaError_t launch_gemm_nn(bool trmm, int batch, int m, int n, int k, double alpha, Op A, Op X,
                           double beta, Op C, OpW D, bool aligned, cudaStream_t s);

// potrf_l (fused = false) and syrk_potrf_ln (fused = true, A and B used).
cudaError_t launch_chol(bool fused, int batch, int n, int k, Op A, Op B, Op C, OpW D,
                        double *dinv, long long sdinv, int *info, bool aligned, cudaStream_t s);

// FP32 lower Cholesky factor of an FP64 input (the mixed-precision solver's
// working factor), written panel-major in single precision.
cudaError_t launch_chol_f32(int batch, int n, Op C, OpWT<float> D, int *info, bool aligned,
                            cudaStream_t s);

cudaError_t launch_trsm_rltn(int batch, int m, int n, double alpha, Op L, const double *dinv,
                             long long sdinv, Op B, OpW D, cudaStream_t s);

// A X = B with the FP64 factor L (potrs), and the mixed-precision solver
// (FP32 factor in the workspace l32 / info32, FP64 iterative refinement).
cudaError_t launch_potrs(int batch, int n, int nrhs, Op L, Op B, OpW X, cudaStream_t s);
cudaError_t launch_posv_adjoint(int batch, int n, int nrhs, Op L, Op X, Op Xbar, OpW Bbar, OpW Abar,
                                cudaStream_t s);
cudaError_t launch_posv_mixed(int batch, int n, int nrhs, Op A, Op B, OpW X, double tol,
                              int max_iter, int *iters, double *resid, float *l32, int *info32,
                              bool aligned, cudaStream_t s);

// Raise a kernel's dynamic shared-memory limit to `bytes`, once per device
// (the attribute is per device; `done` is the call site's bit mask of the
// devices already set, devices >= 64 are set on every call).
inline cudaError_t smem_attr_once(const void *fn, int bytes, std::atomic<unsigned long long> &done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
  return e;
}

// Number of SMs of the current device (cached per device).
inline int device_sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 152;
  if (dev < 64) {
    const int c = cache[dev].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
  if (dev < 64) cache[dev].store(sms, std::memory_order_relaxed);
  return sms;
}

// CTAs of `fn` at `threads` threads (no dynamic shared memory) resident on
// one SM of the current device; `cache` holds one entry per (device, warps)
// for up to 64 devices and 16 warps.
inline int resident_ctas(const void *fn, int threads, std::atomic<int> (&cache)[64 * 17]) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  const int w = (threads + 31) / 32;
  const bool cached = dev < 64 && w <= 16;
  if (cached) {
    const int c = cache[dev * 17 + w].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, 0) != cudaSuccess) return 0;
  if (cached && nb > 0) cache[dev * 17 + w].store(nb, std::memory_order_relaxed);
  return nb;
}

// Check of one operand record of the descriptor-array forms, run by the
// kernels on the device (and by bf_dsub_valid on the host): the same rules as
// the host's check of a strided operand.  The bounds are compared in 64-bit
// arithmetic, so that no offset or size near INT_MAX can wrap round and pass.
__host__ __device__ __forceinline__ bool dsub_ok(const bf_dsub &s, int rows, int cols) {
  const bf_dmat &d = s.mat;
  if (!d.pA || d.ps != PS || ((unsigned long long)d.pA & 7ull) || d.m < 0 || d.n < 0 || d.pm < d.m ||
      d.pm % PS != 0 || d.cn < d.n || rows < 0 || cols < 0)
    return false;
  return s.i >= 0 && (long long)s.i + rows <= (long long)d.m && s.j >= 0 &&
         (long long)s.j + cols <= (long long)d.n;
}

__device__ __forceinline__ Op dsub_op(const bf_dsub &s) { return Op{s.mat.pA, 0, s.mat.cn, s.i, s.j}; }
__device__ __forceinline__ OpW dsub_opw(const bf_dsub &s) { return OpW{s.mat.pA, 0, s.mat.cn, s.i, s.j}; }

// Programmatic dependent launch (griddepcontrol, sm_90 and later).  A kernel
// launched by launch_pdl may be scheduled while the kernel before it on the
// stream is still running; pdl_wait() returns once that kernel has completed
// and its writes are visible, so it comes before the first access to memory
// another kernel may have written.  pdl_allow() lets the next such kernel be
// scheduled once every CTA of this one has called it (or exited).  Both are
// no-ops in a kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_allow() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// !(d > 0) from the bit pattern on the integer pipes: negative (-0 and
// NaNs with the sign bit included), +0, or NaN.  On GB300 a double compare
// issues on the narrow FP64 pipe like an FMA; the pivot test of every
// factorization column runs here instead.
__device__ __forceinline__ bool not_positive(double d) {
  const int hi = __double2hiint(d), lo = __double2loint(d);
  return hi < 0 || (hi | lo) == 0 || hi > 0x7ff00000 || (hi == 0x7ff00000 && lo != 0);
}
__device__ __forceinline__ bool not_positive(float f) { return !(f > 0.0f); }

// d == 0 (either sign) from the bit pattern, for the same reason.
__device__ __forceinline__ bool is_zero(double d) {
  return ((__double2hiint(d) & 0x7fffffff) | __double2loint(d)) == 0;
}

// 8-byte asynchronous global -> shared copy (cp.async, bypasses registers)
__device__ __forceinline__ void cp_async8(double *dst, const double *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Launchers of the descriptor-array forms (problems checked on the device).
cudaError_t launch_gemm_nt_v(bool syrk, int batch, const bf_dsize *size, double alpha, const bf_dsub *A,
                             const bf_dsub *B, double beta, const bf_dsub *C, const bf_dsub *D, int max_m,
                             int max_n, int *status, cudaStream_t s);
cudaError_t launch_chol_v(bool fused, int batch, const bf_dsize *size, const bf_dsub *A, const bf_dsub *B,
                          const bf_dsub *C, const bf_dsub *D, bool want_dinv, int *info, int max_m, int *status,
                          cudaStream_t s);
// The ordered form (records taken in `order`, NULL: their own order; P
// problems of similar size per CTA) and the counting sort that gives the
// order by decreasing size.
cudaError_t launch_chol_vp(bool fused, int batch, const int *order, const bf_dsize *size, const bf_dsub *A,
                           const bf_dsub *B, const bf_dsub *C, const bf_dsub *D, bool want_dinv, int *info,
                           int max_m, int *status, cudaStream_t s);
cudaError_t launch_vbatched_order(int batch, const bf_dsize *size, int max_m, int *order, cudaStream_t s);
cudaError_t launch_trsm_rltn_v(int batch, const bf_dsize *size, double alpha, const bf_dsub *L, bool use_dinv,
                               const bf_dsub *B, const bf_dsub *D, int max_m, int max_n, int *status,
                               cudaStream_t s);

// 1/d in three FP64 operations: the hardware approximation r0 (relative
// error e = 1 - d r0 below 2^-22), then r0 (1 + e + e^2), whose error is of
// order e^3.  Used where one reciprocal is shared by a column of
// multiplications, instead of an IEEE divide.  The approximation flushes a
// subnormal d to zero, and the result is then NaN (tested).
__device__ __forceinline__ double recip3(double d) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
  const double e = fma(-d, r, 1.0);
  return fma(fma(e, e, e), r, r);
}

// x == 1.0 from the bit pattern (a double compare issues on the FP64 pipe)
__device__ __forceinline__ bool is_one(double x) { return __double_as_longlong(x) == 0x3FF0000000000000LL; }

// Argument checks shared by bf_dposv_mixed_batched and its allocation-free
// form (argument positions 1..19 of both signatures).
int posv_mixed_check(int batch, int n, int nrhs, const bf_dmat *sA, int ai, int aj, long long strideA,
                     const bf_dmat *sB, int bi, int bj, long long strideB, const bf_dmat *sX, int xi,
                     int xj, long long strideX, double tol, int max_iter, const int *iters,
                     const double *resid);

// The FP64 iterative refinement of the mixed-precision solvers, given the
// FP32 factor l32 (panel-major, pm x n per problem) and its status info32.
cudaError_t launch_posv_refine(int batch, int n, int nrhs, Op A, Op B, OpW X, double tol, int max_iter, int *iters,
                               double *resid, const float *l32, const int *info32, cudaStream_t s);

// Tensor-core trailing update lower(D) = C - L L^T (bf_tc.cu): L m x k, m <= 128,
// k <= 32 even, L's rows on a panel top and 16-byte aligned; prec 0 BF16,
// 1 TF32, 2 3xTF32.  err[b] = -3 if a wait timed out (err may be NULL).
bool syrk_tc_ok(int m, int k, const Op &L);
cudaError_t launch_syrk_tc(int prec, int batch, int m, int k, Op L, Op C, OpW D, int *err, cudaStream_t s);
// Blocked mixed-precision factorization (FP64 diagonal blocks and panels,
// tensor-core trailing updates) followed by the refinement.
cudaError_t launch_posv_mixed_tc(int prec, int batch, int n, int nrhs, Op A, Op B, OpW X, double tol, int max_iter,
                                 int *iters, double *resid, double *W, double *dinv, float *l32, int *infos,
                                 int *info32, cudaStream_t s);

// LU with partial pivoting (square n <= 512; blocked from n = 96) and
// Householder LQ (m*n <= 16384, or m, n <= 512 blocked).
cudaError_t launch_getrf(int batch, int n, Op C, OpW D, int *ipiv, long long sipiv, int *info, cudaStream_t s);
cudaError_t launch_gelqf(int batch, int m, int n, Op C, OpW D, double *tau, long long stau, cudaStream_t s);
constexpr int GETRF_MAX_N = 512;
constexpr int LU_ONE_CTA_MAX_N = 128;  // the whole-matrix-in-shared-memory getrf kernels
constexpr int GELQF_ONE_CTA_MAX_MN = 16384;  // the whole-matrix-in-shared-memory gelqf kernels
constexpr int GELQF_MAX_DIM = 512;           // the blocked gelqf: m, n <= 512

// Backward Riccati recursion, square-root form (one CTA per instance).
size_t riccati_smem(int max_nx, int max_nu);
cudaError_t launch_riccati(int batch, int N, const bf_riccati_prob *probs, const int *order,
                           int max_nx, int max_nu, int threads, cudaStream_t s);

cudaError_t launch_pack(int batch, int m, int n, const double *A, int lda, long long sA, OpW B,
                        cudaStream_t s);
cudaError_t launch_unpack(int batch, int m, int n, Op A, double *B, int ldb, long long sB,
                          cudaStream_t s);

// ---- kernel layouts (the candidates that bf_layout_set can force and the
// autotuner times; 0 everywhere means the built-in rule) --------------------
enum {
  ROUTINE_GEMM_NT = 0,
  ROUTINE_SYRK_LN = 1,
  ROUTINE_POTRF = 2,
  ROUTINE_TRSM_RLTN = 3,
  ROUTINE_SYRK_POTRF = 4,
  ROUTINE_GETRF = 5,
  ROUTINE_GELQF = 6,
  ROUTINE_COUNT = 7
};
// gemm_nt / syrk_ln: the k-loop of a 4x4 block split over KS lanes
enum { LAYOUT_GEMM_KS1 = 1, LAYOUT_GEMM_KS2 = 2, LAYOUT_GEMM_KS4 = 3, LAYOUT_GEMM_COUNT = 4 };
// potrf / syrk_potrf
enum {
  LAYOUT_CHOL_TINY = 1,      // one lane per problem, registers (n <= 8)
  LAYOUT_CHOL_SMALL_G2 = 2,  // k_chol_small with G = 2, 4, 8, 16, 32 lanes per problem (n <= 31)
  LAYOUT_CHOL_SMALL_G4 = 3,
  LAYOUT_CHOL_SMALL_G8 = 4,
  LAYOUT_CHOL_SMALL_G16 = 5,
  LAYOUT_CHOL_SMALL_G32 = 6,
  LAYOUT_CHOL_ROWS = 7,      // one thread per row, problems per CTA by rule (n <= 512)
  LAYOUT_CHOL_LAT = 8,       // one problem per CTA of four warps (n <= 32)
  LAYOUT_CHOL_SPLIT = 9,     // syrk_potrf: the sum by the syrk kernel, then the row kernels
  LAYOUT_CHOL_BLOCKED = 10,  // two diagonal blocks: potrf, trsm, syrk, potrf (n >= 32)
  LAYOUT_CHOL_ROWS8 = 11,    // one thread per row, eight problems per CTA, 4-column blocks (n <= 64)
  LAYOUT_CHOL_COUNT = 12
};
// trsm_rltn
enum { LAYOUT_TRSM_ROWS = 1, LAYOUT_TRSM_LAT2 = 2, LAYOUT_TRSM_LAT4 = 3, LAYOUT_TRSM_LAT8 = 4, LAYOUT_TRSM_COUNT = 5 };
// getrf: one warp per 32/G problems (n <= 128), one CTA per problem (n <=
// 128), blocked by columns of 32 or 16 (n <= 512)
enum { LAYOUT_LU_WARP = 1, LAYOUT_LU_ROWS = 2, LAYOUT_LU_BLOCKED = 3, LAYOUT_LU_BLOCKED16 = 4, LAYOUT_LU_COUNT = 5 };
// gelqf: one warp per 32/G problems, one CTA per problem (both m*n <=
// 16384), blocked by rows of 32 or 16 (m, n <= 512)
enum { LAYOUT_LQ_WARP = 1, LAYOUT_LQ_ROWS = 2, LAYOUT_LQ_BLOCKED = 3, LAYOUT_LQ_BLOCKED16 = 4, LAYOUT_LQ_COUNT = 5 };

// Layout forced for (routine, n, batch) by bf_layout_set, or 0.
int layout_forced(int routine, int n, int batch);
// The built-in rules, and whether a candidate supports order n.
int chol_layout_rule(bool fused, int batch, int n);
bool chol_layout_ok(int layout, int n);
int gemm_layout_rule(bool syrk, int batch, int m, int n, int k);
int trsm_layout_rule(int batch, int m, int n);
bool trsm_layout_ok(int layout, int n);
int getrf_layout_rule(int batch, int n);
bool getrf_layout_ok(int layout, int n);
int gelqf_layout_rule(int batch, int m, int n);
bool gelqf_layout_ok(int layout, int m, int n);

// Latency kernels (bf_latency.cu): one problem per CTA of four warps for
// potrf / syrk_potrf, R = lanes lanes per row for trsm; order <= 32.
cudaError_t launch_chol_lat(bool fused, int batch, int n, int k, Op A, Op B, Op C, OpW D, double *dinv,
                            long long sdinv, int *info, cudaStream_t s);
cudaError_t launch_trsm_lat(int lanes, int batch, int m, int n, double alpha, Op L, const double *dinv,
                            long long sdinv, Op B, OpW D, cudaStream_t s);
#ifndef BF_CHOL_LAT_MAX_N
#define BF_CHOL_LAT_MAX_N 32
#endif
// the latency kernel serves batches of at most this many problems per SM
// (measured single launches, potrf / syrk_potrf n = 8..32: the latency
// kernel is fastest up to 512 problems, ties the others at 1024)
#ifndef BF_CHOL_LAT_MAX_BATCH_PER_SM
#define BF_CHOL_LAT_MAX_BATCH_PER_SM 4
#endif

// Largest order the factorization kernels accept.
constexpr int CHOL_MAX_N = 512;
constexpr int TRSM_MAX_N = 4096;
// Orders of the solves, set by what one CTA holds in shared memory (at most
// 200 KB, eight right-hand sides): the mixed refinement keeps the FP32 factor
// and two FP64 copies of the right-hand sides (165 KB at n = 256); the FP64
// solve the FP64 factor and one copy (199 KB at 216); the adjoint the FP64
// factor and two copies (198 KB at 208).  The blocked tensor-core form's
// first trailing update must fit one 128-row MMA tile: n - 32 <= 128.
constexpr int POSV_MAX_N = 256;
constexpr int POTRS_MAX_N = 216;
constexpr int ADJOINT_MAX_N = 208;
constexpr int POSV_TC_MAX_N = 160;
constexpr int POSV_MAX_NRHS = 8;

}  // namespace bf
