// bf_dposv_mixed_batched_noalloc: the mixed-precision SPD solver for callers
// that cannot allocate device memory.
//
// bf_dposv_mixed_batched needs scratch memory for the single-precision
// factors, and it takes that scratch from the caller.  Some callers have no
// way to provide it.  A controller running a fixed-period loop may forbid
// allocation on that path, because cudaMalloc can block the whole device and
// can fail at run time.  A plugin may live inside a host application that
// owns all device memory and exposes no allocator.  This entry point serves
// them: its scratch is a fixed array in the library's own device memory.
//
// Properties a caller must know:
//   - The array is BF_NOALLOC_WORK_BYTES (16 MiB) of static device memory.
//     Every GPU that loads this library holds it until the process exits.
//   - Problems are limited to bf_dposv_mixed_worksize(batch, n) <=
//     BF_NOALLOC_WORK_BYTES.  Larger calls return BF_ERR_TOO_LARGE and
//     launch nothing.
//   - The first call on each device looks up the array's device address with
//     cudaGetSymbolAddress, with that device current.  Make that first call
//     before any stream capture on the device.  The address is kept for the
//     life of the process, so no cudaDeviceReset (or other reset of the
//     device's primary context) may come between calls: the array can move.
//   - Every call shares the one array, and it keeps the last call's contents.
//     Nothing in it needs to start at zero: the factorization writes every
//     factor element and status word that the solve later reads.  Calls whose
//     kernels overlap on the GPU (different streams, or other threads) race
//     on the array and corrupt each other's results; serialize them.
//   - It allocates nothing and frees nothing.
#include <mutex>

#include "bf_internal.cuh"

namespace {

static __device__ __align__(256) unsigned char g_posv_scratch[BF_NOALLOC_WORK_BYTES];

constexpr int kMaxDevices = 64;
void *g_scratch_ptr[kMaxDevices];  // device address of g_posv_scratch, per device
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device; looked up once.
cudaError_t scratch_on_current_device(void **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_posv_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int bf_dposv_mixed_batched_noalloc(int batch, int n, int nrhs, const bf_dmat *sA,
                                              int ai, int aj, long long strideA, const bf_dmat *sB,
                                              int bi, int bj, long long strideB, const bf_dmat *sX,
                                              int xi, int xj, long long strideX, double tol,
                                              int max_iter, int *iters, double *resid,
                                              void *stream) {
  // argument errors first, with the workspace form's codes; only a valid
  // call that does not fit the array gets BF_ERR_TOO_LARGE
  if (int r = bf::posv_mixed_check(batch, n, nrhs, sA, ai, aj, strideA, sB, bi, bj, strideB, sX, xi, xj,
                                   strideX, tol, max_iter, iters, resid))
    return r;
  if (batch == 0 || n == 0 || nrhs == 0) return 0;
  if (bf_dposv_mixed_worksize(batch, n) > (size_t)BF_NOALLOC_WORK_BYTES) return BF_ERR_TOO_LARGE;
  void *scratch = nullptr;
  const cudaError_t e = scratch_on_current_device(&scratch);
  if (e != cudaSuccess) return (int)e;
  // the same checks and kernels as the workspace form; the arguments up to
  // resid have the same positions, so its error codes carry over unchanged
  return bf_dposv_mixed_batched(batch, n, nrhs, sA, ai, aj, strideA, sB, bi, bj, strideB, sX, xi, xj,
                                strideX, tol, max_iter, iters, resid, scratch,
                                (size_t)BF_NOALLOC_WORK_BYTES, stream);
}
