// Packing between column-major and panel-major storage (Sec. 4.3.3; the
// packing routines of the auxiliary set, Appendix A.3).  Element (i, j) of the
// column-major matrix (leading dimension ld) maps to element (r, c) = (i0+i,
// j0+j) of the panel-major one, at (r - r%ps)*cn + c*ps + r%ps.
//
// The column-major side may be device memory, mapped (pinned or registered)
// host memory, or plain pageable host memory:
//   - device and mapped host memory: the kernel below copies, one thread per
//     element; over mapped memory it reads or writes the host directly;
//   - pageable host memory: one strided copy per panel row group and
//     problem (cudaMemcpy2DAsync), since no kernel may touch it.
// Packing is quadratic work that the paper amortizes off the hot path
// (Sec. 4.3.3).
#include "bf_internal.cuh"

namespace bf {
namespace {

// One thread per element of the column-major side, in grid-stride order
// over the whole batch: a warp reads (or writes) 32 consecutive elements of
// a column.  That keeps the column-major side coalesced when it is host
// memory that the kernel reaches over the host link (mapped pinned memory).
// Each thread issues the loads of U elements before their stores, so that a
// small grid keeps many loads in flight: the grid is capped so that a copy
// over the host link does not fill the GPU with warps that wait on it.
template <bool PACK>
__global__ void __launch_bounds__(256)
k_pack(int batch, int m, int n, const double *cm_in, double *cm_out, int ld, long long scm,
       const double *pm_in, double *pm_out, int cn, long long spm, int i0, int j0) {
  constexpr int U = 4;
  const long long per = (long long)m * n;
  const long long total = per * batch;
  const long long step = (long long)gridDim.x * blockDim.x;
  for (long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; t0 < total; t0 += U * step) {
    double v[U];
    long long cmo[U], pmo[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const long long t = t0 + u * step;
      if (t < total) {
        const int b = (int)(t / per);
        const long long e = t - (long long)b * per;
        const int i = (int)(e % m);
        const int j = (int)(e / m);
        cmo[u] = (long long)b * scm + (long long)j * ld + i;
        pmo[u] = (long long)b * spm + pm_off(i0 + i, j0 + j, cn);
        v[u] = PACK ? cm_in[cmo[u]] : pm_in[pmo[u]];
      }
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
      if (t0 + u * step < total) {
        if (PACK)
          pm_out[pmo[u]] = v[u];
        else
          cm_out[cmo[u]] = v[u];
      }
    }
  }
}

// Where the column-major side lives, as seen from the current device.
enum class Side { kDevice, kMapped, kPageable };

// Classifies p (cudaPointerGetAttributes) and gives the address a kernel may
// dereference for it (*dp), if any.
Side classify(const void *p, const void **dp) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    (void)cudaGetLastError();  // not a pointer the runtime knows: plain host memory
    *dp = nullptr;
    return Side::kPageable;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
    *dp = p;
    return Side::kDevice;
  }
  if (at.type == cudaMemoryTypeHost && at.devicePointer) {
    *dp = at.devicePointer;
    return Side::kMapped;
  }
  *dp = nullptr;
  return Side::kPageable;
}

unsigned grid_for(long long total, Side side) {
  const long long blocks = (total + 255) / 256;
  // device memory: up to 16 CTAs per SM, each looping; mapped host memory:
  // one per SM (four loads in flight per thread) for the host link
  const long long cap = (long long)device_sm_count() * (side == Side::kMapped ? 1 : 16);
  return (unsigned)(blocks < cap ? blocks : cap);
}

}  // namespace

cudaError_t launch_pack(int batch, int m, int n, const double *A, int lda, long long sA, OpW B,
                        cudaStream_t s) {
  const long long total = (long long)batch * m * n;
  const void *dp = nullptr;
  const Side side = classify(A, &dp);
  if (side == Side::kPageable) {
    // plain host memory: one strided copy per panel row group and problem
    // (the rows of a panel are ps consecutive doubles on both sides)
    for (int b = 0; b < batch; b++)
      for (int i = 0; i < m;) {
        const int r = B.i0 + i;
        const int rows = (PS - (r & (PS - 1))) < (m - i) ? (PS - (r & (PS - 1))) : (m - i);
        double *dst = B.p + (long long)b * B.stride + pm_off(r, B.j0, B.cn);
        const double *src = A + (long long)b * sA + i;
        const cudaError_t e = cudaMemcpy2DAsync(dst, PS * sizeof(double), src, (size_t)lda * sizeof(double),
                                                (size_t)rows * sizeof(double), (size_t)n, cudaMemcpyDefault, s);
        if (e != cudaSuccess) return e;
        i += rows;
      }
    return cudaSuccess;
  }
  k_pack<true><<<grid_for(total, side), 256, 0, s>>>(batch, m, n, (const double *)dp, nullptr, lda, sA,
                                                       nullptr, B.p, B.cn, B.stride, B.i0, B.j0);
  return cudaGetLastError();
}

cudaError_t launch_unpack(int batch, int m, int n, Op A, double *B, int ldb, long long sB,
                          cudaStream_t s) {
  const long long total = (long long)batch * m * n;
  const void *dp = nullptr;
  const Side side = classify(B, &dp);
  if (side == Side::kPageable) {
    for (int b = 0; b < batch; b++)
      for (int i = 0; i < m;) {
        const int r = A.i0 + i;
        const int rows = (PS - (r & (PS - 1))) < (m - i) ? (PS - (r & (PS - 1))) : (m - i);
        const double *src = A.p + (long long)b * A.stride + pm_off(r, A.j0, A.cn);
        double *dst = B + (long long)b * sB + i;
        const cudaError_t e = cudaMemcpy2DAsync(dst, (size_t)ldb * sizeof(double), src, PS * sizeof(double),
                                                (size_t)rows * sizeof(double), (size_t)n, cudaMemcpyDefault, s);
        if (e != cudaSuccess) return e;
        i += rows;
      }
    return cudaSuccess;
  }
  k_pack<false><<<grid_for(total, side), 256, 0, s>>>(batch, m, n, nullptr, (double *)dp, ldb, sB, A.p,
                                                        nullptr, A.cn, A.stride, A.i0, A.j0);
  return cudaGetLastError();
}

}  // namespace bf
