// Packing between column-major and panel-major storage (Sec. 4.3.3; the
// packing routines of the auxiliary set, Appendix A.3).  Element (i, j) of the
// column-major matrix (leading dimension ld) maps to element (r, c) = (i0+i,
// j0+j) of the panel-major one, at (r - r%ps)*cn + c*ps + r%ps.
//
// One thread per element, numbered in column-major order: the column-major
// side is contiguous within a warp and the panel side comes in runs of ps
// consecutive doubles.  Packing
// is quadratic work that the paper amortizes off the hot path (Sec. 4.3.3),
// and it runs off the timed path here too.
#include "bf_internal.cuh"

namespace bf {
namespace {

template <bool PACK>
__global__ void __launch_bounds__(256)
k_pack(int batch, int m, int n, const double *cm_in, double *cm_out, int ld, long long scm,
       const double *pm_in, double *pm_out, int cn, long long spm, int i0, int j0) {
  const long long per = (long long)m * n;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per * batch) return;
  const int b = (int)(t / per);
  const long long e = t - (long long)b * per;
  const int i = (int)(e % m);
  const int j = (int)(e / m);
  const long long cmo = (long long)b * scm + (long long)j * ld + i;
  const long long pmo = (long long)b * spm + pm_off(i0 + i, j0 + j, cn);
  if (PACK)
    pm_out[pmo] = __ldg(cm_in + cmo);
  else
    cm_out[cmo] = __ldg(pm_in + pmo);
}

}  // namespace

cudaError_t launch_pack(int batch, int m, int n, const double *A, int lda, long long sA, OpW B,
                        cudaStream_t s) {
  const long long total = (long long)batch * m * n;
  const long long blocks = (total + 255) / 256;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  k_pack<true><<<(unsigned)blocks, 256, 0, s>>>(batch, m, n, A, nullptr, lda, sA, nullptr, B.p,
                                                B.cn, B.stride, B.i0, B.j0);
  return cudaGetLastError();
}

cudaError_t launch_unpack(int batch, int m, int n, Op A, double *B, int ldb, long long sB,
                          cudaStream_t s) {
  const long long total = (long long)batch * m * n;
  const long long blocks = (total + 255) / 256;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  k_pack<false><<<(unsigned)blocks, 256, 0, s>>>(batch, m, n, nullptr, B, ldb, sB, A.p, nullptr,
                                                 A.cn, A.stride, A.i0, A.j0);
  return cudaGetLastError();
}

}  // namespace bf
