// Microbenchmarks of the GB300 FP64 pipe, behind the design's roofline and
// its lane-utilization arguments.  Prints one JSON line:
//   dfma_full_gflops   DFMA throughput, full warps, 8 independent chains
//   dfma_1lane_ratio   time of the same instruction stream with one active
//                      lane per warp over the full-warp time (1.0: a masked
//                      lane costs as much as an active one)
//   dfma_ilp1_4warps   DFMA throughput with 4 warps per SM and one dependent
//                      chain per thread (one warp per SM sub-partition)
//   dmma_gflops        mma.sync m8n8k4 f64 throughput
//   mixed_*            half the warps of each CTA in a DFMA loop, half in an
//                      mma.sync f64 loop: the time of both together against
//                      each alone tells whether the two share one pipe
//   ffma_gflops        FP32 FMA throughput
//   sqrt_ops, rcp_ops, rsqrt_ops   (x -> f(x) + 1) per second, FP64
// All loops have fixed trip counts.
#include <cuda_runtime.h>

#include <cstdio>

#define CK(x)                                                                  \
  do {                                                                         \
    cudaError_t e_ = (x);                                                      \
    if (e_ != cudaSuccess) {                                                   \
      printf("{\"error\": \"%s at line %d\"}\n", cudaGetErrorString(e_), __LINE__); \
      return 1;                                                                \
    }                                                                          \
  } while (0)

template <int ILP>
__global__ void k_dfma(double *out, int iters, double b, double c, int one_lane) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (one_lane && (threadIdx.x & 31) != 0) return;
  double a[ILP];
#pragma unroll
  for (int i = 0; i < ILP; i++) a[i] = 1.0 + 1e-3 * i + 1e-9 * tid;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < ILP; i++) a[i] = fma(a[i], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < ILP; i++) s += a[i];
  out[tid] = s;
}

__global__ void k_ffma(float *out, int iters, float b, float c) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  float a[8];
#pragma unroll
  for (int i = 0; i < 8; i++) a[i] = 1.0f + 1e-3f * i;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < 8; i++) a[i] = fmaf(a[i], b, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < 8; i++) s += a[i];
  out[tid] = s;
}

// mma.sync m8n8k4 f64: 2*8*8*4 = 512 flops per warp instruction
__global__ void k_dmma(double *out, int iters) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const double a = 1.0 + 1e-6 * (threadIdx.x & 31), b = 0.5;
  double c0[4], c1[4];
#pragma unroll
  for (int i = 0; i < 4; i++) c0[i] = c1[i] = 0.0;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < 4; i++)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                   : "+d"(c0[i]), "+d"(c1[i])
                   : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 4; i++) s += c0[i] + c1[i];
  out[tid] = s;
}

// Even warps: the DFMA loop of k_dfma<8>; odd warps: the mma.sync loop of
// k_dmma.  which: 0 both, 1 DFMA warps only, 2 MMA warps only.
__global__ void k_mixed(double *out, int iters_f, int iters_m, int which) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int warp = threadIdx.x >> 5;
  double s = 0.0;
  if ((warp & 1) == 0) {
    if (which == 2) return;
    double a[8];
#pragma unroll
    for (int i = 0; i < 8; i++) a[i] = 1.0 + 1e-3 * i + 1e-9 * tid;
    for (int it = 0; it < iters_f; it++) {
#pragma unroll
      for (int i = 0; i < 8; i++) a[i] = fma(a[i], 0.999999, 1e-6);
    }
#pragma unroll
    for (int i = 0; i < 8; i++) s += a[i];
  } else {
    if (which == 1) return;
    const double a = 1.0 + 1e-6 * (threadIdx.x & 31), b = 0.5;
    double c0[4], c1[4];
#pragma unroll
    for (int i = 0; i < 4; i++) c0[i] = c1[i] = 0.0;
    for (int it = 0; it < iters_m; it++) {
#pragma unroll
      for (int i = 0; i < 4; i++)
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                     : "+d"(c0[i]), "+d"(c1[i])
                     : "d"(a), "d"(b));
    }
#pragma unroll
    for (int i = 0; i < 4; i++) s += c0[i] + c1[i];
  }
  out[tid] = s;
}

// mode 0: sqrt, 1: reciprocal, 2: rsqrt (each followed by + 1)
__global__ void k_special(double *out, int iters, int mode) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  double x[4];
#pragma unroll
  for (int i = 0; i < 4; i++) x[i] = 2.0 + 1e-3 * i + 1e-9 * tid;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < 4; i++) {
      if (mode == 0)
        x[i] = sqrt(x[i]) + 1.0;
      else if (mode == 1)
        x[i] = 1.0 / x[i] + 1.0;
      else
        x[i] = rsqrt(x[i]) + 1.0;
    }
  }
  out[tid] = x[0] + x[1] + x[2] + x[3];
}

int main() {
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
  const int threads = 256;
  double *dout;
  float *fout;
  CK(cudaMalloc(&dout, (size_t)sms * 8 * threads * sizeof(double)));
  CK(cudaMalloc(&fout, (size_t)sms * 8 * threads * sizeof(float)));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float ms = 0.0f;

  // DFMA: 4 blocks of 256 threads per SM, 8 chains per thread
  double t_full = 0.0, t_one = 0.0, gf_full = 0.0;
  {
    const int blocks = sms * 4, iters = 2000;
    for (int one = 0; one < 2; one++) {
      k_dfma<8><<<blocks, threads>>>(dout, 10, 0.999999, 1e-6, one);
      CK(cudaEventRecord(e0));
      k_dfma<8><<<blocks, threads>>>(dout, iters, 0.999999, 1e-6, one);
      CK(cudaEventRecord(e1));
      CK(cudaEventSynchronize(e1));
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (one)
        t_one = ms;
      else {
        t_full = ms;
        gf_full = 2.0 * 8 * iters * (double)blocks * threads / (ms * 1e-3) / 1e9;
      }
    }
  }
  // DFMA, one dependent chain per thread, 4 warps per SM
  double gf_ilp1 = 0.0;
  {
    const int blocks = sms, iters = 20000;
    k_dfma<1><<<blocks, 128>>>(dout, 10, 0.999999, 1e-6, 0);
    CK(cudaEventRecord(e0));
    k_dfma<1><<<blocks, 128>>>(dout, iters, 0.999999, 1e-6, 0);
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms, e0, e1));
    gf_ilp1 = 2.0 * iters * (double)blocks * 128 / (ms * 1e-3) / 1e9;
  }
  double gf_ffma = 0.0;
  {
    const int blocks = sms * 8, iters = 20000;
    k_ffma<<<blocks, threads>>>(fout, 10, 0.999f, 1e-3f);
    CK(cudaEventRecord(e0));
    k_ffma<<<blocks, threads>>>(fout, iters, 0.999f, 1e-3f);
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms, e0, e1));
    gf_ffma = 2.0 * 8 * iters * (double)blocks * threads / (ms * 1e-3) / 1e9;
  }
  double gf_dmma = 0.0;
  {
    const int blocks = sms * 2, iters = 2000;
    k_dmma<<<blocks, threads>>>(dout, 10);
    CK(cudaEventRecord(e0));
    k_dmma<<<blocks, threads>>>(dout, iters);
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms, e0, e1));
    gf_dmma = 512.0 * 4 * iters * (double)blocks * threads / 32 / (ms * 1e-3) / 1e9;
  }
  // DFMA and MMA warps side by side (4 CTAs of 8 warps per SM, 4 + 4 each)
  double t_mixed[3] = {0.0, 0.0, 0.0}, gf_mixed = 0.0;
  {
    const int blocks = sms * 4, iters_f = 2000, iters_m = 440;
    for (int which = 0; which < 3; which++) {
      k_mixed<<<blocks, threads>>>(dout, 10, 2, which);
      CK(cudaEventRecord(e0));
      k_mixed<<<blocks, threads>>>(dout, iters_f, iters_m, which);
      CK(cudaEventRecord(e1));
      CK(cudaEventSynchronize(e1));
      CK(cudaEventElapsedTime(&ms, e0, e1));
      t_mixed[which] = ms;
    }
    const double warps_half = (double)blocks * threads / 64;
    const double flops = warps_half * (32.0 * 2 * 8 * iters_f + 512.0 * 4 * iters_m);
    gf_mixed = flops / (t_mixed[0] * 1e-3) / 1e9;
  }
  double special[3] = {0.0, 0.0, 0.0};
  for (int mode = 0; mode < 3; mode++) {
    const int blocks = sms * 8, iters = 500;
    k_special<<<blocks, threads>>>(dout, 10, mode);
    CK(cudaEventRecord(e0));
    k_special<<<blocks, threads>>>(dout, iters, mode);
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms, e0, e1));
    special[mode] = 4.0 * iters * (double)blocks * threads / (ms * 1e-3);
  }
  CK(cudaGetLastError());
  printf("{\"sms\": %d, \"dfma_full_gflops\": %.1f, \"dfma_1lane_ratio\": %.3f, \"dfma_ilp1_4warps_gflops\": %.1f, "
         "\"dmma_gflops\": %.1f, \"ffma_gflops\": %.1f, \"sqrt_ops\": %.4g, \"rcp_ops\": %.4g, \"rsqrt_ops\": %.4g, "
         "\"mixed_ms_both\": %.4f, \"mixed_ms_dfma_only\": %.4f, \"mixed_ms_mma_only\": %.4f, "
         "\"mixed_gflops\": %.1f}\n",
         sms, gf_full, t_one / t_full, gf_ilp1, gf_dmma, gf_ffma, special[0], special[1], special[2], t_mixed[0],
         t_mixed[1], t_mixed[2], gf_mixed);
  CK(cudaFree(dout));
  CK(cudaFree(fout));
  return 0;
}
