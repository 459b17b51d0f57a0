// peaks.cu -- throughput probes of the FP32 FMA pipe, used to state the
// roofline of the ALU-bound kernels (the one-sided Jacobi) against a peak
// measured on the device itself rather than derived from unit counts.
//
// Each thread runs eight independent FMA chains (sixteen with the paired
// instruction __ffma2_rn), long enough to hide the FMA latency at 32 warps
// per SM; the result is stored only under a condition that never holds, so
// the work is kept but nothing is written.
#include "lrstv_internal.cuh"

namespace lrstv {

namespace {

template <int PAIRED>
__global__ void __launch_bounds__(256) k_fma_peak(long long iters, float seed, float *sink) {
  const float b = 0.99999994f, c = 1.0e-8f;
  float s = 0.0f;
  if (PAIRED) {
    float2 a[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = make_float2(seed + 1e-3f * (float)u, seed - 1e-3f * (float)u);
    const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
#pragma unroll 4
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = __ffma2_rn(a[u], b2, c2);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) s += a[u].x + a[u].y;
  } else {
    float a[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = seed + 1e-3f * (float)u;
#pragma unroll 4
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = fmaf(a[u], b, c);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) s += a[u];
  }
  if (s == -1.0f) sink[threadIdx.x] = s;  // never: the chains stay positive
}

}  // namespace

cudaError_t launch_fma_peak(int paired, int nsm, long long iters, float *sink, cudaStream_t st,
                            double *flops) {
  const int blocks = nsm * 4, threads = 256;  // 32 warps per SM
  *flops = 2.0 * (paired ? 16.0 : 8.0) * (double)iters * blocks * threads;
  if (paired)
    k_fma_peak<1><<<blocks, threads, 0, st>>>(iters, 0.5f, sink);
  else
    k_fma_peak<0><<<blocks, threads, 0, st>>>(iters, 0.5f, sink);
  return cudaGetLastError();
}

}  // namespace lrstv
