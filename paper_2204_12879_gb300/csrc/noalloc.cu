// noalloc.cu -- lrstv_tsvt_noalloc: the standalone t-SVT for callers that
// cannot allocate device memory when they call it.
//
// Some callers are not free to allocate: a plug-in whose host application
// owns the device's memory pool, a process that reserves all of its device
// memory up front, or a latency-critical loop that must never reach the
// driver's allocator.  They can pass inputs and outputs but no workspace.
// This entry point takes its scratch from one file-scope device array of
// LRSTV_NOALLOC_SCRATCH_BYTES instead.  The array is part of the loaded
// library, so every GPU that loads liblrstv.so holds it until the process
// exits; the entry point itself calls no cudaMalloc, cudaFree or other
// allocating routine.
#include <math.h>

#include "lrstv.h"
#include "lrstv_internal.cuh"

namespace {

static __device__ __align__(256) unsigned char g_scratch[LRSTV_NOALLOC_SCRATCH_BYTES];

// The name g_scratch in host code is only a host-side handle for the symbol;
// the array's device address belongs to the context that loaded this file's
// device code.  It is asked for on every call, in the calling thread's current
// context: a cached address would go stale if the host application tore its
// context down and made a new one (cudaDeviceReset, or a driver-API context of
// its own).  Once the module is loaded the lookup allocates nothing.
int scratch_address(void **out) {
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
    cudaGetLastError();
    return LRSTV_ERR_CUDA;
  }
  *out = p;
  return LRSTV_OK;
}

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" int lrstv_tsvt_noalloc(const float *A, int n1, int n2, int n3, float t, float *out,
                                  int *sweeps_host, void *stream) {
  // the argument and shape checks of lrstv_tsvt
  if (!A || !out) return LRSTV_ERR_ARG;
  const int rc_shape = lrstv::check_shape(n1, n2, n3);
  if (rc_shape != LRSTV_OK) return rc_shape;
  if (!isfinite(t) || t < 0.0f) return LRSTV_ERR_ARG;
  const lrstv::Dims d = lrstv::make_dims(n1, n2, n3);
  // scratch layout: specA, specB (h P complex), V (h nc^2 complex), twiddles, sweeps
  const size_t spec = up256(sizeof(float2) * (size_t)d.h * d.P);
  const size_t vbytes = up256(sizeof(float2) * (size_t)d.h * d.nc * d.nc);
  const size_t twb = up256(sizeof(float2) * (size_t)d.n3);
  const size_t swb = up256(sizeof(int) * (size_t)d.h);
  if (2 * spec + vbytes + twb + swb > (size_t)LRSTV_NOALLOC_SCRATCH_BYTES) return LRSTV_ERR_SHAPE;
  void *base = nullptr;
  int rc = scratch_address(&base);
  if (rc != LRSTV_OK) return rc;
  char *c = (char *)base;
  float2 *specA = (float2 *)c;
  float2 *specB = (float2 *)(c + spec);
  float2 *V = (float2 *)(c + 2 * spec);
  float2 *tw = (float2 *)(c + 2 * spec + vbytes);
  int *sw = (int *)(c + 2 * spec + vbytes + twb);
  cudaStream_t st = (cudaStream_t)stream;
  if (lrstv::tsvt_plain(d, A, t, out, tw, specA, specB, V, sw, st) != cudaSuccess) {
    cudaGetLastError();
    return LRSTV_ERR_CUDA;
  }
  if (sweeps_host) {
    int h[lrstv::kMaxBands / 2 + 1];  // h <= n3/2 + 1 slices
    if (cudaMemcpyAsync(h, sw, sizeof(int) * d.h, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      cudaGetLastError();
      return LRSTV_ERR_CUDA;
    }
    int worst = 0, capped = 0;
    for (int k = 0; k < d.h; ++k) {
      if (h[k] < 0) capped = h[k];
      else if (h[k] > worst) worst = h[k];
    }
    *sweeps_host = capped ? capped : worst;
  }
  return LRSTV_OK;
}
