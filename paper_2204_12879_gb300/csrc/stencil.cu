// stencil.cu -- HBM-bound voxel kernels of the LRSTV ADMM iteration
// (arXiv 2204.12879, Section III-C): the fused L-update / T_z assembly, the
// fused F / S / multiplier update, and the standalone difference operators.
//
// Thread mapping: one thread per (i, j) pixel column and a chunk of bands k;
// a warp spans 32 consecutive i (coalesced 128-byte rows).  Walking k inside
// the thread keeps the mode-3 neighbour in a register, so each cube is read
// once; the mode-1 / mode-2 neighbours come from L1 (the same block read
// them).  Chunks of k are sized so the grid fills all SMs several times.
#include "lrstv_internal.cuh"

namespace lrstv {

namespace {

constexpr int kBX = 32, kBY = 8;

// max that keeps a NaN (fmaxf drops it), so non-finite iterates show in the residual
__device__ __forceinline__ float nanmax(float a, float b) {
  return (a != a || b != b) ? __int_as_float(0x7fc00000) : fmaxf(a, b);
}

__device__ __forceinline__ float soft_thr(float x, float d) {
  // R_d(x) = sign(x) max(|x| - d, 0)
  return x > d ? x - d : (x < -d ? x + d : 0.0f);
}

struct Chunking {
  dim3 grid;
  int kchunk;
};

Chunking chunking(const Dims &d) {
  // aim for ~2048 resident threads on each of 152 SMs, four times over
  const size_t want = 152ull * 2048ull * 4ull;
  size_t cols = d.P;
  int chunks = (int)((want + cols - 1) / cols);
  if (chunks < 1) chunks = 1;
  if (chunks > d.n3) chunks = d.n3;
  int kchunk = (d.n3 + chunks - 1) / chunks;
  chunks = (d.n3 + kchunk - 1) / kchunk;
  Chunking c;
  c.grid = dim3((d.n1 + kBX - 1) / kBX, (d.n2 + kBY - 1) / kBY, chunks);
  c.kchunk = kchunk;
  return c;
}

__global__ void __launch_bounds__(kBX *kBY)
    k_l_tz(int n1, int n2, int n3, size_t N, int kchunk, const float *__restrict__ Y,
           const float *__restrict__ S, const float *__restrict__ Z, const float *__restrict__ G1,
           const float *__restrict__ G2, const float *__restrict__ F, const float *__restrict__ G3,
           float mu, float w0, float w1, float w2, float *__restrict__ L, float *__restrict__ T) {
  const int i = blockIdx.x * kBX + threadIdx.x;
  const int j = blockIdx.y * kBY + threadIdx.y;
  if (i >= n1 || j >= n2) return;
  const int k0 = blockIdx.z * kchunk;
  const int k1 = min(n3, k0 + kchunk);
  const size_t P = (size_t)n1 * n2;
  const size_t col = (size_t)i + (size_t)n1 * j;
  const size_t colm1 = (i == 0) ? col + n1 - 1 : col - 1;                 // v - e1
  const size_t colm2 = (j == 0) ? col + (size_t)n1 * (n2 - 1) : col - n1;  // v - e2
  const float *F1 = F, *F2 = F + N, *F3 = F + 2 * N;
  const float *H1 = G3, *H2 = G3 + N, *H3 = G3 + 2 * N;
  // q_n = mu F_n - Gamma3_n; D_n^T q(v) = q(v - e_n) - q(v)
  const int km = (k0 == 0) ? n3 - 1 : k0 - 1;
  float q3prev = mu * F3[col + P * km] - H3[col + P * km];
  for (int k = k0; k < k1; ++k) {
    const size_t v = col + P * k;
    const size_t vm1 = colm1 + P * k;
    const size_t vm2 = colm2 + P * k;
    const float q1 = mu * F1[v] - H1[v], q1m = mu * F1[vm1] - H1[vm1];
    const float q2 = mu * F2[v] - H2[v], q2m = mu * F2[vm2] - H2[vm2];
    const float q3 = mu * F3[v] - H3[v];
    const float adj = w0 * (q1m - q1) + w1 * (q2m - q2) + w2 * (q3prev - q3);
    const float g2 = G2[v];
    const float l = 0.5f * (Y[v] - S[v] + Z[v] + (G1[v] - g2) / mu);
    L[v] = l;
    T[v] = mu * l + g2 + adj;
    q3prev = q3;
  }
}

__global__ void __launch_bounds__(kBX *kBY)
    k_fs_dual(int n1, int n2, int n3, size_t N, int kchunk, const float *__restrict__ Y,
              const float *__restrict__ L, const float *__restrict__ Z, float *__restrict__ S,
              float *__restrict__ G1, float *__restrict__ G2, float *__restrict__ F,
              const float *__restrict__ E, float *__restrict__ G3, const float *__restrict__ G4,
              float mu, float thr_f, float thr_s, float w0, float w1, float w2,
              unsigned *__restrict__ res2) {
  const int i = blockIdx.x * kBX + threadIdx.x;
  const int j = blockIdx.y * kBY + threadIdx.y;
  float r1max = 0.0f, r2max = 0.0f;
  if (i < n1 && j < n2) {
    const int k0 = blockIdx.z * kchunk;
    const int k1 = min(n3, k0 + kchunk);
    const size_t P = (size_t)n1 * n2;
    const size_t col = (size_t)i + (size_t)n1 * j;
    const size_t colp1 = (i == n1 - 1) ? col + 1 - n1 : col + 1;                 // v + e1
    const size_t colp2 = (j == n2 - 1) ? col - (size_t)n1 * (n2 - 1) : col + n1;  // v + e2
    float zc = Z[col + P * k0];
    for (int k = k0; k < k1; ++k) {
      const size_t v = col + P * k;
      const int kp = (k == n3 - 1) ? 0 : k + 1;
      const float z3 = Z[col + P * kp];
      const float g[3] = {w0 * (Z[colp1 + P * k] - zc), w1 * (Z[colp2 + P * k] - zc),
                          w2 * (z3 - zc)};
#pragma unroll
      for (int n = 0; n < 3; ++n) {
        const size_t vn = v + (size_t)n * N;
        const float h3 = G3[vn];
        const float t1 = g[n] + h3 / mu;
        const float t2 = E[vn] + G4[vn] / mu;
        const float f = soft_thr(0.5f * (t1 + t2), thr_f);
        F[vn] = f;
        G3[vn] = h3 + mu * (g[n] - f);
      }
      const float y = Y[v], l = L[v], g1 = G1[v];
      const float s = soft_thr(y - l + g1 / mu, thr_s);
      S[v] = s;
      const float r1 = y - l - s;
      const float r2 = l - zc;
      G1[v] = g1 + mu * r1;
      G2[v] = G2[v] + mu * r2;
      r1max = nanmax(r1max, fabsf(r1));
      r2max = nanmax(r2max, fabsf(r2));
      zc = z3;
    }
  }
  if (res2 == nullptr) return;
  // block max (order-independent, so the result is deterministic)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    r1max = nanmax(r1max, __shfl_xor_sync(0xffffffffu, r1max, o));
    r2max = nanmax(r2max, __shfl_xor_sync(0xffffffffu, r2max, o));
  }
  __shared__ float s1[kBY], s2[kBY];
  const int lane = threadIdx.x, wid = threadIdx.y;
  if (lane == 0) { s1[wid] = r1max; s2[wid] = r2max; }
  __syncthreads();
  if (wid == 0) {
    r1max = lane < kBY ? s1[lane] : 0.0f;
    r2max = lane < kBY ? s2[lane] : 0.0f;
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
      r1max = nanmax(r1max, __shfl_xor_sync(0xffffffffu, r1max, o));
      r2max = nanmax(r2max, __shfl_xor_sync(0xffffffffu, r2max, o));
    }
    if (lane == 0) {
      // non-negative floats order like their bit patterns; a positive NaN sorts above Inf
      atomicMax(res2 + 0, __float_as_uint(r1max));
      atomicMax(res2 + 1, __float_as_uint(r2max));
    }
  }
}

__global__ void __launch_bounds__(kBX *kBY)
    k_diff(int n1, int n2, int n3, size_t N, int kchunk, const float *__restrict__ x, float w0,
           float w1, float w2, float *__restrict__ g) {
  const int i = blockIdx.x * kBX + threadIdx.x;
  const int j = blockIdx.y * kBY + threadIdx.y;
  if (i >= n1 || j >= n2) return;
  const int k0 = blockIdx.z * kchunk;
  const int k1 = min(n3, k0 + kchunk);
  const size_t P = (size_t)n1 * n2;
  const size_t col = (size_t)i + (size_t)n1 * j;
  const size_t colp1 = (i == n1 - 1) ? col + 1 - n1 : col + 1;
  const size_t colp2 = (j == n2 - 1) ? col - (size_t)n1 * (n2 - 1) : col + n1;
  float xc = x[col + P * k0];
  for (int k = k0; k < k1; ++k) {
    const size_t v = col + P * k;
    const int kp = (k == n3 - 1) ? 0 : k + 1;
    const float x3 = x[col + P * kp];
    g[v] = w0 * (x[colp1 + P * k] - xc);
    g[v + N] = w1 * (x[colp2 + P * k] - xc);
    g[v + 2 * N] = w2 * (x3 - xc);
    xc = x3;
  }
}

__global__ void __launch_bounds__(kBX *kBY)
    k_diff_adjoint(int n1, int n2, int n3, size_t N, int kchunk, const float *__restrict__ g,
                   float w0, float w1, float w2, float *__restrict__ x) {
  const int i = blockIdx.x * kBX + threadIdx.x;
  const int j = blockIdx.y * kBY + threadIdx.y;
  if (i >= n1 || j >= n2) return;
  const int k0 = blockIdx.z * kchunk;
  const int k1 = min(n3, k0 + kchunk);
  const size_t P = (size_t)n1 * n2;
  const size_t col = (size_t)i + (size_t)n1 * j;
  const size_t colm1 = (i == 0) ? col + n1 - 1 : col - 1;
  const size_t colm2 = (j == 0) ? col + (size_t)n1 * (n2 - 1) : col - n1;
  const float *g1 = g, *g2 = g + N, *g3 = g + 2 * N;
  const int km = (k0 == 0) ? n3 - 1 : k0 - 1;
  float g3prev = g3[col + P * km];
  for (int k = k0; k < k1; ++k) {
    const size_t v = col + P * k;
    const float c3 = g3[v];
    x[v] = w0 * (g1[colm1 + P * k] - g1[v]) + w1 * (g2[colm2 + P * k] - g2[v]) + w2 * (g3prev - c3);
    g3prev = c3;
  }
}

__global__ void k_soft(const float *__restrict__ x, size_t n, float thr, float *__restrict__ y) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x)
    y[e] = soft_thr(x[e], thr);
}

}  // namespace

cudaError_t launch_l_tz(const Dims &d, const float *Y, const float *S, const float *Z,
                        const float *G1, const float *G2, const float *F, const float *G3,
                        float mu, const float w[3], float *L, float *T, cudaStream_t st) {
  Chunking c = chunking(d);
  k_l_tz<<<c.grid, dim3(kBX, kBY), 0, st>>>(d.n1, d.n2, d.n3, d.N, c.kchunk, Y, S, Z, G1, G2, F,
                                            G3, mu, w[0], w[1], w[2], L, T);
  return cudaGetLastError();
}

cudaError_t launch_fs_dual(const Dims &d, const float *Y, const float *L, const float *Z,
                           float *S, float *G1, float *G2, float *F, const float *E, float *G3,
                           const float *G4, float mu, float thr_f, float thr_s, const float w[3],
                           unsigned *res2, cudaStream_t st) {
  Chunking c = chunking(d);
  k_fs_dual<<<c.grid, dim3(kBX, kBY), 0, st>>>(d.n1, d.n2, d.n3, d.N, c.kchunk, Y, L, Z, S, G1,
                                               G2, F, E, G3, G4, mu, thr_f, thr_s, w[0], w[1],
                                               w[2], res2);
  return cudaGetLastError();
}

cudaError_t launch_diff(const Dims &d, const float *x, const float w[3], float *g,
                        cudaStream_t st) {
  Chunking c = chunking(d);
  k_diff<<<c.grid, dim3(kBX, kBY), 0, st>>>(d.n1, d.n2, d.n3, d.N, c.kchunk, x, w[0], w[1], w[2],
                                            g);
  return cudaGetLastError();
}

cudaError_t launch_diff_adjoint(const Dims &d, const float *g, const float w[3], float *x,
                                cudaStream_t st) {
  Chunking c = chunking(d);
  k_diff_adjoint<<<c.grid, dim3(kBX, kBY), 0, st>>>(d.n1, d.n2, d.n3, d.N, c.kchunk, g, w[0],
                                                    w[1], w[2], x);
  return cudaGetLastError();
}

cudaError_t launch_soft(const float *x, size_t n, float thr, float *y, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  size_t blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_soft<<<(unsigned)blocks, 256, 0, st>>>(x, n, thr, y);
  return cudaGetLastError();
}

}  // namespace lrstv
