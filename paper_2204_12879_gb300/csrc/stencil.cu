// stencil.cu -- HBM-bound voxel kernels of the LRSTV ADMM iteration
// (arXiv 2204.12879, Section III-C): the fused L-update / T_z assembly, the
// fused F / S / multiplier update, and the standalone difference operators.
//
// Thread mapping: one thread per (i, j) pixel column and a chunk of bands k;
// a warp spans 32 consecutive i (coalesced 128-byte rows).  Walking k inside
// the thread keeps the mode-3 neighbour in a register, so each cube is read
// once; the mode-1 / mode-2 neighbours come from L1 (the same block read
// them).  Chunks of k are sized so the grid fills all SMs several times.
#include <initializer_list>

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

// Group soft threshold of the 3-vector x (the prox of d ||.||_2): the
// isotropic F-update of eq. CRSSTV_iso, one voxel's three gradient entries
// scaled together by max(1 - d / ||x||_2, 0).
__device__ __forceinline__ void group_thr3(float (&x)[3], float d) {
  const float nrm = sqrtf(fmaf(x[0], x[0], fmaf(x[1], x[1], x[2] * x[2])));
  const float g = nrm > d ? 1.0f - d / nrm : 0.0f;
  x[0] *= g;
  x[1] *= g;
  x[2] *= g;
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
    k_l_tz(int n1, int n2, int n3, size_t N, int kchunk, int cchunks,
           const float *__restrict__ Y, const float *__restrict__ S, const float *__restrict__ Z,
           const float *__restrict__ G1, const float *__restrict__ G2,
           const float *__restrict__ F, const float *__restrict__ G3, float mu, float w0,
           float w1, float w2, float *__restrict__ L, float *__restrict__ T) {
  const int i = blockIdx.x * kBX + threadIdx.x;
  const int j = blockIdx.y * kBY + threadIdx.y;
  if (i >= n1 || j >= n2) return;
  // cube of a packed multi-cube launch (cchunks band chunks a cube)
  const size_t cb = blockIdx.z / cchunks;
  Y += cb * N; S += cb * N; Z += cb * N; G1 += cb * N; G2 += cb * N; L += cb * N; T += cb * N;
  F += 3 * cb * N; G3 += 3 * cb * N;
  const int k0 = (blockIdx.z % cchunks) * kchunk;
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

template <int ISO>
__global__ void __launch_bounds__(kBX *kBY)
    k_fs_dual(int n1, int n2, int n3, size_t N, int kchunk, int cchunks,
              const float *__restrict__ Y, const float *__restrict__ L,
              const float *__restrict__ Z, float *__restrict__ S, float *__restrict__ G1,
              float *__restrict__ G2, float *__restrict__ F, const float *__restrict__ E,
              float *__restrict__ G3, const float *__restrict__ G4, float mu, float thr_f,
              float thr_s, float w0, float w1, float w2, unsigned *__restrict__ res2,
              size_t rs) {
  const int i = blockIdx.x * kBX + threadIdx.x;
  const int j = blockIdx.y * kBY + threadIdx.y;
  float r1max = 0.0f, r2max = 0.0f;
  // cube of a packed multi-cube launch (cchunks band chunks a cube); its
  // residual maxima go rs words after the previous cube's
  const size_t cb = blockIdx.z / cchunks;
  Y += cb * N; L += cb * N; Z += cb * N; S += cb * N; G1 += cb * N; G2 += cb * N;
  F += 3 * cb * N; E += 3 * cb * N; G3 += 3 * cb * N; G4 += 3 * cb * N;
  if (res2) res2 += cb * rs;
  if (i < n1 && j < n2) {
    const int k0 = (blockIdx.z % cchunks) * kchunk;
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
      float h3[3], x[3];
#pragma unroll
      for (int n = 0; n < 3; ++n) {
        const size_t vn = v + (size_t)n * N;
        h3[n] = G3[vn];
        const float t1 = g[n] + h3[n] / mu;
        const float t2 = E[vn] + G4[vn] / mu;
        x[n] = 0.5f * (t1 + t2);
      }
      if (ISO) group_thr3(x, thr_f);
#pragma unroll
      for (int n = 0; n < 3; ++n) {
        const size_t vn = v + (size_t)n * N;
        const float f = ISO ? x[n] : soft_thr(x[n], thr_f);
        F[vn] = f;
        G3[vn] = h3[n] + mu * (g[n] - f);
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

// ---------------------------------------------------------------------------
// Vector forms (n1 % 4 == 0, 16-byte aligned cubes): one thread per four
// consecutive voxels along mode 1, no loop, so every load of a thread is
// independent and in flight at once.  The mode-1 neighbours outside the
// float4 are single floats (v - 1 for the adjoint, v + 4 for the forward
// difference); the mode-2 and mode-3 neighbours are whole float4s.
__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }

struct Vox4 {
  size_t v, vm2, vm3, vp2, vp3;  // v and its mode-2 / mode-3 neighbours (backward, forward)
  size_t im1, ip4;               // the single neighbours along mode 1
};

__device__ __forceinline__ bool vox4(int n1, int n2, int n3, size_t q, Vox4 &o) {
  const int n1q = n1 >> 2;
  const size_t P = (size_t)n1 * n2;
  const int iq = (int)(q % n1q);
  const size_t r = q / n1q;
  const int j = (int)(r % n2);
  const int k = (int)(r / n2);
  if (k >= n3) return false;
  const int i = 4 * iq;
  const size_t col = (size_t)n1 * j;
  const size_t plane = P * k;
  o.v = plane + col + i;
  o.vm2 = plane + (j == 0 ? (size_t)n1 * (n2 - 1) : col - n1) + i;
  o.vp2 = plane + (j == n2 - 1 ? 0 : col + n1) + i;
  o.vm3 = (k == 0 ? P * (n3 - 1) : plane - P) + col + i;
  o.vp3 = (k == n3 - 1 ? 0 : plane + P) + col + i;
  o.im1 = plane + col + (i == 0 ? n1 - 1 : i - 1);
  o.ip4 = plane + col + (i + 4 == n1 ? 0 : i + 4);
  return true;
}

__global__ void __launch_bounds__(256)
    k_l_tz4(int n1, int n2, int n3, size_t N, const float *__restrict__ Y,
            const float *__restrict__ S, const float *__restrict__ Z, const float *__restrict__ G1,
            const float *__restrict__ G2, const float *__restrict__ F, const float *__restrict__ G3,
            float mu, float w0, float w1, float w2, float *__restrict__ L, float *__restrict__ T) {
  Vox4 o;
  if (!vox4(n1, n2, n3, blockIdx.x * (size_t)blockDim.x + threadIdx.x, o)) return;
  const size_t cb = blockIdx.y;  // cube of a packed multi-cube launch
  Y += cb * N; S += cb * N; Z += cb * N; G1 += cb * N; G2 += cb * N; L += cb * N; T += cb * N;
  F += 3 * cb * N; G3 += 3 * cb * N;
  const float *F1 = F, *F2 = F + N, *F3 = F + 2 * N;
  const float *H1 = G3, *H2 = G3 + N, *H3 = G3 + 2 * N;
  const float4 y = ld4(Y + o.v), s = ld4(S + o.v), z = ld4(Z + o.v), g1 = ld4(G1 + o.v),
               g2 = ld4(G2 + o.v);
  const float4 f1 = ld4(F1 + o.v), h1 = ld4(H1 + o.v), f2 = ld4(F2 + o.v), h2 = ld4(H2 + o.v),
               f3 = ld4(F3 + o.v), h3 = ld4(H3 + o.v);
  const float4 f2m = ld4(F2 + o.vm2), h2m = ld4(H2 + o.vm2), f3m = ld4(F3 + o.vm3),
               h3m = ld4(H3 + o.vm3);
  const float f1m = F1[o.im1], h1m = H1[o.im1];
  // q_n = mu F_n - Gamma3_n; D_n^T q(v) = q(v - e_n) - q(v)
  const float q1[5] = {mu * f1m - h1m, mu * f1.x - h1.x, mu * f1.y - h1.y, mu * f1.z - h1.z,
                       mu * f1.w - h1.w};
  const float yy[4] = {y.x, y.y, y.z, y.w}, ss[4] = {s.x, s.y, s.z, s.w},
              zz[4] = {z.x, z.y, z.z, z.w}, a1[4] = {g1.x, g1.y, g1.z, g1.w},
              a2[4] = {g2.x, g2.y, g2.z, g2.w};
  const float F2c[4] = {f2.x, f2.y, f2.z, f2.w}, H2c[4] = {h2.x, h2.y, h2.z, h2.w},
              F2m[4] = {f2m.x, f2m.y, f2m.z, f2m.w}, H2m[4] = {h2m.x, h2m.y, h2m.z, h2m.w},
              F3c[4] = {f3.x, f3.y, f3.z, f3.w}, H3c[4] = {h3.x, h3.y, h3.z, h3.w},
              F3m[4] = {f3m.x, f3m.y, f3m.z, f3m.w}, H3m[4] = {h3m.x, h3m.y, h3m.z, h3m.w};
  float lo[4], to[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float q2 = mu * F2c[e] - H2c[e], q2m = mu * F2m[e] - H2m[e];
    const float q3 = mu * F3c[e] - H3c[e], q3m = mu * F3m[e] - H3m[e];
    const float adj = w0 * (q1[e] - q1[e + 1]) + w1 * (q2m - q2) + w2 * (q3m - q3);
    const float l = 0.5f * (yy[e] - ss[e] + zz[e] + (a1[e] - a2[e]) / mu);
    lo[e] = l;
    to[e] = mu * l + a2[e] + adj;
  }
  st4(L + o.v, make_float4(lo[0], lo[1], lo[2], lo[3]));
  st4(T + o.v, make_float4(to[0], to[1], to[2], to[3]));
}

template <int ISO>
__global__ void __launch_bounds__(256)
    k_fs_dual4(int n1, int n2, int n3, size_t N, const float *__restrict__ Y,
               const float *__restrict__ L, const float *__restrict__ Z, float *__restrict__ S,
               float *__restrict__ G1, float *__restrict__ G2, float *__restrict__ F,
               const float *__restrict__ E, float *__restrict__ G3, const float *__restrict__ G4,
               float mu, float thr_f, float thr_s, float w0, float w1, float w2,
               unsigned *__restrict__ res2, size_t rs) {
  float r1max = 0.0f, r2max = 0.0f;
  // cube of a packed multi-cube launch; its residual maxima go rs words after
  // the previous cube's
  const size_t cb = blockIdx.y;
  Y += cb * N; L += cb * N; Z += cb * N; S += cb * N; G1 += cb * N; G2 += cb * N;
  F += 3 * cb * N; E += 3 * cb * N; G3 += 3 * cb * N; G4 += 3 * cb * N;
  if (res2) res2 += cb * rs;
  Vox4 o;
  if (vox4(n1, n2, n3, blockIdx.x * (size_t)blockDim.x + threadIdx.x, o)) {
    const float4 z = ld4(Z + o.v), zp2 = ld4(Z + o.vp2), zp3 = ld4(Z + o.vp3);
    const float zp1 = Z[o.ip4];
    const float zc[4] = {z.x, z.y, z.z, z.w};
    const float z1[4] = {z.y, z.z, z.w, zp1};  // z(v + e1)
    const float z2[4] = {zp2.x, zp2.y, zp2.z, zp2.w}, z3[4] = {zp3.x, zp3.y, zp3.z, zp3.w};
    float g[3][4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      g[0][e] = w0 * (z1[e] - zc[e]);
      g[1][e] = w1 * (z2[e] - zc[e]);
      g[2][e] = w2 * (z3[e] - zc[e]);
    }
    float x[3][4], H[3][4];
#pragma unroll
    for (int n = 0; n < 3; ++n) {
      const size_t vn = o.v + (size_t)n * N;
      const float4 h3 = ld4(G3 + vn), ev = ld4(E + vn), h4 = ld4(G4 + vn);
      const float EE[4] = {ev.x, ev.y, ev.z, ev.w}, H4[4] = {h4.x, h4.y, h4.z, h4.w};
      H[n][0] = h3.x; H[n][1] = h3.y; H[n][2] = h3.z; H[n][3] = h3.w;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float t1 = g[n][e] + H[n][e] / mu;
        const float t2 = EE[e] + H4[e] / mu;
        x[n][e] = 0.5f * (t1 + t2);
      }
    }
    if (ISO) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        float xv[3] = {x[0][e], x[1][e], x[2][e]};
        group_thr3(xv, thr_f);
        x[0][e] = xv[0]; x[1][e] = xv[1]; x[2][e] = xv[2];
      }
    }
#pragma unroll
    for (int n = 0; n < 3; ++n) {
      const size_t vn = o.v + (size_t)n * N;
      float fo[4], ho[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float f = ISO ? x[n][e] : soft_thr(x[n][e], thr_f);
        fo[e] = f;
        ho[e] = H[n][e] + mu * (g[n][e] - f);
      }
      st4(F + vn, make_float4(fo[0], fo[1], fo[2], fo[3]));
      st4(G3 + vn, make_float4(ho[0], ho[1], ho[2], ho[3]));
    }
    const float4 y4 = ld4(Y + o.v), l4 = ld4(L + o.v), a4 = ld4(G1 + o.v), b4 = ld4(G2 + o.v);
    const float yy[4] = {y4.x, y4.y, y4.z, y4.w}, ll[4] = {l4.x, l4.y, l4.z, l4.w},
                a1[4] = {a4.x, a4.y, a4.z, a4.w}, a2[4] = {b4.x, b4.y, b4.z, b4.w};
    float so[4], g1o[4], g2o[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float sv = soft_thr(yy[e] - ll[e] + a1[e] / mu, thr_s);
      so[e] = sv;
      const float r1 = yy[e] - ll[e] - sv;
      const float r2 = ll[e] - zc[e];
      g1o[e] = a1[e] + mu * r1;
      g2o[e] = a2[e] + mu * r2;
      r1max = nanmax(r1max, fabsf(r1));
      r2max = nanmax(r2max, fabsf(r2));
    }
    st4(S + o.v, make_float4(so[0], so[1], so[2], so[3]));
    st4(G1 + o.v, make_float4(g1o[0], g1o[1], g1o[2], g1o[3]));
    st4(G2 + o.v, make_float4(g2o[0], g2o[1], g2o[2], g2o[3]));
  }
  if (res2 == nullptr) return;
#pragma unroll
  for (int o2 = 16; o2 > 0; o2 >>= 1) {
    r1max = nanmax(r1max, __shfl_xor_sync(0xffffffffu, r1max, o2));
    r2max = nanmax(r2max, __shfl_xor_sync(0xffffffffu, r2max, o2));
  }
  __shared__ float s1[8], s2[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { s1[wid] = r1max; s2[wid] = r2max; }
  __syncthreads();
  if (wid == 0) {
    r1max = lane < 8 ? s1[lane] : 0.0f;
    r2max = lane < 8 ? s2[lane] : 0.0f;
#pragma unroll
    for (int o2 = 4; o2 > 0; o2 >>= 1) {
      r1max = nanmax(r1max, __shfl_xor_sync(0xffffffffu, r1max, o2));
      r2max = nanmax(r2max, __shfl_xor_sync(0xffffffffu, r2max, o2));
    }
    if (lane == 0) {
      atomicMax(res2 + 0, __float_as_uint(r1max));
      atomicMax(res2 + 1, __float_as_uint(r2max));
    }
  }
}

bool vec4_ok(const Dims &d, std::initializer_list<const void *> ptrs) {
  if (d.n1 % 4 != 0) return false;
  for (const void *p : ptrs)
    if (((uintptr_t)p & 15u) != 0) return false;
  return true;
}

unsigned vec4_blocks(const Dims &d) { return (unsigned)((d.N / 4 + 255) / 256); }

}  // namespace

// The chunked (scalar) form takes nb cubes in one launch while nb times its
// band chunks fit the grid's z extent; beyond that one launch per cube.
constexpr int kMaxGridZ = 65535;

cudaError_t launch_l_tz(const Dims &d, const float *Y, const float *S, const float *Z,
                        const float *G1, const float *G2, const float *F, const float *G3,
                        float mu, const float w[3], float *L, float *T, cudaStream_t st, int nb) {
  if (nb < 1 || nb > kMaxGridZ) return cudaErrorInvalidValue;
  if (vec4_ok(d, {Y, S, Z, G1, G2, F, G3, L, T})) {
    k_l_tz4<<<dim3(vec4_blocks(d), nb), 256, 0, st>>>(d.n1, d.n2, d.n3, d.N, Y, S, Z, G1, G2, F,
                                                       G3, mu, w[0], w[1], w[2], L, T);
    return cudaGetLastError();
  }
  Chunking c = chunking(d);
  const int chunks = (int)c.grid.z;
  const int per = (long long)nb * chunks <= kMaxGridZ ? nb : 1;
  for (int b0 = 0; b0 < nb; b0 += per) {
    const size_t o = (size_t)b0 * d.N;
    c.grid.z = per * chunks;
    k_l_tz<<<c.grid, dim3(kBX, kBY), 0, st>>>(d.n1, d.n2, d.n3, d.N, c.kchunk, chunks, Y + o,
                                              S + o, Z + o, G1 + o, G2 + o, F + 3 * o,
                                              G3 + 3 * o, mu, w[0], w[1], w[2], L + o, T + o);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_fs_dual(const Dims &d, const float *Y, const float *L, const float *Z,
                           float *S, float *G1, float *G2, float *F, const float *E, float *G3,
                           const float *G4, float mu, float thr_f, float thr_s, const float w[3],
                           unsigned *res2, cudaStream_t st, int iso, int nb, size_t rs) {
  if (nb < 1 || nb > kMaxGridZ) return cudaErrorInvalidValue;
  if (vec4_ok(d, {Y, L, Z, S, G1, G2, F, E, G3, G4})) {
    auto k = iso ? k_fs_dual4<1> : k_fs_dual4<0>;
    k<<<dim3(vec4_blocks(d), nb), 256, 0, st>>>(d.n1, d.n2, d.n3, d.N, Y, L, Z, S, G1, G2, F, E,
                                                G3, G4, mu, thr_f, thr_s, w[0], w[1], w[2], res2,
                                                rs);
    return cudaGetLastError();
  }
  Chunking c = chunking(d);
  const int chunks = (int)c.grid.z;
  const int per = (long long)nb * chunks <= kMaxGridZ ? nb : 1;
  auto k = iso ? k_fs_dual<1> : k_fs_dual<0>;
  for (int b0 = 0; b0 < nb; b0 += per) {
    const size_t o = (size_t)b0 * d.N;
    c.grid.z = per * chunks;
    k<<<c.grid, dim3(kBX, kBY), 0, st>>>(d.n1, d.n2, d.n3, d.N, c.kchunk, chunks, Y + o, L + o,
                                         Z + o, S + o, G1 + o, G2 + o, F + 3 * o, E + 3 * o,
                                         G3 + 3 * o, G4 + 3 * o, mu, thr_f, thr_s, w[0], w[1],
                                         w[2], res2 ? res2 + (size_t)b0 * rs : nullptr, rs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
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
