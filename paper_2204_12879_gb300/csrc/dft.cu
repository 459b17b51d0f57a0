// dft.cu -- discrete Fourier transforms of the LRSTV iteration
// (arXiv 2204.12879, eq. Z_solution and eq. E_solution):
//  - mode-3 (spectral) real <-> half-complex DFTs, with the t-SVT prologue
//    (F - Gamma4/mu) and epilogue (E, Gamma4 update) fused in;
//  - a batched complex GEMM that applies the spatial DFT matrices of modes 1
//    and 2 (and the SVT reconstruction W V^H), with the Z-solve's spectral
//    division fused into its epilogue.
// Non-power-of-two lengths (31, 80, 145, 191, 200, 220 ...) are handled by
// direct sums: every transform is a dense product with a table of twiddles
// built in FP64 (sincospi) and rounded once to FP32.
#include "lrstv_internal.cuh"

namespace lrstv {

namespace {

// ------------------------------------------------------------------ tables
__global__ void k_dft_matrix(int n, float2 *__restrict__ F, float2 *__restrict__ G) {
  const size_t total = (size_t)n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t a = e % n, t = e / n;
    const size_t m = (a * t) % (size_t)n;
    double s, c;
    sincospi(2.0 * (double)m / (double)n, &s, &c);
    F[e] = make_float2((float)c, (float)-s);  // exp(-2 pi i a t / n)
    G[e] = make_float2((float)c, (float)s);   // exp(+2 pi i a t / n)
  }
}

__global__ void k_tw3(int n3, float2 *__restrict__ tw) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n3; m += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)m / (double)n3, &s, &c);
    tw[m] = make_float2((float)c, (float)-s);
  }
}

// lam[a] = w^2 |exp(2 pi i a / n) - 1|^2 = w^2 4 sin^2(pi a / n): the DFT
// eigenvalues of w^2 D^T D for a circular forward difference of length n.
__global__ void k_lam(int n, double w, float *__restrict__ lam) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x) {
    const double s = sinpi((double)a / (double)n);
    lam[a] = (float)(w * w * 4.0 * s * s);
  }
}

// --------------------------------------------------------- mode-3 DFTs
// One thread per pixel and kKF frequencies (r2c) or bands (c2r).  The block
// stages the twiddles of its kKF frequencies for a chunk of kCB bands (or
// the reverse) in shared memory, so the inner loop is a broadcast 16-byte
// read of two twiddles and four FMAs; every sum runs over bands (or
// frequencies) in increasing order.  The inputs of the next four bands (or
// frequencies) are loaded while the current four's products run.  The
// blocks of one pixel tile's frequency (or band) groups are adjacent in
// launch order (blockIdx.x = tile * groups + group), so the tile's inputs,
// which every group reads, come from DRAM once and from L2 after that.
constexpr int kPix = 128;  // pixels per block
constexpr int kKF = 48;    // frequencies (or bands) per thread
constexpr int kCB = 64;    // bands (or frequencies) per staged chunk
static_assert(kCB % 4 == 0, "the four-deep loads step across chunks");

// X_k(p) = sum_c (x(p, c) - ycoef y(p, c)) exp(-2 pi i k c / n3), k < h; the
// y term is present when kY.
template <bool kY>
__global__ void __launch_bounds__(kPix, 4)
    k_r2c3(int n1, int n2, int n3, int h, size_t N, size_t P, const float *__restrict__ x,
           const float *__restrict__ y, float ycoef, float2 *__restrict__ out, int trans,
           const float2 *__restrict__ tw3) {
  __shared__ float4 s_t[kCB][kKF / 2];  // s_t[c][f/2] = twiddles of frequencies f, f + 1
  const int groups = (h + kKF - 1) / kKF;
  const size_t p = (blockIdx.x / groups) * (size_t)kPix + threadIdx.x;
  const bool live = p < P;
  const int kbase = (blockIdx.x % groups) * kKF;
  const int b = blockIdx.z;
  const float *xb = x + (size_t)b * N;
  const float *yb = kY ? y + (size_t)b * N : nullptr;
  float2 acc[kKF];
#pragma unroll
  for (int f = 0; f < kKF; ++f) acc[f] = make_float2(0.f, 0.f);
  // the inputs of bands c .. c + 3 (zero past n3), combined only when they
  // are used, so that no thread waits for its loads where it issues them
  float nx[4], ny[4];
  auto load4 = [&](int c) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const bool in = c + u < n3;
      nx[u] = in ? xb[p + P * (c + u)] : 0.0f;
      if (kY) ny[u] = in ? yb[p + P * (c + u)] : 0.0f;
    }
  };
  if (live) load4(0);
  for (int c0 = 0; c0 < n3; c0 += kCB) {
    const int cn = min(kCB, n3 - c0);
    __syncthreads();
    float2 *st = reinterpret_cast<float2 *>(&s_t[0][0]);
    for (int e = threadIdx.x; e < cn * kKF; e += blockDim.x) {
      const int cc = e / kKF, f = e % kKF;
      const unsigned m = ((unsigned)(kbase + f) * (unsigned)(c0 + cc)) % (unsigned)n3;  // k c < 2^24
      st[cc * kKF + f] = tw3[m];
    }
    __syncthreads();
    if (live) {
      // kCB is a multiple of 4, so the next four bands start the next
      // chunk when this one ends
      for (int cc = 0; cc < cn; cc += 4) {
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = kY ? nx[u] - ycoef * ny[u] : nx[u];
        load4(c0 + cc + 4);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (cc + u >= cn) break;
#pragma unroll
          for (int f2 = 0; f2 < kKF / 2; ++f2) {
            const float4 t = s_t[cc + u][f2];
            acc[2 * f2].x = fmaf(v[u], t.x, acc[2 * f2].x);
            acc[2 * f2].y = fmaf(v[u], t.y, acc[2 * f2].y);
            acc[2 * f2 + 1].x = fmaf(v[u], t.z, acc[2 * f2 + 1].x);
            acc[2 * f2 + 1].y = fmaf(v[u], t.w, acc[2 * f2 + 1].y);
          }
        }
      }
    }
  }
  if (!live) return;
  size_t pos = p;
  if (trans) {
    const size_t i = p % n1, j = p / n1;
    pos = j + (size_t)n2 * i;
  }
  float2 *ob = out + (size_t)b * h * P;
#pragma unroll
  for (int f = 0; f < kKF; ++f) {
    const int k = kbase + f;
    if (k < h) ob[(size_t)k * P + pos] = trans ? make_float2(acc[f].x, -acc[f].y) : acc[f];
  }
}

// x(p, c) = (1/n3) [X_0 + 2 sum_{0<k<n3/2} Re(X_k e^{2 pi i k c/n3}) + X_{n3/2} (-1)^c],
// the Nyquist term present for even n3 only.
__global__ void __launch_bounds__(kPix, 5)
    k_c2r3(int n1, int n2, int n3, int h, size_t N, size_t P, const float2 *__restrict__ spec,
           int trans, const float2 *__restrict__ tw3, float *__restrict__ out, int mode,
           float *__restrict__ G4, const float *__restrict__ F, float mu, int gamma4) {
  __shared__ float4 s_t[kCB][kKF / 2];  // s_t[k][c/2] = twiddles of bands c, c + 1
  const int groups = (n3 + kKF - 1) / kKF;
  const size_t p = (blockIdx.x / groups) * (size_t)kPix + threadIdx.x;
  const bool live = p < P;
  const int cbase = (blockIdx.x % groups) * kKF;
  const int b = blockIdx.z;
  size_t pos = p;
  if (trans) {
    const size_t i = p % n1, j = p / n1;
    pos = j + (size_t)n2 * i;
  }
  const float2 *sb = spec + (size_t)b * h * P + pos;
  float acc[kKF];
#pragma unroll
  for (int f = 0; f < kKF; ++f) acc[f] = 0.f;
  // the coefficients of frequencies k .. k + 3 (zero past h)
  float2 nX[4];
  auto load4 = [&](int k) {
#pragma unroll
    for (int u = 0; u < 4; ++u) nX[u] = k + u < h ? sb[(size_t)(k + u) * P] : make_float2(0.f, 0.f);
  };
  if (live) load4(0);
  for (int k0 = 0; k0 < h; k0 += kCB) {
    const int kn = min(kCB, h - k0);
    __syncthreads();
    float2 *st = reinterpret_cast<float2 *>(&s_t[0][0]);
    for (int e = threadIdx.x; e < kn * kKF; e += blockDim.x) {
      const int kk = e / kKF, f = e % kKF;
      const unsigned m = ((unsigned)(k0 + kk) * (unsigned)(cbase + f)) % (unsigned)n3;  // k c < 2^24
      st[kk * kKF + f] = tw3[m];  // (cos, -sin) of 2 pi k c / n3
    }
    __syncthreads();
    if (live) {
      // kCB is a multiple of 4, so the next four frequencies start the next
      // chunk when this one ends
      for (int kk = 0; kk < kn; kk += 4) {
        float2 Xs[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) Xs[u] = nX[u];
        load4(k0 + kk + 4);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (kk + u >= kn) break;
          const int k = k0 + kk + u;
          float2 X = Xs[u];
          if (trans) X.y = -X.y;
          const float wk = (k == 0 || 2 * k == n3) ? 1.0f : 2.0f;
          X.x *= wk;
          X.y *= wk;
#pragma unroll
          for (int f2 = 0; f2 < kKF / 2; ++f2) {
            const float4 t = s_t[kk + u][f2];
            acc[2 * f2] = fmaf(X.x, t.x, acc[2 * f2]);
            acc[2 * f2] = fmaf(X.y, t.y, acc[2 * f2]);
            acc[2 * f2 + 1] = fmaf(X.x, t.z, acc[2 * f2 + 1]);
            acc[2 * f2 + 1] = fmaf(X.y, t.w, acc[2 * f2 + 1]);
          }
        }
      }
    }
  }
  if (!live) return;
  const float inv = 1.0f / (float)n3;
  float *ob = out + (size_t)b * N;
#pragma unroll
  for (int f = 0; f < kKF; ++f) {
    const int c = cbase + f;
    if (c >= n3) break;
    const size_t v = p + P * c;
    const float r = acc[f] * inv;
    ob[v] = r;
    if (mode == 1 && gamma4) {
      const size_t vb = (size_t)b * N + v;
      G4[vb] = G4[vb] + mu * (r - F[vb]);
    }
  }
}

// ------------------------------------------------------------- complex GEMM
constexpr int BM = 64, BN = 64, BK = 16, GT = 256;

template <int OPA, int OPB, int EPI>
__global__ void __launch_bounds__(GT) k_cgemm(CGemm g) {
  __shared__ float2 As[BK][BM];
  __shared__ float2 Bs[BK][BN];
  const int b = blockIdx.z;
  const float2 *A = g.A + (size_t)b * g.sA;
  const float2 *B = g.B + (size_t)b * g.sB;
  float2 *C = g.C + (size_t)b * g.sC;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  float2 acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int s = 0; s < 4; ++s) acc[r][s] = make_float2(0.f, 0.f);

  for (int k0 = 0; k0 < g.K; k0 += BK) {
#pragma unroll
    for (int r = 0; r < (BM * BK) / GT; ++r) {
      const int e = tid + GT * r;
      if (OPA == 0) {
        const int m = e % BM, k = e / BM;
        const int gm = m0 + m, gk = k0 + k;
        As[k][m] = (gm < g.M && gk < g.K) ? A[gm + (size_t)g.lda * gk] : make_float2(0.f, 0.f);
      } else {
        // op(A)(m, k) = conj(A(k, m)), A stored K x M column-major
        const int k = e % BK, m = e / BK;
        const int gm = m0 + m, gk = k0 + k;
        float2 v = (gm < g.M && gk < g.K) ? A[gk + (size_t)g.lda * gm] : make_float2(0.f, 0.f);
        v.y = -v.y;
        As[k][m] = v;
      }
    }
#pragma unroll
    for (int r = 0; r < (BK * BN) / GT; ++r) {
      const int e = tid + GT * r;
      if (OPB == 0) {
        const int k = e % BK, n = e / BK;
        const int gk = k0 + k, gn = n0 + n;
        Bs[k][n] = (gk < g.K && gn < g.N) ? B[gk + (size_t)g.ldb * gn] : make_float2(0.f, 0.f);
      } else {
        // op(B)(k, n) = conj(B(n, k)), B stored N x K column-major
        const int n = e % BN, k = e / BN;
        const int gk = k0 + k, gn = n0 + n;
        float2 v = (gk < g.K && gn < g.N) ? B[gn + (size_t)g.ldb * gk] : make_float2(0.f, 0.f);
        v.y = -v.y;
        Bs[k][n] = v;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float2 a[4], bb[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][tx + 16 * r];
#pragma unroll
      for (int s = 0; s < 4; ++s) bb[s] = Bs[kk][ty + 16 * s];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          acc[r][s].x = fmaf(a[r].x, bb[s].x, acc[r][s].x);
          acc[r][s].x = fmaf(-a[r].y, bb[s].y, acc[r][s].x);
          acc[r][s].y = fmaf(a[r].x, bb[s].y, acc[r][s].y);
          acc[r][s].y = fmaf(a[r].y, bb[s].x, acc[r][s].y);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int m = m0 + tx + 16 * r;
    if (m >= g.M) continue;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int n = n0 + ty + 16 * s;
      if (n >= g.N) continue;
      float2 v = acc[r][s];
      if (EPI == 1) {
        const int lb = g.lam3_period > 0 ? b % g.lam3_period : b;
        const float den = g.mu * (1.0f + g.lam1[m] + g.lam2[n] + g.lam3[lb]);
        const float q = g.scale / den;
        v.x *= q;
        v.y *= q;
      }
      if (EPI == 2) {
        const float2 c = C[m + (size_t)g.ldc * n];
        v.x += c.x;
        v.y += c.y;
      }
      C[m + (size_t)g.ldc * n] = v;
    }
  }
}

}  // namespace

cudaError_t launch_tw3(int n3, float2 *tw3, cudaStream_t st) {
  k_tw3<<<(n3 + 255) / 256, 256, 0, st>>>(n3, tw3);
  return cudaGetLastError();
}

cudaError_t launch_tables(const Dims &d, const float w[3], float2 *tw3, float2 *F1, float2 *G1,
                          float2 *F2, float2 *G2, float *lam1, float *lam2, float *lam3,
                          cudaStream_t st) {
  cudaError_t e = launch_tw3(d.n3, tw3, st);
  if (e != cudaSuccess) return e;
  auto blocks = [](size_t n) { return (unsigned)((n + 255) / 256 > 1024 ? 1024 : (n + 255) / 256); };
  k_dft_matrix<<<blocks((size_t)d.n1 * d.n1), 256, 0, st>>>(d.n1, F1, G1);
  k_dft_matrix<<<blocks((size_t)d.n2 * d.n2), 256, 0, st>>>(d.n2, F2, G2);
  k_lam<<<blocks(d.n1), 256, 0, st>>>(d.n1, (double)w[0], lam1);
  k_lam<<<blocks(d.n2), 256, 0, st>>>(d.n2, (double)w[1], lam2);
  k_lam<<<blocks(d.n3), 256, 0, st>>>(d.n3, (double)w[2], lam3);
  return cudaGetLastError();
}

cudaError_t launch_r2c3(const Dims &d, int nb, const float *x, const float *y, float ycoef,
                        float2 *out, int work_orient, const float2 *tw3, cudaStream_t st,
                        GemmSel gs) {
  if (gs.tc && gs.dft) {
    Dft3 f{};
    f.x = x;
    f.y = y;
    f.ycoef = ycoef;
    f.spec_out = out;
    f.tw3 = tw3;
    f.n1 = d.n1;
    f.n2 = d.n2;
    f.n3 = d.n3;
    f.h = d.h;
    f.trans = work_orient && d.trans;
    f.P = d.P;
    f.N = d.N;
    return launch_dft3_tc(1, f, nb, gs.err, st, gs.prec);
  }
  const size_t tiles = (d.P + kPix - 1) / kPix, groups = (d.h + kKF - 1) / kKF;
  dim3 grid((unsigned)(tiles * groups), 1, nb);
  if (y)
    k_r2c3<true><<<grid, kPix, 0, st>>>(d.n1, d.n2, d.n3, d.h, d.N, d.P, x, y, ycoef, out,
                                        work_orient && d.trans, tw3);
  else
    k_r2c3<false><<<grid, kPix, 0, st>>>(d.n1, d.n2, d.n3, d.h, d.N, d.P, x, y, ycoef, out,
                                         work_orient && d.trans, tw3);
  return cudaGetLastError();
}

cudaError_t launch_c2r3(const Dims &d, int nb, const float2 *spec, int work_orient,
                        const float2 *tw3, float *out, int mode, float *G4, const float *F,
                        float mu, int gamma4, cudaStream_t st, GemmSel gs) {
  if (gs.tc && gs.dft) {
    Dft3 f{};
    f.spec = spec;
    f.out = out;
    f.G4 = G4;
    f.F = F;
    f.mu = mu;
    f.mode = mode;
    f.gamma4 = gamma4;
    f.tw3 = tw3;
    f.n1 = d.n1;
    f.n2 = d.n2;
    f.n3 = d.n3;
    f.h = d.h;
    f.trans = work_orient && d.trans;
    f.P = d.P;
    f.N = d.N;
    return launch_dft3_tc(2, f, nb, gs.err, st, gs.prec);
  }
  const size_t tiles = (d.P + kPix - 1) / kPix, groups = (d.n3 + kKF - 1) / kKF;
  dim3 grid((unsigned)(tiles * groups), 1, nb);
  k_c2r3<<<grid, kPix, 0, st>>>(d.n1, d.n2, d.n3, d.h, d.N, d.P, spec, work_orient && d.trans,
                                tw3, out, mode, G4, F, mu, gamma4);
  return cudaGetLastError();
}

cudaError_t launch_cgemm(const CGemm &g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  dim3 grid((g.M + BM - 1) / BM, (g.N + BN - 1) / BN, g.batch);
  if (g.opA == 0 && g.opB == 0 && g.epi == 0) k_cgemm<0, 0, 0><<<grid, GT, 0, st>>>(g);
  else if (g.opA == 0 && g.opB == 0 && g.epi == 1) k_cgemm<0, 0, 1><<<grid, GT, 0, st>>>(g);
  else if (g.opA == 0 && g.opB == 1 && g.epi == 0) k_cgemm<0, 1, 0><<<grid, GT, 0, st>>>(g);
  else if (g.opA == 1 && g.opB == 0 && g.epi == 0) k_cgemm<1, 0, 0><<<grid, GT, 0, st>>>(g);
  else if (g.opA == 0 && g.opB == 0 && g.epi == 2) k_cgemm<0, 0, 2><<<grid, GT, 0, st>>>(g);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace lrstv
