// tucker.cu -- the L-update of the full TDLRSTV model (Section III-C, step 1,
// eq. X_solution with the Tucker-3 model of eq. LRTAmodel): the target
// X = 1/2 (Y - S + Z + (Gamma1 - Gamma2)/mu) is replaced by its Tucker
// projection X x1 U1 U1^T x2 U2 U2^T x3 U3 U3^T, the factors coming from one
// HOOI sweep per ADMM iteration (U1, U2, U3 in turn, each the r_n leading
// eigenvectors of the mode-n Gram matrix of X multiplied by the other
// factors' transposes), started from the previous iteration's factors or, in
// the first iteration, from the truncated HOSVD of X.
//
// Every mode product is one (batched) real GEMM on an FP32 SIMT kernel with
// FP64 accumulation across K tiles (the cube's column-major layout makes each
// unfolding or each frontal slice a strided matrix); each Gram matrix (n_n x n_n, at most 512) is diagonalised
// by the one-sided Jacobi kernel of the t-SVT (svt.cu): the right singular
// vectors of a symmetric positive semi-definite matrix are its eigenvectors
// and its column norms after the sweeps are the eigenvalues.
#include <float.h>
#include <stdint.h>

#include "lrstv_internal.cuh"

namespace lrstv {

namespace {

unsigned grid_for(size_t n) {
  size_t b = (n + 255) / 256;
  return (unsigned)(b < 1 ? 1 : (b > 152ull * 16 ? 152ull * 16 : b));
}

// ------------------------------------------------------------ real GEMM
// C_b (M x N) = op(A_b) op(B_b) (+ C_b when ACC), column-major, op = N or T.
// With kc > 0 the batch index is a K chunk instead: batch b takes the
// products k in [b kc, min(K, (b + 1) kc)) (sA, sB: the element offsets of
// one chunk) and writes its partial sum to C + b sC.
struct SGemm {
  const float *A; long long sA; int lda;
  const float *B; long long sB; int ldb;
  float *C; long long sC; int ldc;
  int M, N, K, batch;
  int kc;
};

constexpr int SBM = 64, SBN = 64, SBK = 16, SGT = 256;

template <int TA, int TB, int ACC>
__global__ void __launch_bounds__(SGT) k_sgemm(SGemm g) {
  __shared__ float As[SBK][SBM + 1];
  __shared__ float Bs[SBK][SBN + 1];
  const int b = blockIdx.z;
  const float *A = g.A + (size_t)b * g.sA;
  const float *B = g.B + (size_t)b * g.sB;
  float *C = g.C + (size_t)b * g.sC;
  const int m0 = blockIdx.x * SBM, n0 = blockIdx.y * SBN;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int K = g.kc > 0 ? min(g.kc, g.K - b * g.kc) : g.K;
  // each K tile of 16 products is summed in FP32, the tiles in FP64: the Gram
  // matrices sum thousands of same-signed terms, and their leading eigenvalue
  // (the cube's mean) would otherwise bury the smaller kept ones in rounding
  double accd[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int s = 0; s < 4; ++s) accd[r][s] = 0.0;
  for (int k0 = 0; k0 < K; k0 += SBK) {
    float acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int s = 0; s < 4; ++s) acc[r][s] = 0.f;
#pragma unroll
    for (int r = 0; r < (SBM * SBK) / SGT; ++r) {
      const int e = tid + SGT * r;
      int m, k;
      if (TA == 0) {  // A(m, k) at m + lda k: consecutive threads along m
        m = e % SBM;
        k = e / SBM;
      } else {        // op(A)(m, k) = A(k, m) at k + lda m: along k
        k = e % SBK;
        m = e / SBK;
      }
      const int gm = m0 + m, gk = k0 + k;
      float v = 0.f;
      if (gm < g.M && gk < K) v = TA == 0 ? A[gm + (size_t)g.lda * gk] : A[gk + (size_t)g.lda * gm];
      As[k][m] = v;
    }
#pragma unroll
    for (int r = 0; r < (SBK * SBN) / SGT; ++r) {
      const int e = tid + SGT * r;
      int n, k;
      if (TB == 0) {  // B(k, n) at k + ldb n: along k
        k = e % SBK;
        n = e / SBK;
      } else {        // op(B)(k, n) = B(n, k) at n + ldb k: along n
        n = e % SBN;
        k = e / SBN;
      }
      const int gn = n0 + n, gk = k0 + k;
      float v = 0.f;
      if (gn < g.N && gk < K) v = TB == 0 ? B[gk + (size_t)g.ldb * gn] : B[gn + (size_t)g.ldb * gk];
      Bs[k][n] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < SBK; ++kk) {
      float a[4], bb[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][tx + 16 * r];
#pragma unroll
      for (int s = 0; s < 4; ++s) bb[s] = Bs[kk][ty + 16 * s];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int s = 0; s < 4; ++s) acc[r][s] = fmaf(a[r], bb[s], acc[r][s]);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int s = 0; s < 4; ++s) accd[r][s] += (double)acc[r][s];
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
      float *c = C + m + (size_t)g.ldc * n;
      *c = ACC ? (float)((double)*c + accd[r][s]) : (float)accd[r][s];
    }
  }
}

cudaError_t sgemm(const SGemm &g, int ta, int tb, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  dim3 grid((g.M + SBM - 1) / SBM, (g.N + SBN - 1) / SBN, g.batch);
  if (ta == 0 && tb == 0) k_sgemm<0, 0, 0><<<grid, SGT, 0, st>>>(g);
  else if (ta == 0 && tb == 1) k_sgemm<0, 1, 0><<<grid, SGT, 0, st>>>(g);
  else if (ta == 1 && tb == 0) k_sgemm<1, 0, 0><<<grid, SGT, 0, st>>>(g);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

SGemm mk(const float *A, long long sA, int lda, const float *B, long long sB, int ldb, float *C,
         long long sC, int ldc, int M, int N, int K, int batch) {
  SGemm g;
  g.A = A; g.sA = sA; g.lda = lda;
  g.B = B; g.sB = sB; g.ldb = ldb;
  g.C = C; g.sC = sC; g.ldc = ldc;
  g.M = M; g.N = N; g.K = K; g.batch = batch;
  g.kc = 0;
  return g;
}

// C[m + ldc n] = sum over b of P[b M N + m + M n], in order, in FP64.
__global__ void k_sum_partials(int M, int N, int nb, const float *__restrict__ P, float *__restrict__ C,
                               int ldc) {
  const size_t MN = (size_t)M * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < MN;
       e += (size_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int b = 0; b < nb; ++b) acc += (double)P[(size_t)b * MN + e];
    C[(e % M) + (size_t)ldc * (e / M)] = (float)acc;
  }
}

// A product with few output tiles and a long K (the Gram matrices: n x n
// from K up to n1 n2) split along K so that the grid covers the GPU: chunks
// of at least 512 products, about two CTAs per SM in all, partial sums in
// `scratch` (room for `room` floats), added in a fixed order.
cudaError_t sgemm_splitk(SGemm g, int ta, int tb, float *scratch, size_t room, cudaStream_t st) {
  const long long tiles = (long long)((g.M + SBM - 1) / SBM) * ((g.N + SBN - 1) / SBN);
  const size_t MN = (size_t)g.M * g.N;
  long long nb = (2 * 152 + tiles - 1) / tiles;
  const long long kmax = (g.K + 511) / 512;
  if (nb > kmax) nb = kmax;
  if (MN > 0 && (size_t)nb * MN > room) nb = (long long)(room / MN);
  if (nb <= 1 || g.batch != 1) return sgemm(g, ta, tb, st);
  const int kc = (int)((g.K + nb - 1) / nb);
  nb = (g.K + kc - 1) / kc;
  float *C = g.C;
  const int ldc = g.ldc;
  g.kc = kc;
  g.batch = (int)nb;
  g.sA = (long long)kc * (ta ? 1 : g.lda);
  g.sB = (long long)kc * (tb ? g.ldb : 1);
  g.C = scratch;
  g.ldc = g.M;
  g.sC = (long long)MN;
  cudaError_t e = sgemm(g, ta, tb, st);
  if (e != cudaSuccess) return e;
  k_sum_partials<<<grid_for(MN), 256, 0, st>>>(g.M, g.N, (int)nb, scratch, C, ldc);
  return cudaGetLastError();
}

// ------------------------------------------------------------- helpers
__global__ void k_real_to_c2(size_t n, const float *__restrict__ x, float2 *__restrict__ y) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x)
    y[e] = make_float2(x[e], 0.0f);
}

// U := 1.5 U - 0.5 D with D = U (U^T U): one Newton-Schulz step towards
// orthonormal columns.
__global__ void k_ns_real(size_t n, float *__restrict__ U, const float *__restrict__ D) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x)
    U[e] = fmaf(1.5f, U[e], -0.5f * D[e]);
}

__global__ void k_c2_to_real(size_t n, const float2 *__restrict__ x, float *__restrict__ y) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x)
    y[e] = x[e].x;
}

// (i, j, k) -> row i + a k, column j of an (a c) x b matrix: the mode-2
// unfolding's transpose laid out as a column-major matrix.
__global__ void k_perm_mode2(int a, int b, int c, const float *__restrict__ X,
                             float *__restrict__ Y) {
  const size_t N = (size_t)a * b * c;
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < N;
       v += (size_t)gridDim.x * blockDim.x) {
    const size_t i = v % a, j = (v / a) % b, k = v / ((size_t)a * b);
    Y[i + (size_t)a * k + (size_t)a * c * j] = X[v];
  }
}

// After the Jacobi sweeps on a Gram matrix G (n x n): W = G V, so the norm of
// column i of W is eigenvalue i.  U (n x r) receives the real parts of the r
// columns of V with the largest eigenvalues, in decreasing order (ties by
// index).  One block.
__global__ void __launch_bounds__(256)
    k_select_top(int n, int r, const float2 *__restrict__ W, const float2 *__restrict__ V,
                 float *__restrict__ U) {
  __shared__ float lam[kMaxSpatial];
  __shared__ int pos[kMaxSpatial];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int i = warp; i < n; i += nw) {
    float s = 0.f;
    for (int row = lane; row < n; row += 32) {
      const float2 w = W[(size_t)n * i + row];
      s = fmaf(w.x, w.x, fmaf(w.y, w.y, s));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) lam[i] = s;
  }
  __syncthreads();
  for (int i = tid; i < n; i += blockDim.x) {
    int k = 0;
    const float li = lam[i];
    for (int j = 0; j < n; ++j) k += (lam[j] > li) || (lam[j] == li && j < i);
    pos[i] = k;
  }
  __syncthreads();
  for (size_t e = tid; e < (size_t)n * n; e += blockDim.x) {
    const int i = (int)(e / n), row = (int)(e % n);
    const int k = pos[i];
    if (k < r) U[(size_t)n * k + row] = V[(size_t)n * i + row].x;
  }
}

// ------------------------------------------------ symmetric eigen-solver
// Two-sided cyclic Jacobi for a real symmetric n x n matrix B (n <= kSyevjMax)
// held in shared memory: B := J^T B J and V := V J over rounds of n/2 disjoint
// column pairs (the round-robin order of the t-SVT's kernel), each rotation
// the symmetric Schur 2x2 (Golub & Van Loan, Matrix Computations, Section
// 8.4) in FP32 (IEEE square roots and divisions).  A pair is rotated while
// |b_pq| > tol sqrt(|b_pp b_qq|) and |b_pq| > eps max_i |b_ii|: the second
// test leaves entries at the rounding level of B alone, so that the null
// block of a rank-deficient matrix does not chase its own rounding, while a
// leading eigenvector's component of size c along a null direction (an entry
// of about lambda c) is still rotated away down to c ~ eps.  Checking a pair
// reads three entries of B, and the disjoint pairs of a round are applied in
// parallel as 2 x 2 blocks of B (rows of pair P, columns of pair Q), so a
// sweep over a nearly diagonal B (a warm start) costs little more than its
// pair checks.  One CTA; V is n x n column-major in global memory (the
// identity is written when warm = 0); lam receives diag(B); *sweeps_out the
// sweeps used, -max_sweeps at the cap.
constexpr int kSyevjMax = 224;
constexpr int kSyevjThreads = 1024;
constexpr int kVBatch = 8;  // V items a thread has in flight

size_t syevj_smem(int n) {
  const int m = n + (n & 1);
  return sizeof(float) * (size_t)m * m;
}

__global__ void __launch_bounds__(kSyevjThreads, 1)
    k_syevj(int n, const float *__restrict__ B0, float *__restrict__ V, int warm,
            float *__restrict__ lam, int max_sweeps, int *__restrict__ sweeps_out) {
  extern __shared__ float sB[];  // m x m, row-major
  __shared__ int s_p[kSyevjMax / 2], s_q[kSyevjMax / 2], s_go[kSyevjMax / 2];
  __shared__ float s_c[kSyevjMax / 2], s_s[kSyevjMax / 2], s_t[kSyevjMax / 2];
  __shared__ int s_rot[kSyevjMax / 2], s_still[kSyevjMax / 2];  // rotated / other pairs
  __shared__ float s_red[32];
  __shared__ int s_any, s_nrot, s_nstill, s_sweep_any;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m = n + (n & 1), h = m / 2;
  const float eps = FLT_EPSILON * 0.5f;
  const float tol = 8.0f * sqrtf((float)n) * eps;
  // B0 is symmetric to rounding (V^T (G V) rounds its two triangles apart):
  // the mean of the two is exact for an exactly symmetric B0
  for (int e = tid; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e % m;
    sB[e] = (i < n && j < n) ? 0.5f * (B0[i + (size_t)n * j] + B0[j + (size_t)n * i]) : 0.0f;
  }
  if (!warm)
    for (int e = tid; e < n * n; e += blockDim.x) V[e] = (e % n) == (e / n) ? 1.0f : 0.0f;
  float dmax = 0.0f;
  for (int i = tid; i < n; i += blockDim.x) dmax = fmaxf(dmax, fabsf(B0[i + (size_t)n * i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
  if (lane == 0) s_red[warp] = dmax;
  __syncthreads();
  if (warp == 0) {
    float v = lane < (int)(blockDim.x >> 5) ? s_red[lane] : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) s_red[0] = v;
  }
  __syncthreads();
  const float floor_abs = eps * s_red[0];

  int sweeps = 0;
  bool converged = n < 2;
  if (converged) sweeps = 1;
  for (int sweep = 1; sweep <= max_sweeps && !converged; ++sweep) {
    if (tid == 0) s_sweep_any = 0;
    for (int r = 0; r < m - 1; ++r) {
      if (tid == 0) {
        s_any = 0;
        s_nrot = 0;
        s_nstill = 0;
      }
      __syncthreads();
      if (tid < h) {
        int p, q;
        if (tid == 0) {
          p = r;
          q = m - 1;
        } else {
          p = (r + tid) % (m - 1);
          q = (r - tid + m - 1) % (m - 1);
        }
        if (p > q) {
          const int x = p;
          p = q;
          q = x;
        }
        int go = 0;
        float c = 1.0f, sn = 0.0f, t = 0.0f;
        if (q < n) {
          const float app = sB[p * m + p], aqq = sB[q * m + q], apq = sB[p * m + q];
          const float aa = fabsf(apq);
          if (aa > floor_abs && aa > tol * sqrtf(fabsf(app)) * sqrtf(fabsf(aqq))) {
            // tan of the angle, |t| <= 1; for |tau| beyond 1e18 (tau^2 would
            // overflow) t = 1 / (2 tau) to within rounding
            const float tau = (aqq - app) / (2.0f * apq);
            const float at = fabsf(tau);
            const float tn = at > 1e18f ? 0.5f / at : 1.0f / (at + sqrtf(fmaf(at, at, 1.0f)));
            t = tau >= 0.0f ? tn : -tn;
            c = 1.0f / sqrtf(fmaf(t, t, 1.0f));
            sn = t * c;
            go = 1;
          }
        }
        s_p[tid] = p;
        s_q[tid] = q;
        s_c[tid] = c;
        s_s[tid] = sn;
        s_t[tid] = t;
        s_go[tid] = go;
        // the rotated pairs and the others, each in some order: every block
        // update depends only on its own entries and its two pairs, so the
        // order of the lists does not change any result
        if (go) {
          s_rot[atomicAdd(&s_nrot, 1)] = tid;
          s_any = 1;
          s_sweep_any = 1;
        } else {
          s_still[atomicAdd(&s_nstill, 1)] = tid;
        }
      }
      __syncthreads();
      if (s_any) {
        // B := J^T B J over the 2 x 2 blocks (rows of pair P, columns of pair
        // Q) that a rotation touches: with Q = thread mod h fixed (its
        // columns and rotation in registers) a thread walks the rows of every
        // rotated pair, then, if Q itself is rotated, the rows of the others.
        // A warp shares P, so the pair data it reads are broadcasts.
        const int k = s_nrot;
        const int groups = kSyevjThreads / h;
        const int Q = tid % h, g = tid / h;
        if (g < groups) {
          const int b0 = s_p[Q], b1 = s_q[Q], gq = s_go[Q];
          const float cq = s_c[Q], sq = s_s[Q];
          for (int i = g; i < k; i += groups) {
            const int P = s_rot[i];
            const int a0 = s_p[P], a1 = s_q[P];
            float x00 = sB[a0 * m + b0], x01 = sB[a0 * m + b1];
            float x10 = sB[a1 * m + b0], x11 = sB[a1 * m + b1];
            if (P == Q) {  // the rotated pair's own block: exact diagonal form
              const float tt = s_t[P];
              sB[a0 * m + a0] = x00 - tt * x01;
              sB[a1 * m + a1] = x11 + tt * x01;
              sB[a0 * m + a1] = 0.0f;
              sB[a1 * m + a0] = 0.0f;
              continue;
            }
            const float cp = s_c[P], sp = s_s[P];
            float y00 = cp * x00 - sp * x10, y10 = sp * x00 + cp * x10;
            float y01 = cp * x01 - sp * x11, y11 = sp * x01 + cp * x11;
            if (gq) {
              x00 = cq * y00 - sq * y01;
              x01 = sq * y00 + cq * y01;
              x10 = cq * y10 - sq * y11;
              x11 = sq * y10 + cq * y11;
            } else {
              x00 = y00; x01 = y01; x10 = y10; x11 = y11;
            }
            sB[a0 * m + b0] = x00;
            sB[a0 * m + b1] = x01;
            sB[a1 * m + b0] = x10;
            sB[a1 * m + b1] = x11;
          }
          if (gq)
            for (int i = g; i < h - k; i += groups) {
              const int P = s_still[i];
              const int a0 = s_p[P], a1 = s_q[P];
              const float x00 = sB[a0 * m + b0], x01 = sB[a0 * m + b1];
              const float x10 = sB[a1 * m + b0], x11 = sB[a1 * m + b1];
              sB[a0 * m + b0] = cq * x00 - sq * x01;
              sB[a0 * m + b1] = sq * x00 + cq * x01;
              sB[a1 * m + b0] = cq * x10 - sq * x11;
              sB[a1 * m + b1] = sq * x10 + cq * x11;
            }
        }
        // V := V J on the rotated pairs' columns (global memory, L2-resident):
        // each thread loads a batch of its items before it stores any, so the
        // loads' latencies overlap
        for (int base = tid; base < k * n; base += kSyevjThreads * kVBatch) {
          float vp[kVBatch], vq[kVBatch];
          int ip[kVBatch], iq[kVBatch], pr[kVBatch];
#pragma unroll
          for (int u = 0; u < kVBatch; ++u) {
            const int e = base + kSyevjThreads * u;
            pr[u] = -1;
            if (e < k * n) {
              const int P = s_rot[e / n], row = e % n;
              pr[u] = P;
              ip[u] = row + n * s_p[P];
              iq[u] = row + n * s_q[P];
              vp[u] = V[ip[u]];
              vq[u] = V[iq[u]];
            }
          }
#pragma unroll
          for (int u = 0; u < kVBatch; ++u) {
            if (pr[u] < 0) continue;
            const float c = s_c[pr[u]], sn = s_s[pr[u]];
            V[ip[u]] = c * vp[u] - sn * vq[u];
            V[iq[u]] = sn * vp[u] + c * vq[u];
          }
        }
      }
      __syncthreads();
    }
    sweeps = sweep;
    converged = (s_sweep_any == 0);
    __syncthreads();
  }
  for (int i = tid; i < n; i += blockDim.x) lam[i] = sB[i * m + i];
  if (tid == 0) *sweeps_out = converged ? sweeps : -max_sweeps;
}

// U (n x r) receives the r columns of V (n x n, real) with the largest lam,
// in decreasing order (ties by index).  One block.
__global__ void __launch_bounds__(256)
    k_select_top_real(int n, int r, const float *__restrict__ lam, const float *__restrict__ V,
                      float *__restrict__ U) {
  __shared__ float sl[kMaxSpatial];
  __shared__ int pos[kMaxSpatial];
  const int tid = threadIdx.x;
  for (int i = tid; i < n; i += blockDim.x) sl[i] = lam[i];
  __syncthreads();
  for (int i = tid; i < n; i += blockDim.x) {
    int k = 0;
    const float li = sl[i];
    for (int j = 0; j < n; ++j) k += (sl[j] > li) || (sl[j] == li && j < i);
    pos[i] = k;
  }
  __syncthreads();
  for (size_t e = tid; e < (size_t)n * n; e += blockDim.x) {
    const int i = (int)(e / n), row = (int)(e % n);
    const int k = pos[i];
    if (k < r) U[(size_t)n * k + row] = V[(size_t)n * i + row];
  }
}

// T_z = mu L + Gamma2 + D_w^*(mu F - Gamma3) for a given L (eq. Z_solution),
// D_n^T q(v) = q(v - e_n) - q(v).
__global__ void __launch_bounds__(256)
    k_tz(int n1, int n2, int n3, size_t N, const float *__restrict__ L,
         const float *__restrict__ G2, const float *__restrict__ F, const float *__restrict__ G3,
         float mu, float w0, float w1, float w2, float *__restrict__ T) {
  const size_t P = (size_t)n1 * n2;
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < N;
       v += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(v % n1);
    const int j = (int)((v / n1) % n2);
    const int k = (int)(v / P);
    const size_t col = (size_t)n1 * j, plane = P * k;
    const size_t b[3] = {plane + col + (i == 0 ? n1 - 1 : i - 1),
                         plane + (j == 0 ? (size_t)n1 * (n2 - 1) : col - n1) + i,
                         (k == 0 ? P * (n3 - 1) : plane - P) + col + i};
    const float w[3] = {w0, w1, w2};
    float adj = 0.f;
#pragma unroll
    for (int n = 0; n < 3; ++n) {
      const float qm = mu * F[b[n] + n * N] - G3[b[n] + n * N];
      const float q = mu * F[v + n * N] - G3[v + n * N];
      adj += w[n] * (qm - q);
    }
    T[v] = mu * L[v] + G2[v] + adj;
  }
}


}  // namespace

namespace {

// The workspace's pieces, in order; with a null base the carver only counts.
void layout(Carver &c, TuckerWs &t, int n1, int n2, int n3, const int r[3]) {
  const size_t N = (size_t)n1 * n2 * n3;
  const int nmax = n1 > n2 ? (n1 > n3 ? n1 : n3) : (n2 > n3 ? n2 : n3);
  t.U[0] = c.take<float>((size_t)n1 * r[0]);
  t.U[1] = c.take<float>((size_t)n2 * r[1]);
  t.U[2] = c.take<float>((size_t)n3 * r[2]);
  t.s0 = c.take<float>(N);
  t.s1 = c.take<float>(N);
  t.G = c.take<float>((size_t)nmax * nmax);
  t.W = c.take<float2>((size_t)nmax * nmax);
  t.D = c.take<float2>((size_t)nmax * nmax);
  t.Vr = c.take<float>((size_t)nmax * nmax);
  t.Wr = c.take<float>((size_t)nmax * nmax);
  t.Vm[0] = c.take<float2>((size_t)n1 * n1);
  t.Vm[1] = c.take<float2>((size_t)n2 * n2);
  t.Vm[2] = c.take<float2>((size_t)n3 * n3);
  t.sweeps = c.take<int>(kTuckerSweepSlots);
}

}  // namespace

// Carves the workspace (tucker_ws_bytes bytes at ws, 256-byte aligned).
void tucker_carve(TuckerWs &t, void *ws, int n1, int n2, int n3, const int r[3]) {
  Carver c(ws);
  t.n[0] = n1; t.n[1] = n2; t.n[2] = n3;
  t.r[0] = r[0]; t.r[1] = r[1]; t.r[2] = r[2];
  layout(c, t, n1, n2, n3, r);
  t.valid = 0;
  t.vvalid[0] = t.vvalid[1] = t.vvalid[2] = 0;
  t.warm = 0;
}

size_t tucker_ws_bytes(int n1, int n2, int n3, const int r[3]) {
  Carver c(nullptr);
  TuckerWs t{};
  layout(c, t, n1, n2, n3, r);
  return c.off;
}

namespace {

// One Newton-Schulz step U := 1.5 U - 0.5 U (U^T U) on an n x r factor, with
// FP64-accumulated products (scratch: r x r in sA, n x r in sB).
cudaError_t ns_step(float *U, int n, int r, float *sA, float *sB, cudaStream_t st) {
  cudaError_t e;
  if ((e = sgemm(mk(U, 0, n, U, 0, n, sA, 0, r, r, r, n, 1), 1, 0, st))) return e;  // U^T U
  if ((e = sgemm(mk(U, 0, n, sA, 0, r, sB, 0, n, n, r, r, 1), 0, 0, st))) return e;
  const size_t nr = (size_t)n * r;
  k_ns_real<<<grid_for(nr), 256, 0, st>>>(nr, U, sB);
  return cudaGetLastError();
}

// The r_n leading eigenvectors of the n x n Gram matrix t.G of mode `mode`
// into U.  With t.warm set, the solve starts from the eigenvectors of that
// mode's previous solve when there is one, otherwise from the identity.  Its
// sweep count goes to t.sweeps[slot].
//
// n <= kSyevjMax: the two-sided Jacobi (k_syevj) on B = V^T G V, V the warm
// basis made orthonormal again by one Newton-Schulz step (B = G cold), both
// products real and FP64-accumulated; V (real) is kept in Vm[mode].
// Larger n: the t-SVT's one-sided Jacobi on W = G V (the right singular
// vectors of a symmetric positive semi-definite matrix are its eigenvectors,
// its column norms the eigenvalues), with every nonzero column rotated
// (negl_rel = 0): a Gram matrix of a cube of lower multilinear rank than n
// has null columns at the rounding level, and skipping them would leave the
// leading eigenvectors with null-space components of about
// (n eps) ||G|| / lambda_r, which nothing else corrects.
//
// Either way the selected factor then gets one Newton-Schulz step with
// FP64-accumulated products: each rotation is orthogonal only to about an
// ulp, and a rank-deficient Gram matrix takes many sweeps, so the columns of
// U drift from unit norm by up to 1e-4, which U U^T would turn into a scaling
// of the projection.
cudaError_t eig_top(TuckerWs &t, int mode, int n, int r, float *U, int slot, cudaStream_t st) {
  const size_t nn = (size_t)n * n;
  const int warm = t.warm && t.vvalid[mode];
  cudaError_t e;
  if (n <= kSyevjMax) {
    float *V = reinterpret_cast<float *>(t.Vm[mode]);
    float *scr = reinterpret_cast<float *>(t.W);  // 2 n^2 floats
    float *lam = reinterpret_cast<float *>(t.D);
    const float *B0 = t.G;
    if (warm) {
      if ((e = ns_step(V, n, n, scr, scr + nn, st)) != cudaSuccess) return e;
      if ((e = sgemm(mk(t.G, 0, n, V, 0, n, t.Wr, 0, n, n, n, n, 1), 0, 0, st))) return e;  // G V
      if ((e = sgemm(mk(V, 0, n, t.Wr, 0, n, t.Vr, 0, n, n, n, n, 1), 1, 0, st))) return e;
      B0 = t.Vr;  // V^T G V
    }
    const size_t smem = syevj_smem(n);
    if ((e = cudaFuncSetAttribute(k_syevj, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
      return e;
    k_syevj<<<1, kSyevjThreads, smem, st>>>(n, B0, V, warm, lam, kMaxSweeps, t.sweeps + slot);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_select_top_real<<<1, 256, 0, st>>>(n, r, lam, V, U);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  } else {
    float2 *V = t.Vm[mode];
    if (warm) {
      CGemm g{};
      g.batch = 1;
      g.M = n; g.N = n; g.K = n;
      g.lda = n; g.ldb = n; g.ldc = n;
      g.A = V; g.B = V; g.opB = 1; g.C = t.W;  // V V^H
      if ((e = launch_cgemm(g, st)) != cudaSuccess) return e;
      g.A = t.W; g.B = V; g.opB = 0; g.C = t.D;  // (V V^H) V
      if ((e = launch_cgemm(g, st)) != cudaSuccess) return e;
      if ((e = launch_ns_update(n, 1, nn, V, t.D, st)) != cudaSuccess) return e;
      k_c2_to_real<<<grid_for(nn), 256, 0, st>>>(nn, V, t.Vr);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if ((e = sgemm(mk(t.G, 0, n, t.Vr, 0, n, t.Wr, 0, n, n, n, n, 1), 0, 0, st))) return e;
    }
    k_real_to_c2<<<grid_for(nn), 256, 0, st>>>(nn, warm ? t.Wr : t.G, t.W);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const Dims dj = make_dims(n, n, 1);
    JacOpt o;
    o.warm = warm;
    o.negl_rel = 0.0f;
    if ((e = launch_jacobi(dj, 1, t.W, V, -1.0f, kMaxSweeps, t.sweeps + slot, nullptr, st, o)) !=
        cudaSuccess)
      return e;
    k_select_top<<<1, 256, 0, st>>>(n, r, t.W, V, U);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if ((e = ns_step(U, n, r, t.Wr, t.Vr, st)) != cudaSuccess) return e;
  t.vvalid[mode] = 1;
  return cudaSuccess;
}

// Gram matrix of mode `mode` of X x_m Uo[m]^T (m != mode), into t.G, then
// the leading eigenvectors into `out`.  Uo[m] is n_m x ro[m].
cudaError_t mode_update(TuckerWs &t, const float *X, int mode, const float *const Uo[3],
                        const int ro[3], float *out, cudaStream_t st) {
  const int a = t.n[0], b = t.n[1], c = t.n[2];
  const size_t room = (size_t)a * b * c;  // s0 is free once s1 is formed
  cudaError_t e;
  if (mode == 0) {
    // s0 = X x3 U3^T: (ab x c) (c x r3); s1 = s0 x2 U2^T per k': (a x b)(b x r2)
    if ((e = sgemm(mk(X, 0, a * b, Uo[2], 0, c, t.s0, 0, a * b, a * b, ro[2], c, 1), 0, 0, st)))
      return e;
    if ((e = sgemm(mk(t.s0, (long long)a * b, a, Uo[1], 0, b, t.s1, (long long)a * ro[1], a, a,
                      ro[1], b, ro[2]), 0, 0, st)))
      return e;
    // G = s1 s1^T, s1 as a x (r2 r3)
    if ((e = sgemm_splitk(mk(t.s1, 0, a, t.s1, 0, a, t.G, 0, a, a, a, ro[1] * ro[2], 1), 0, 1, t.s0, room, st)))
      return e;
    return eig_top(t, 0, a, t.r[0], out, 0, st);
  }
  if (mode == 1) {
    // s0 = X x3 U3^T; s1 (rows (i', k'), columns j) = U1^T s0_k' per k'
    if ((e = sgemm(mk(X, 0, a * b, Uo[2], 0, c, t.s0, 0, a * b, a * b, ro[2], c, 1), 0, 0, st)))
      return e;
    if ((e = sgemm(mk(Uo[0], 0, a, t.s0, (long long)a * b, a, t.s1, ro[0], ro[0] * ro[2], ro[0], b,
                      a, ro[2]), 1, 0, st)))
      return e;
    // G = s1^T s1, s1 as (r1 r3) x b
    if ((e = sgemm_splitk(mk(t.s1, 0, ro[0] * ro[2], t.s1, 0, ro[0] * ro[2], t.G, 0, b, b, b,
                             ro[0] * ro[2], 1), 1, 0, t.s0, room, st)))
      return e;
    return eig_top(t, 1, b, t.r[1], out, 1, st);
  }
  // mode 2: s0 = U1^T X (r1 x bc); s1 = s0_k U2 per k (r1 x r2); G = s1^T s1, s1 as (r1 r2) x c
  if ((e = sgemm(mk(Uo[0], 0, a, X, 0, a, t.s0, 0, ro[0], ro[0], b * c, a, 1), 1, 0, st))) return e;
  if ((e = sgemm(mk(t.s0, (long long)ro[0] * b, ro[0], Uo[1], 0, b, t.s1, (long long)ro[0] * ro[1],
                    ro[0], ro[0], ro[1], b, c), 0, 0, st)))
    return e;
  if ((e = sgemm_splitk(mk(t.s1, 0, ro[0] * ro[1], t.s1, 0, ro[0] * ro[1], t.G, 0, c, c, c,
                           ro[0] * ro[1], 1), 1, 0, t.s0, room, st)))
    return e;
  return eig_top(t, 2, c, t.r[2], out, 2, st);
}

// Gram matrix of mode `mode` of X itself (the truncated HOSVD's), into t.G,
// then the leading eigenvectors into U[mode].
cudaError_t hosvd_mode(TuckerWs &t, const float *X, int mode, cudaStream_t st) {
  const int a = t.n[0], b = t.n[1], c = t.n[2];
  const size_t room = (size_t)a * b * c;  // s0 holds nothing here
  cudaError_t e;
  if (mode == 0) {
    if ((e = sgemm_splitk(mk(X, 0, a, X, 0, a, t.G, 0, a, a, a, b * c, 1), 0, 1, t.s0, room, st))) return e;
    return eig_top(t, 0, a, t.r[0], t.U[0], 3, st);
  }
  if (mode == 1) {
    k_perm_mode2<<<grid_for((size_t)a * b * c), 256, 0, st>>>(a, b, c, X, t.s1);
    if ((e = cudaGetLastError())) return e;
    if ((e = sgemm_splitk(mk(t.s1, 0, a * c, t.s1, 0, a * c, t.G, 0, b, b, b, a * c, 1), 1, 0, t.s0, room, st)))
      return e;
    return eig_top(t, 1, b, t.r[1], t.U[1], 4, st);
  }
  if ((e = sgemm_splitk(mk(X, 0, a * b, X, 0, a * b, t.G, 0, c, c, c, a * b, 1), 1, 0, t.s0, room, st))) return e;
  return eig_top(t, 2, c, t.r[2], t.U[2], 5, st);
}

}  // namespace

// X (n1 x n2 x n3, in place) := its Tucker projection after one HOOI sweep
// started from the factors of the previous call (from the truncated HOSVD of
// X when t.valid == 0).
cudaError_t tucker_project(TuckerWs &t, float *X, cudaStream_t st) {
  const int a = t.n[0], b = t.n[1], c = t.n[2];
  const int *r = t.r;
  cudaError_t e;
  if (!t.valid)
    for (int n = 0; n < 3; ++n)
      if ((e = hosvd_mode(t, X, n, st)) != cudaSuccess) return e;
  // HOOI sweep: each factor from the current others
  for (int n = 0; n < 3; ++n) {
    const float *Uo[3] = {t.U[0], t.U[1], t.U[2]};
    if ((e = mode_update(t, X, n, Uo, r, t.U[n], st)) != cudaSuccess) return e;
  }
  // s1 holds X x1 U1^T x2 U2^T ((r1 r2) x c) from the mode-3 update
  // core = s1 U3 ((r1 r2) x r3) -> s0
  if ((e = sgemm(mk(t.s1, 0, r[0] * r[1], t.U[2], 0, c, t.s0, 0, r[0] * r[1], r[0] * r[1], r[2], c,
                    1), 0, 0, st)))
    return e;
  // core x3 U3 = core U3^T ((r1 r2) x c) -> s1
  if ((e = sgemm(mk(t.s0, 0, r[0] * r[1], t.U[2], 0, c, t.s1, 0, r[0] * r[1], r[0] * r[1], c, r[2],
                    1), 0, 1, st)))
    return e;
  // x2 U2 per band: (r1 x r2)(r2 x b) -> s0 (r1 x b x c)
  if ((e = sgemm(mk(t.s1, (long long)r[0] * r[1], r[0], t.U[1], 0, b, t.s0, (long long)r[0] * b,
                    r[0], r[0], b, r[1], c), 0, 1, st)))
    return e;
  // x1 U1: (a x r1)(r1 x bc) -> X
  if ((e = sgemm(mk(t.U[0], 0, a, t.s0, 0, r[0], X, 0, a, a, b * c, r[0], 1), 0, 0, st))) return e;
  t.valid = 1;
  return cudaSuccess;
}

cudaError_t launch_tz(const Dims &d, const float *L, const float *G2, const float *F,
                      const float *G3, float mu, const float w[3], float *T, cudaStream_t st) {
  k_tz<<<grid_for(d.N), 256, 0, st>>>(d.n1, d.n2, d.n3, d.N, L, G2, F, G3, mu, w[0], w[1], w[2], T);
  return cudaGetLastError();
}

}  // namespace lrstv
