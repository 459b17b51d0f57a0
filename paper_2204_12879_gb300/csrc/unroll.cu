// unroll.cu -- the plain-LRSTV iteration (Algorithm 1, Section III-C)
// unrolled over K iterations with free per-iteration scalars theta_k = (tau,
// alpha, lambda, mu) on a batch of B equal-shape cubes, and its hand-written
// adjoint: the gradient of a loss on the last L with respect to every theta_k
// and to the noisy input Y.
//
// Forward: iteration k reads state slot k and writes slot k+1 (every slot is
// kept: 17 B N floats each, the per-iteration checkpoints), and keeps the SVD
// factors W_k, V_k and the singular values of every Fourier slice of the
// E-update.  With LRSTV_FLAG_UNROLL_RECOMPUTE it keeps one slot of W and
// sigma (and of V without a warm start) and the backward pass reruns
// iteration k's factorisation from the checkpoints before its t-SVT adjoint.
// The kernels are those of the plain iteration (the Jacobi with a negative
// threshold keeps V unscaled; a separate kernel forms sigma and the
// thresholded V exactly as the Jacobi epilogue does).
//
// Backward, per iteration in reverse, with adjoint buffers a* in the layout of
// a state slot (the adjoint of the new state on entry, of the old on exit):
//   k_adj_sdual  multipliers, S soft threshold, seeds of the E and F adjoints
//   t-SVT adjoint  DFT -> P = G V -> H = W^H P -> coefficients -> X = W K' + P
//                  diag(q) -> X V^H -> inverse DFT
//   k_adj_f      F soft threshold, the E-step's B = F - Gamma4/mu
//   k_adj_dz     bZ += D_w^T bg
//   Z-solve      bT = (mu (I + D^T D))^{-1} bZ (the operator is symmetric)
//   k_adj_l      T_z assembly and the L-update
// The scalars' gradients: FP32 partial sums per thread, added per block in FP64
// with the scalar factors applied once, then atomically.
//
// SVT adjoint (per slice, working orientation A = W diag(1/s) . diag(s) V^H,
// f = max(s - t, 0), q = f / s, kept: s > t): with H = U^H G V,
//   M_ij = a_ij H_ij + b_ij conj(H_ji),  M_ii = Re H_ii + i q_i Im H_ii (kept)
//   both kept:  a = 1 - t / (s_i + s_j),  b = t / (s_i + s_j)
//   one kept (i):  a = s_i f_i / (s_i^2 - s_j^2),  b = s_j f_i / (s_i^2 - s_j^2)
//   (s_i - s_j >= f_i > 0 there, so no coefficient exceeds 1 in magnitude)
// and dA = (U (M - H diag q) + G V diag q) V^H, which also carries the parts
// of G outside the range of A (V is the full unitary factor).  k_svt_coef
// forms diag(1/s)(M - H diag q) in a closed form that never divides by a cut
// singular value.
#include <math.h>
#include <new>
#include <stdlib.h>
#include <string.h>

#include "lrstv.h"
#include "lrstv_internal.cuh"

namespace lrstv {

namespace {

constexpr int kT = 256;

// theta slot indices
enum { kTau = 0, kAlpha = 1, kLam = 2, kMu = 3 };

// out[s] += sum_c m[s][c] R_c for the raw sums R_c of a kernel: each block
// adds its threads' FP32 partials r[c] in FP64 and applies the scalar factors
// (1/mu^2, tau/mu^2, ...) once, with one atomic per nonzero slot.  Every
// thread of the block must call it.
struct Lin {
  double m[4][4];
};

__device__ void block_lin(const float (&r)[4], const Lin &L, double *out) {
  __shared__ double sh[4][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    double v = (double)r[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[c][wid] = v;
  }
  __syncthreads();
  if (wid == 0) {
    double R[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      double v = lane < nw ? sh[c][lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      R[c] = v;
    }
    if (lane == 0) {
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        double acc = 0.0;
#pragma unroll
        for (int c = 0; c < 4; ++c) acc += L.m[o][c] * R[c];
        if (acc != 0.0) atomicAdd(out + o, acc);
      }
    }
  }
}

struct Geo {
  int n1, n2, n3;
  size_t N, P;
};

// voxel q of a cube -> its circular neighbours q + e_n / q - e_n
__device__ __forceinline__ void nbrs(const Geo &g, size_t q, size_t (&fw)[3], size_t (&bw)[3]) {
  const int i = (int)(q % g.n1);
  const size_t r = q / g.n1;
  const int j = (int)(r % g.n2);
  const int k = (int)(r / g.n2);
  const size_t col = (size_t)g.n1 * j, plane = g.P * k;
  fw[0] = plane + col + (i + 1 == g.n1 ? 0 : i + 1);
  bw[0] = plane + col + (i == 0 ? g.n1 - 1 : i - 1);
  fw[1] = plane + (j + 1 == g.n2 ? 0 : col + g.n1) + i;
  bw[1] = plane + (j == 0 ? (size_t)g.n1 * (g.n2 - 1) : col - g.n1) + i;
  fw[2] = (k + 1 == g.n3 ? 0 : plane + g.P) + col + i;
  bw[2] = (k == 0 ? g.P * (g.n3 - 1) : plane - g.P) + col + i;
}

__device__ __forceinline__ bool soft_keep(float x, float d, float &sgn) {
  // R_d(x) = sign(x) max(|x| - d, 0): derivative 1 where x > d or x < -d
  sgn = x > d ? 1.0f : -1.0f;
  return x > d || x < -d;
}

struct AdjPtrs {
  // state before (o*) and after (n*) the iteration
  const float *Y, *oS, *oG1, *oG2, *oF, *oE, *oG3, *oG4;
  const float *nL, *nZ, *nS, *nF, *nE;
  // adjoint buffers
  float *aY, *aL, *aZ, *aS, *aG1, *aG2, *aF, *aE, *aG3, *aG4;
  float *X3;  // 3 B N: bB from the t-SVT adjoint, then bg
  float *bT;  // B N
  double *dth;  // this iteration's 4 gradient slots
};

// Multipliers and S (eq. S_solution) backwards; seeds the E and F adjoints.
// Raw sums: R0 = <aG1, Y-L-S> + <aG2, L-Z> + <aG3, D_wZ-F> + <aG4, E-F>,
// R1 = sum over kept S entries of bS sign(u), R2 = <bu, Gamma1_old>.
__global__ void __launch_bounds__(kT)
    k_adj_sdual(Geo g, int B, AdjPtrs p, float mu, float thr_s, float w0, float w1, float w2,
                Lin lin) {
  float r[4] = {0.f, 0.f, 0.f, 0.f};
  const float w[3] = {w0, w1, w2};
  const size_t total = (size_t)B * g.N;
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < total;
       v += (size_t)gridDim.x * blockDim.x) {
    const size_t b = v / g.N, q = v - b * g.N;
    const float y = p.Y[v], l1 = p.nL[v], s1 = p.nS[v], z1 = p.nZ[v], g1 = p.oG1[v];
    const float bG1 = p.aG1[v], bG2 = p.aG2[v];
    const float u = y - l1 + g1 / mu;  // the forward's operation order
    float sgn;
    const bool keep = soft_keep(u, thr_s, sgn);
    const float bSe = p.aS[v] - mu * bG1;
    const float bu = keep ? bSe : 0.0f;
    p.aY[v] += mu * bG1 + bu;
    p.aG1[v] = bG1 + bu / mu;
    p.aL[v] = p.aL[v] - mu * bG1 + mu * bG2 - bu;
    p.aZ[v] = p.aZ[v] - mu * bG2;
    float r0 = bG1 * (y - l1 - s1) + bG2 * (l1 - z1);
    r[1] += bu * sgn;
    r[2] += bu * g1;
    size_t fw[3], bw[3];
    nbrs(g, q, fw, bw);
    const float *zc = p.nZ + b * g.N;
#pragma unroll
    for (int n = 0; n < 3; ++n) {
      const size_t vn = b * 3 * g.N + n * g.N + q;
      const float gn = w[n] * (zc[fw[n]] - z1);
      const float bG3 = p.aG3[vn], bG4 = p.aG4[vn], f1 = p.nF[vn], e1 = p.nE[vn];
      p.aE[vn] = p.aE[vn] + mu * bG4;
      p.aF[vn] = p.aF[vn] - mu * bG3 - mu * bG4;
      r0 += bG3 * (gn - f1) + bG4 * (e1 - f1);
    }
    r[0] += r0;
  }
  block_lin(r, lin, p.dth);
}

// F (eq. F_solution) and the E-step input B = F - Gamma4/mu backwards.
// Raw sums: R0 = <bB, Gamma4_old>, R1 = sum over kept F entries of bF sign(a),
// R2 = <ba, Gamma3_old + Gamma4_old>.
__global__ void __launch_bounds__(kT)
    k_adj_f(Geo g, int B, AdjPtrs p, float mu, float thr_f, float w0, float w1, float w2,
            Lin lin) {
  float r[4] = {0.f, 0.f, 0.f, 0.f};
  const float w[3] = {w0, w1, w2};
  const size_t total = (size_t)B * g.N;
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < total;
       v += (size_t)gridDim.x * blockDim.x) {
    const size_t b = v / g.N, q = v - b * g.N;
    size_t fw[3], bw[3];
    nbrs(g, q, fw, bw);
    const float *zc = p.nZ + b * g.N;
    const float z1 = zc[q];
#pragma unroll
    for (int n = 0; n < 3; ++n) {
      const size_t vn = b * 3 * g.N + n * g.N + q;
      const float gn = w[n] * (zc[fw[n]] - z1);
      const float h3 = p.oG3[vn], ee = p.oE[vn], h4 = p.oG4[vn];
      // the forward's operation order, so the mask is the forward's
      const float t1 = gn + h3 / mu;
      const float t2 = ee + h4 / mu;
      const float x = 0.5f * (t1 + t2);
      float sgn;
      const bool keep = soft_keep(x, thr_f, sgn);
      const float bB = p.X3[vn];
      const float bF = p.aF[vn] + bB;
      const float ba = keep ? bF : 0.0f;
      r[0] += bB * h4;
      r[1] += ba * sgn;
      r[2] += ba * (h3 + h4);
      p.X3[vn] = mu * p.aG3[vn] + 0.5f * ba;  // bg
      p.aG3[vn] += 0.5f * ba / mu;
      p.aE[vn] = 0.5f * ba;
      p.aG4[vn] = p.aG4[vn] - bB / mu + 0.5f * ba / mu;
    }
  }
  block_lin(r, lin, p.dth);
}

// bZ += D_w^T bg.  Raw sum: R0 = <bZ, Z1> (the Z-solve's mu derivative).
__global__ void __launch_bounds__(kT)
    k_adj_dz(Geo g, int B, AdjPtrs p, float w0, float w1, float w2, Lin lin) {
  float r[4] = {0.f, 0.f, 0.f, 0.f};
  const float w[3] = {w0, w1, w2};
  const size_t total = (size_t)B * g.N;
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < total;
       v += (size_t)gridDim.x * blockDim.x) {
    const size_t b = v / g.N, q = v - b * g.N;
    size_t fw[3], bw[3];
    nbrs(g, q, fw, bw);
    float adj = 0.0f;
#pragma unroll
    for (int n = 0; n < 3; ++n) {
      const float *bg = p.X3 + b * 3 * g.N + n * g.N;
      adj += w[n] * (bg[bw[n]] - bg[q]);
    }
    const float bz = p.aZ[v] + adj;
    p.aZ[v] = bz;
    r[0] += bz * p.nZ[v];
  }
  block_lin(r, lin, p.dth);
}

// T_z = mu L1 + Gamma2 + D_w^*(mu F - Gamma3) and L (eq. X_solution) backwards.
// Raw sums: R0 = <bT, L1> + <D_w bT, F_old>, R1 = <bL, Gamma1_old - Gamma2_old>.
__global__ void __launch_bounds__(kT)
    k_adj_l(Geo g, int B, AdjPtrs p, float mu, float w0, float w1, float w2, Lin lin) {
  float r[4] = {0.f, 0.f, 0.f, 0.f};
  const float w[3] = {w0, w1, w2};
  const size_t total = (size_t)B * g.N;
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < total;
       v += (size_t)gridDim.x * blockDim.x) {
    const size_t b = v / g.N, q = v - b * g.N;
    size_t fw[3], bw[3];
    nbrs(g, q, fw, bw);
    const float *bt = p.bT + b * g.N;
    const float bT = bt[q];
    const float bL = p.aL[v] + mu * bT;
    float r0 = bT * p.nL[v];
#pragma unroll
    for (int n = 0; n < 3; ++n) {
      const size_t vn = b * 3 * g.N + n * g.N + q;
      const float bp = w[n] * (bt[fw[n]] - bT);
      p.aF[vn] = mu * bp;
      p.aG3[vn] -= bp;
      r0 += bp * p.oF[vn];
    }
    const float g1 = p.oG1[v], g2 = p.oG2[v];
    p.aY[v] += 0.5f * bL;
    p.aS[v] = -0.5f * bL;
    p.aZ[v] = 0.5f * bL;
    p.aG1[v] += 0.5f * bL / mu;
    p.aG2[v] = p.aG2[v] + bT - 0.5f * bL / mu;
    p.aL[v] = 0.0f;
    r[0] += r0;
    r[1] += bL * (g1 - g2);
  }
  block_lin(r, lin, p.dth);
}

// Per slice: Hraw = W^H G V (nc x nc) -> K' in place, P = G V (nr x nc) ->
// P diag q in place, with (kept: s > t, decided in FP64 like the forward)
//   K'_ij = c_ij (Hraw_ij + conj(Hraw_ji)),
//   c_ij = t / (s_i s_j (s_i + s_j))            both kept,
//   c_ij = f_k / (s_k (s_k^2 - s_o^2))          only k kept (o the other),
//   c_ij = 0                                    neither kept,
// which is diag(1/s) (M - H diag q) of the header comment with H = diag(1/s)
// Hraw written out; it never divides by a singular value that is cut, and
// every c_ij <= 1 / s_k^2.  Raw sum R0 = -sum_kept Re Hraw_ii / s_i times the
// slice's multiplicity (1 or 2 for its conjugate twin).
__global__ void __launch_bounds__(kT)
    k_svt_coef(int nr, int nc, int h, int n3, size_t pstride, float2 *__restrict__ H,
               float2 *__restrict__ Pm, const double *__restrict__ sig, float t, Lin lin,
               double *dth) {
  __shared__ float s_s[kMaxSpatial], s_q[kMaxSpatial];
  __shared__ unsigned char s_k[kMaxSpatial];
  const int s = blockIdx.x;
  const double *sg = sig + (size_t)s * nc;
  float2 *Hs = H + (size_t)s * nc * nc;
  float2 *Ps = Pm + (size_t)s * pstride;
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    const double si = sg[i];
    const bool kept = si > (double)t;
    s_s[i] = (float)si;
    s_k[i] = kept ? 1 : 0;
    s_q[i] = kept ? (float)((si - (double)t) / si) : 0.0f;
  }
  __syncthreads();
  float tb = 0.0f;
  for (int e = threadIdx.x; e < nc * nc; e += blockDim.x) {
    const int i = e % nc, j = e / nc;
    if (i > j) continue;
    const bool ki = s_k[i], kj = s_k[j];
    const float si = s_s[i], sj = s_s[j];
    const float2 hij = Hs[i + (size_t)nc * j];
    float c = 0.0f;
    if (ki && kj) {
      c = t / (si * sj * (si + sj));
    } else if (ki || kj) {
      // (s_k - t) / (s_k - s_o) lies in (0, 1]: formed in FP64, where both
      // differences are positive (s_o <= t < s_k was decided there)
      const double dk = ki ? sg[i] : sg[j], dn = ki ? sg[j] : sg[i];
      const float ratio = (float)((dk - (double)t) / (dk - dn));
      const float sk = ki ? si : sj, so = ki ? sj : si;
      c = ratio / (sk * (sk + so));
    }
    if (i == j) {
      if (ki) tb -= hij.x / si;
      Hs[i + (size_t)nc * i] = make_float2(2.0f * c * hij.x, 0.0f);
      continue;
    }
    const float2 hji = Hs[j + (size_t)nc * i];
    const float zr = hij.x + hji.x, zi = hij.y - hji.y;  // Hraw_ij + conj(Hraw_ji)
    Hs[i + (size_t)nc * j] = make_float2(c * zr, c * zi);
    Hs[j + (size_t)nc * i] = make_float2(c * zr, -c * zi);
  }
  for (size_t e = threadIdx.x; e < (size_t)nr * nc; e += blockDim.x) {
    const float qj = s_q[e / nr];
    const float2 v = Ps[e];
    Ps[e] = make_float2(v.x * qj, v.y * qj);
  }
  // every full-spectrum slice counts: k and n3 - k are conjugate twins
  const int k = s % h;
  const float mult = (k == 0 || (n3 % 2 == 0 && k == n3 / 2)) ? 1.0f : 2.0f;
  float r[4] = {tb * mult, 0.f, 0.f, 0.f};
  block_lin(r, lin, dth);
}

__global__ void k_sum3(size_t n, const float *a, const float *b, const float *c, float *out) {
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < n;
       v += (size_t)gridDim.x * blockDim.x)
    out[v] = a[v] + b[v] + c[v];
}

unsigned grid_for(size_t n) {
  size_t b = (n + kT - 1) / kT;
  const size_t cap = 152ull * 8ull;
  return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

}  // namespace lrstv

using namespace lrstv;

// One state slot: 17 B N floats, fields back to back (scalar fields B N each,
// the gradient fields 3 B N each, cube-major inside a field).
struct UnrollSlot {
  float *L, *Z, *S, *G1, *G2, *F, *E, *G3, *G4;
};

struct lrstv_unroll {
  Dims d;
  int B, K;
  float w[3];
  unsigned flags;
  void *arena;
  size_t arena_bytes;
  size_t slot_floats;  // 17 B N
  float *Y;
  float *slots;        // (K + 1) slots
  float *adj;          // one slot-shaped adjoint state
  float *aY, *T, *X3, *bT;
  float2 *specA, *specB;
  // SVD factors of the E-updates, in slots of 3 B h Fourier slices (P and
  // nc^2 complex each, nc doubles of sigma): one slot per iteration, or, for a
  // handle that recomputes them in the backward pass, one slot of W and sigma
  // and one of V (K of V with a warm start: iteration k starts from V_{k-1})
  int nw, nv;          // slots of W and sigma, of V
  float2 *W, *V;
  double *sig;
  float2 *Hs;          // 3 B h nc^2 complex: thresholded V, then H / K'
  int *sweeps;         // K x 3 B h
  int *jsched;         // task-graph Jacobi scratch (jacobi_task_ints(3 B h))
  float *ms2;          // 3 B: per gradient tensor, largest mean-square column norm
  int *gemm_err;
  Tables tb;
  double *theta;       // host copy of the last forward's scalars (K x 4)
  int have_forward;
};

namespace {

UnrollSlot slot_at(const lrstv_unroll *u, float *base) {
  const size_t BN = (size_t)u->B * u->d.N;
  UnrollSlot s;
  s.L = base;
  s.Z = base + BN;
  s.S = base + 2 * BN;
  s.G1 = base + 3 * BN;
  s.G2 = base + 4 * BN;
  s.F = base + 5 * BN;
  s.E = base + 8 * BN;
  s.G3 = base + 11 * BN;
  s.G4 = base + 14 * BN;
  return s;
}

UnrollSlot slot_k(const lrstv_unroll *u, int k) { return slot_at(u, u->slots + (size_t)k * u->slot_floats); }

// iteration k's factor slots (a single slot is shared by every iteration)
float2 *w_slot(const lrstv_unroll *u, int k) {
  return u->W + (size_t)(k % u->nw) * 3 * u->B * u->d.h * u->d.P;
}
float2 *v_slot(const lrstv_unroll *u, int k) {
  return u->V + (size_t)(k % u->nv) * 3 * u->B * u->d.h * u->d.nc * u->d.nc;
}
double *sig_slot(const lrstv_unroll *u, int k) {
  return u->sig + (size_t)(k % u->nw) * 3 * u->B * u->d.h * u->d.nc;
}

size_t unroll_layout(lrstv_unroll *u, void *base) {
  const Dims &d = u->d;
  const size_t BN = (size_t)u->B * d.N;
  const size_t ns = (size_t)3 * u->B * d.h;  // Fourier slices of one E-update
  Carver c(base);
  u->Y = c.take<float>(BN);
  u->slots = c.take<float>(u->slot_floats * (size_t)(u->K + 1));
  u->adj = c.take<float>(u->slot_floats);
  u->aY = c.take<float>(BN);
  u->T = c.take<float>(BN);
  u->X3 = c.take<float>(3 * BN);
  u->bT = c.take<float>(BN);
  u->specA = c.take<float2>(ns * d.P);
  u->specB = c.take<float2>(ns * d.P);
  u->W = c.take<float2>((size_t)u->nw * ns * d.P);
  u->V = c.take<float2>((size_t)u->nv * ns * d.nc * d.nc);
  u->sig = c.take<double>((size_t)u->nw * ns * d.nc);
  u->Hs = c.take<float2>(ns * d.nc * d.nc);
  u->sweeps = c.take<int>((size_t)u->K * ns);
  u->jsched = c.take<int>(jacobi_task_ints((int)ns));
  u->ms2 = c.take<float>((size_t)3 * u->B);
  u->gemm_err = c.take<int>(1);
  carve_tables(c, d, u->tb);
  return c.off;
}

GemmSel unroll_gemm(const lrstv_unroll *u) {
  if (u->flags & LRSTV_FLAG_SIMT_GEMM) return kSimt;
  // 3xTF32: the unrolled form has no mixed-precision mode
  return GemmSel{true, u->gemm_err, 0, (u->flags & LRSTV_FLAG_SIMT_DFT) == 0};
}

#define UCK(x)                                  \
  do {                                          \
    if ((x) != cudaSuccess) return LRSTV_ERR_CUDA; \
  } while (0)

// The factor half of iteration k's E-update: the SVDs of the Fourier slices of
// F - Gamma4_k/mu (F the iteration's new F, Gamma4_k the multiplier it started
// from), into W_k, V_k and sigma_k, and the thresholded V into Hs.  The same
// call in the backward pass of a recomputing handle reproduces the forward's
// factors bit for bit: every kernel here is deterministic, and a warm start
// reads V_{k-1}, which such a handle keeps.
int e_factor(lrstv_unroll *u, int k, const float *F, const float *G4, double mu, double alpha,
             cudaStream_t st) {
  const Dims &d = u->d;
  const int B = u->B;
  const size_t ns = (size_t)3 * B * d.h;
  const GemmSel gs = unroll_gemm(u);
  float2 *Wk = w_slot(u, k);
  float2 *Vk = v_slot(u, k);
  double *sk = sig_slot(u, k);
  const int warm = (u->flags & LRSTV_FLAG_WARM_START) && k > 0;
  if (warm) {
    // start from the previous iteration's right singular vectors, made
    // unitary again by one Newton-Schulz step, exactly as a plan does
    const long long nc2 = (long long)d.nc * d.nc, P = (long long)d.P;
    UCK(launch_r2c3(d, 3 * B, F, G4, (float)(1.0 / mu), u->specA, 1, u->tb.tw3, st, gs));
    UCK(cudaMemcpyAsync(Vk, v_slot(u, k - 1), sizeof(float2) * ns * d.nc * d.nc,
                        cudaMemcpyDeviceToDevice, st));
    CGemm g{};
    g.batch = (int)ns;
    g.A = Vk; g.sA = nc2; g.lda = d.nc;
    g.B = Vk; g.sB = nc2; g.ldb = d.nc; g.opB = 1;
    g.C = u->Hs; g.sC = nc2; g.ldc = d.nc;
    g.M = d.nc; g.N = d.nc; g.K = d.nc;
    UCK(gemm(g, gs, st));
    g.A = u->Hs; g.B = Vk; g.opB = 0;
    g.C = u->specB; g.sC = P; g.ldc = d.nc;
    UCK(gemm(g, gs, st));
    UCK(launch_ns_update(d.nc, (int)ns, (size_t)P, Vk, u->specB, st));
    g.A = u->specA; g.sA = P; g.lda = d.nr;
    g.B = Vk; g.sB = nc2; g.ldb = d.nc; g.opB = 0;
    g.C = Wk; g.sC = P; g.ldc = d.nr;
    g.M = d.nr; g.N = d.nc; g.K = d.nc;
    UCK(gemm(g, gs, st));
  } else {
    UCK(launch_r2c3(d, 3 * B, F, G4, (float)(1.0 / mu), Wk, 1, u->tb.tw3, st, gs));
  }
  const float t = (float)(alpha / mu);
  UCK(launch_group_ms2(d, (int)ns, Wk, d.h, u->ms2, st));
  JacOpt o;
  o.warm = warm;
  o.t_svt = t;
  o.ms2 = u->ms2;
  o.group = d.h;
  o.sched = (u->flags & LRSTV_FLAG_JACOBI_PER_SLICE) ? nullptr : u->jsched;
  o.pw = (u->flags & LRSTV_FLAG_JACOBI_PANEL16) ? 16 : 32;
  o.sort = (u->flags & LRSTV_FLAG_JACOBI_FIXED_ORDER) ? 0 : 1;
  UCK(launch_jacobi(d, (int)ns, Wk, Vk, -1.0f, kMaxSweeps, u->sweeps + (size_t)k * ns, nullptr,
                    st, o));
  UCK(launch_sigma_scale(d, (int)ns, Wk, Vk, t, sk, u->Hs, st));
  return LRSTV_OK;
}

int unroll_forward(lrstv_unroll *u, cudaStream_t st) {
  const Dims &d = u->d;
  const int B = u->B;
  const size_t N = d.N, ns = (size_t)3 * B * d.h;
  const GemmSel gs = unroll_gemm(u);
  for (int k = 0; k < u->K; ++k) {
    const double *th = u->theta + 4 * k;
    const double tau = th[kTau], alpha = th[kAlpha], lam = th[kLam], mu = th[kMu];
    float *src = u->slots + (size_t)k * u->slot_floats;
    float *dst = src + u->slot_floats;
    UCK(cudaMemcpyAsync(dst, src, sizeof(float) * u->slot_floats, cudaMemcpyDeviceToDevice, st));
    const UnrollSlot s = slot_at(u, dst);
    const float muf = (float)mu;
    // L and T_z, then Z (all cubes in one launch each)
    UCK(launch_l_tz(d, u->Y, s.S, s.Z, s.G1, s.G2, s.F, s.G3, muf, u->w, s.L, u->T, st, B));
    UCK(zsolve_core(d, B, u->tb, u->T, muf, s.Z, u->specA, u->specB, st, nullptr, gs));
    // F, S and Gamma1..3
    const float thr_f = (float)(tau / mu), thr_s = (float)(lam / mu);
    UCK(launch_fs_dual(d, u->Y, s.L, s.Z, s.S, s.G1, s.G2, s.F, s.E, s.G3, s.G4, muf, thr_f, thr_s,
                       u->w, nullptr, st, 0, B));
    // E: t-SVT of F - Gamma4/mu for all 3 B gradient cubes
    UCK(e_factor(u, k, s.F, s.G4, mu, alpha, st));
    float2 *Wk = w_slot(u, k);
    CGemm g{};
    g.A = Wk; g.sA = (long long)d.P; g.lda = d.nr;
    g.B = u->Hs; g.sB = (long long)d.nc * d.nc; g.ldb = d.nc; g.opB = 1;
    g.C = u->specB; g.sC = (long long)d.P; g.ldc = d.nr;
    g.M = d.nr; g.N = d.nc; g.K = d.nc; g.batch = (int)ns;
    UCK(gemm(g, gs, st));
    UCK(launch_c2r3(d, 3 * B, u->specB, 1, u->tb.tw3, s.E, 1, s.G4, s.F, muf, 1, st, gs));
  }
  return LRSTV_OK;
}

int unroll_backward(lrstv_unroll *u, double *dtheta, cudaStream_t st) {
  const Dims &d = u->d;
  const int B = u->B;
  const size_t BN = (size_t)B * d.N, ns = (size_t)3 * B * d.h;
  const GemmSel gs = unroll_gemm(u);
  const Geo geo{d.n1, d.n2, d.n3, d.N, d.P};
  const UnrollSlot a = slot_at(u, u->adj);
  const unsigned g1 = grid_for(BN);
  for (int k = u->K - 1; k >= 0; --k) {
    const double *th = u->theta + 4 * k;
    const double tau = th[kTau], alpha = th[kAlpha], lam = th[kLam], mu = th[kMu];
    const float muf = (float)mu;
    const UnrollSlot o = slot_k(u, k), n = slot_k(u, k + 1);
    AdjPtrs p;
    p.Y = u->Y;
    p.oS = o.S; p.oG1 = o.G1; p.oG2 = o.G2; p.oF = o.F; p.oE = o.E; p.oG3 = o.G3; p.oG4 = o.G4;
    p.nL = n.L; p.nZ = n.Z; p.nS = n.S; p.nF = n.F; p.nE = n.E;
    p.aY = u->aY; p.aL = a.L; p.aZ = a.Z; p.aS = a.S; p.aG1 = a.G1; p.aG2 = a.G2;
    p.aF = a.F; p.aE = a.E; p.aG3 = a.G3; p.aG4 = a.G4;
    p.X3 = u->X3; p.bT = u->bT;
    p.dth = dtheta + 4 * k;
    const double m2 = mu * mu;
    Lin ls{};  // d/dmu and d/dlambda of the S step and the multipliers
    ls.m[kMu][0] = 1.0; ls.m[kMu][1] = lam / m2; ls.m[kMu][2] = -1.0 / m2;
    ls.m[kLam][1] = -1.0 / mu;
    k_adj_sdual<<<g1, kT, 0, st>>>(geo, B, p, muf, (float)(lam / mu), u->w[0], u->w[1], u->w[2],
                                   ls);
    UCK(cudaGetLastError());
    // t-SVT adjoint of the three gradient tensors of every cube
    if (u->nw < u->K) {
      // recompute iteration k's factors from its checkpoints: the new F
      // (slot k + 1) and the Gamma4 the iteration started from (slot k)
      const int rc = e_factor(u, k, n.F, o.G4, mu, alpha, st);
      if (rc != LRSTV_OK) return rc;
    }
    float2 *Wk = w_slot(u, k);
    float2 *Vk = v_slot(u, k);
    const double *sk = sig_slot(u, k);
    UCK(launch_r2c3(d, 3 * B, a.E, nullptr, 0.0f, u->specA, 1, u->tb.tw3, st, gs));
    CGemm g{};
    g.batch = (int)ns;
    // P = G V
    g.A = u->specA; g.sA = (long long)d.P; g.lda = d.nr;
    g.B = Vk; g.sB = (long long)d.nc * d.nc; g.ldb = d.nc; g.opB = 0;
    g.C = u->specB; g.sC = (long long)d.P; g.ldc = d.nr;
    g.M = d.nr; g.N = d.nc; g.K = d.nc;
    UCK(gemm(g, kSimt, st));
    // Hraw = W^H P
    g.A = Wk; g.sA = (long long)d.P; g.lda = d.nr; g.opA = 1;
    g.B = u->specB; g.sB = (long long)d.P; g.ldb = d.nr; g.opB = 0;
    g.C = u->Hs; g.sC = (long long)d.nc * d.nc; g.ldc = d.nc;
    g.M = d.nc; g.N = d.nc; g.K = d.nr;
    UCK(gemm(g, kSimt, st));
    const float t = (float)(alpha / mu);
    Lin le{};  // the threshold t = alpha / mu, summed over the n3 slices of the full spectrum
    le.m[kAlpha][0] = 1.0 / (d.n3 * mu);
    le.m[kMu][0] = -alpha / (d.n3 * m2);
    k_svt_coef<<<(unsigned)ns, kT, 0, st>>>(d.nr, d.nc, d.h, d.n3, d.P, u->Hs, u->specB, sk, t,
                                           le, p.dth);
    UCK(cudaGetLastError());
    // X = P diag q + W K'
    g.A = Wk; g.sA = (long long)d.P; g.lda = d.nr; g.opA = 0;
    g.B = u->Hs; g.sB = (long long)d.nc * d.nc; g.ldb = d.nc; g.opB = 0;
    g.C = u->specB; g.sC = (long long)d.P; g.ldc = d.nr; g.epi = 2;
    g.M = d.nr; g.N = d.nc; g.K = d.nc;
    UCK(gemm(g, kSimt, st));
    // dA = X V^H
    g.A = u->specB; g.sA = (long long)d.P; g.lda = d.nr;
    g.B = Vk; g.sB = (long long)d.nc * d.nc; g.ldb = d.nc; g.opB = 1;
    g.C = u->specA; g.sC = (long long)d.P; g.ldc = d.nr; g.epi = 0;
    UCK(gemm(g, kSimt, st));
    UCK(launch_c2r3(d, 3 * B, u->specA, 1, u->tb.tw3, u->X3, 0, nullptr, nullptr, 0.0f, 0, st, gs));
    Lin lf{};  // the F threshold tau / mu and B = F - Gamma4 / mu
    lf.m[kMu][0] = 1.0 / m2; lf.m[kMu][1] = tau / m2; lf.m[kMu][2] = -0.5 / m2;
    lf.m[kTau][1] = -1.0 / mu;
    k_adj_f<<<g1, kT, 0, st>>>(geo, B, p, muf, (float)(tau / mu), u->w[0], u->w[1], u->w[2], lf);
    UCK(cudaGetLastError());
    Lin lz{};  // Z = T / mu in the spectral domain
    lz.m[kMu][0] = -1.0 / mu;
    k_adj_dz<<<g1, kT, 0, st>>>(geo, B, p, u->w[0], u->w[1], u->w[2], lz);
    UCK(cudaGetLastError());
    UCK(zsolve_core(d, B, u->tb, a.Z, muf, u->bT, u->specA, u->specB, st, nullptr, gs));
    Lin ll{};  // T_z and the L-update
    ll.m[kMu][0] = 1.0; ll.m[kMu][1] = -0.5 / m2;
    k_adj_l<<<g1, kT, 0, st>>>(geo, B, p, muf, u->w[0], u->w[1], u->w[2], ll);
    UCK(cudaGetLastError());
  }
  return LRSTV_OK;
}

void unroll_free(lrstv_unroll *u) {
  if (!u) return;
  if (u->arena) cudaFree(u->arena);
  free(u->theta);
  delete u;
}

}  // namespace

extern "C" {

int lrstv_unroll_create(int n1, int n2, int n3, int batch, int iters, const float w[3],
                        unsigned flags, lrstv_unroll **out) {
  if (!out) return LRSTV_ERR_ARG;
  *out = nullptr;
  int rc = check_shape(n1, n2, n3);
  if (rc) return rc;
  if (batch < 1 || iters < 1 || iters > 4096) return LRSTV_ERR_ARG;
  if (flags & ~(unsigned)(LRSTV_FLAG_SIMT_GEMM | LRSTV_FLAG_WARM_START | LRSTV_FLAG_SIMT_DFT |
                          LRSTV_FLAG_JACOBI_PER_SLICE | LRSTV_FLAG_JACOBI_PANEL16 |
                          LRSTV_FLAG_JACOBI_FIXED_ORDER | LRSTV_FLAG_UNROLL_RECOMPUTE))
    return LRSTV_ERR_ARG;
  float wl[3] = {1.0f, 1.0f, 1.0f};
  if (w)
    for (int n = 0; n < 3; ++n) {
      if (!isfinite(w[n]) || w[n] < 0.0f) return LRSTV_ERR_ARG;
      wl[n] = w[n];
    }
  lrstv_unroll *u = new (std::nothrow) lrstv_unroll();
  if (!u) return LRSTV_ERR_ALLOC;
  u->d = make_dims(n1, n2, n3);
  u->B = batch;
  u->K = iters;
  memcpy(u->w, wl, sizeof(wl));
  u->flags = flags;
  u->slot_floats = 17 * (size_t)batch * u->d.N;
  const bool recompute = (flags & LRSTV_FLAG_UNROLL_RECOMPUTE) != 0;
  u->nw = recompute ? 1 : iters;
  u->nv = recompute && !(flags & LRSTV_FLAG_WARM_START) ? 1 : iters;
  u->theta = (double *)calloc(4 * (size_t)iters, sizeof(double));
  if (!u->theta) {
    unroll_free(u);
    return LRSTV_ERR_ALLOC;
  }
  u->arena_bytes = unroll_layout(u, nullptr);
  if (cudaMalloc(&u->arena, u->arena_bytes) != cudaSuccess) {
    cudaGetLastError();
    u->arena = nullptr;
    unroll_free(u);
    return LRSTV_ERR_ALLOC;
  }
  unroll_layout(u, u->arena);
  const Tables &t = u->tb;
  if (cudaMemset(u->gemm_err, 0, sizeof(int)) != cudaSuccess ||
      launch_tables(u->d, u->w, t.tw3, t.F1, t.G1, t.F2, t.G2, t.lam1, t.lam2, t.lam3, 0) !=
          cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    unroll_free(u);
    return LRSTV_ERR_CUDA;
  }
  *out = u;
  return LRSTV_OK;
}

int lrstv_unroll_destroy(lrstv_unroll *u) {
  if (!u) return LRSTV_ERR_ARG;
  cudaDeviceSynchronize();
  unroll_free(u);
  return LRSTV_OK;
}

int lrstv_unroll_bytes(const lrstv_unroll *u, size_t *bytes) {
  if (!u || !bytes) return LRSTV_ERR_ARG;
  *bytes = u->arena_bytes;
  return LRSTV_OK;
}

int lrstv_unroll_forward(lrstv_unroll *u, const float *Y, const double *theta, float *X,
                         void *stream) {
  if (!u || !Y || !theta) return LRSTV_ERR_ARG;
  for (int k = 0; k < u->K; ++k) {
    const double *th = theta + 4 * k;
    for (int i = 0; i < 4; ++i)
      if (!isfinite(th[i]) || th[i] < 0.0) return LRSTV_ERR_ARG;
    if (!(th[kMu] > 0.0)) return LRSTV_ERR_ARG;
  }
  memcpy(u->theta, theta, sizeof(double) * 4 * (size_t)u->K);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t BN = (size_t)u->B * u->d.N;
  // initial state: L = Z = Y, everything else zero
  const UnrollSlot s0 = slot_k(u, 0);
  UCK(cudaMemcpyAsync(u->Y, Y, sizeof(float) * BN, cudaMemcpyDeviceToDevice, st));
  UCK(cudaMemsetAsync(u->slots, 0, sizeof(float) * u->slot_floats, st));
  UCK(cudaMemcpyAsync(s0.L, Y, sizeof(float) * BN, cudaMemcpyDeviceToDevice, st));
  UCK(cudaMemcpyAsync(s0.Z, Y, sizeof(float) * BN, cudaMemcpyDeviceToDevice, st));
  u->have_forward = 0;
  int rc = unroll_forward(u, st);
  if (rc != LRSTV_OK) return rc;
  if (X) UCK(cudaMemcpyAsync(X, slot_k(u, u->K).L, sizeof(float) * BN, cudaMemcpyDeviceToDevice, st));
  u->have_forward = 1;
  return LRSTV_OK;
}

int lrstv_unroll_backward(lrstv_unroll *u, const float *dX, double *dtheta, float *dY,
                          void *stream) {
  if (!u || !dX || !dtheta) return LRSTV_ERR_ARG;
  if (!u->have_forward) return LRSTV_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t BN = (size_t)u->B * u->d.N;
  const UnrollSlot a = slot_at(u, u->adj);
  UCK(cudaMemsetAsync(u->adj, 0, sizeof(float) * u->slot_floats, st));
  UCK(cudaMemsetAsync(u->aY, 0, sizeof(float) * BN, st));
  UCK(cudaMemcpyAsync(a.L, dX, sizeof(float) * BN, cudaMemcpyDeviceToDevice, st));
  UCK(cudaMemsetAsync(dtheta, 0, sizeof(double) * 4 * (size_t)u->K, st));
  int rc = unroll_backward(u, dtheta, st);
  if (rc != LRSTV_OK) return rc;
  if (dY) {
    // the initial state is L = Z = Y
    k_sum3<<<grid_for(BN), kT, 0, st>>>(BN, u->aY, a.Z, a.L, dY);
    UCK(cudaGetLastError());
  }
  return LRSTV_OK;
}

int lrstv_unroll_stats(lrstv_unroll *u, int *unconverged, int *gemm_errors, void *stream) {
  if (!u) return LRSTV_ERR_ARG;
  UCK(cudaStreamSynchronize((cudaStream_t)stream));
  const size_t n = (size_t)u->K * 3 * u->B * u->d.h;
  int *h = (int *)malloc(sizeof(int) * n);
  if (!h) return LRSTV_ERR_ALLOC;
  int bad = 0, gerr = 0;
  if (cudaMemcpy(h, u->sweeps, sizeof(int) * n, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&gerr, u->gemm_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    free(h);
    cudaGetLastError();
    return LRSTV_ERR_CUDA;
  }
  for (size_t i = 0; i < n; ++i) bad += h[i] < 0;
  free(h);
  if (unconverged) *unconverged = bad;
  if (gemm_errors) *gemm_errors = gerr;
  return LRSTV_OK;
}

}  // extern "C"
