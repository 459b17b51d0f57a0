// svt.cu -- singular value thresholding of the Fourier frontal slices in the
// t-SVT of the E-update (arXiv 2204.12879, eq. E_solution; the slice-wise
// form follows Theorem 4.2's t-SVD).
//
// Each slice's working matrix W (nr x nc complex, nr >= nc) is orthogonalised
// by one-sided (Hestenes) Jacobi: column pairs (p, q) are rotated until
// |w_p^H w_q| <= tol |w_p| |w_q|.  The rotations accumulate in V, so W = A V
// has orthogonal columns sigma_i u_i and SVT_t(A) = W diag(g) V^H with
// g_i = max(1 - t / sigma_i, 0) (a negative t leaves V unscaled, so that the
// factors W and V of the SVD itself are kept).  U is never formed; the reconstruction
// W (V diag g)^H is a batched complex GEMM (dft.cu).  One CTA per slice; the
// sweep loop is capped and a slice that reaches the cap reports it.
//
// Two kernels share the rotation formula and differ in how columns move:
//  - k_jacobi_pk (nr <= 256, the common case): 32-column panels staged in
//    shared memory, a panel's W and V columns held in registers while later
//    panels stream past, one column pair per half-warp, paired FP32
//    instructions (__ffma2_rn) on a split row-pair layout;
//  - k_jacobi (any nr up to 512): round-robin over all columns in global
//    memory (L2-resident), one pair per warp.
#include <float.h>

#include "lrstv_internal.cuh"

namespace lrstv {

// fewer slices than resident CTAs (defined with the launchers below)
bool tasks_pay(int nslices, int nr, int pw);

namespace {

__device__ __forceinline__ void pair_of(int r, int i, int np, int &p, int &q) {
  if (i == 0) {
    p = r;
    q = np - 1;
  } else {
    p = (r + i) % (np - 1);
    q = (r - i + np - 1) % (np - 1);
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int R>
__global__ void __launch_bounds__(R <= 8 ? 1024 : 512)
    k_jacobi(int nr, int nc, size_t wstride, size_t vstride, float2 *W_all, float2 *V_all,
             float t, int max_sweeps, float tol, float negl_rel, int *__restrict__ sweeps_out,
             unsigned long long *__restrict__ work, JacOpt o) {
  const int warm = o.warm;
  const float skip_t = o.t_svt;
  const float gms2 = o.ms2 ? o.ms2[blockIdx.x / o.group] : -1.0f;
  float2 *W = W_all + (size_t)blockIdx.x * wstride;
  float2 *V = V_all + (size_t)blockIdx.x * vstride;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  __shared__ float s_red[32];
  __shared__ int s_rot;

  if (!warm)  // warm: V holds the basis W was multiplied by
    for (int e = tid; e < nc * nc; e += blockDim.x)
      V[e] = make_float2((e % nc) == (e / nc) ? 1.0f : 0.0f, 0.0f);

  // ||W||_F^2: columns whose squared norm is below negl_rel ||W||_F^2 are
  // rounding residue and take part in no rotation.
  float part = 0.0f;
  for (size_t e = tid; e < (size_t)nr * nc; e += blockDim.x) {
    const float2 x = W[e];
    part = fmaf(x.x, x.x, fmaf(x.y, x.y, part));
  }
  part = warp_sum(part);
  if (lane == 0) s_red[warp] = part;
  __syncthreads();
  if (warp == 0) {
    float v = lane < nwarps ? s_red[lane] : 0.0f;
    v = warp_sum(v);
    if (lane == 0) s_red[0] = v;
  }
  __syncthreads();
  const float negl = negl_rel * s_red[0];

  const int np = nc + (nc & 1);
  unsigned long long n_pairs = 0, n_rot = 0;  // counted by lane 0 of each warp
  // a slice with fewer than two columns is diagonal already: one empty sweep
  int sweeps = (nc < 2) ? 1 : 0;
  bool converged = (nc < 2);
  // every singular value is at most ||W||_F: at or below the threshold the SVT
  // is zero whatever the sweeps would find, so none is run
  if (skip_t >= 0.0f && s_red[0] <= skip_t * skip_t) {
    sweeps = 0;
    converged = true;
  }
  // A pair left with relative inner product g moves the SVT result by at most
  // about t g (both values kept: t g s_p / (s_p + s_q); one kept: g s_cut <= t g;
  // both cut: nothing), so with the threshold t below the columns' RMS norm the
  // relative tolerance is raised to tol rms / t: the absolute error stays at
  // the level tol rms that a threshold near the RMS norm already allows.  The
  // RMS norm is the largest over the slices of one tensor when it is given
  // (ms2): the inverse DFT mixes the slices, so all of them are resolved to
  // the same absolute precision.
  if (skip_t > 0.0f && nc > 0) {
    const float ms2 = gms2 >= 0.0f ? gms2 : s_red[0] / (float)nc;
    tol = fmaxf(tol, tol * (sqrtf(ms2) / skip_t));
  }
  for (int sweep = 1; sweep <= max_sweeps && !converged; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int r = 0; r < np - 1; ++r) {
      for (int pr = warp; pr < np / 2; pr += nwarps) {
        int p, q;
        pair_of(r, pr, np, p, q);
        if (p >= nc || q >= nc) continue;
        n_pairs += 1;
        float2 *wp = W + (size_t)nr * p, *wq = W + (size_t)nr * q;
        float2 a[R], b[R];
        float al = 0.f, be = 0.f, gr = 0.f, gi = 0.f;
#pragma unroll
        for (int k = 0; k < R; ++k) {
          const int row = lane + 32 * k;
          if (row < nr) {
            a[k] = wp[row];
            b[k] = wq[row];
          } else {
            a[k] = make_float2(0.f, 0.f);
            b[k] = make_float2(0.f, 0.f);
          }
          al = fmaf(a[k].x, a[k].x, fmaf(a[k].y, a[k].y, al));
          be = fmaf(b[k].x, b[k].x, fmaf(b[k].y, b[k].y, be));
          // conj(a) * b
          gr = fmaf(a[k].x, b[k].x, fmaf(a[k].y, b[k].y, gr));
          gi = fmaf(a[k].x, b[k].y, fmaf(-a[k].y, b[k].x, gi));
        }
        al = warp_sum(al);
        be = warp_sum(be);
        gr = warp_sum(gr);
        gi = warp_sum(gi);
        const float ag = hypotf(gr, gi);
        if (!(al > negl && be > negl)) continue;
        if (!(ag > tol * sqrtf(al) * sqrtf(be))) continue;
        // 2x2 Hermitian [[al, g], [conj g, be]]: remove the phase of g, then
        // the real symmetric Schur rotation tan = sign(z) / (|z| + sqrt(1+z^2)).
        const float zeta = (be - al) / (2.0f * ag);
        const float az = fabsf(zeta);
        const float tn = (az > 1e18f ? 0.5f / az : 1.0f / (az + sqrtf(fmaf(az, az, 1.0f))));
        const float tt = zeta >= 0.0f ? tn : -tn;
        const float c = 1.0f / sqrtf(fmaf(tt, tt, 1.0f));
        const float s = c * tt;
        const float er = gr / ag, ei = -gi / ag;  // conj(g) / |g|
#pragma unroll
        for (int k = 0; k < R; ++k) {
          const int row = lane + 32 * k;
          if (row < nr) {
            const float2 bb = make_float2(er * b[k].x - ei * b[k].y, er * b[k].y + ei * b[k].x);
            wp[row] = make_float2(c * a[k].x - s * bb.x, c * a[k].y - s * bb.y);
            wq[row] = make_float2(s * a[k].x + c * bb.x, s * a[k].y + c * bb.y);
          }
        }
        float2 *vp = V + (size_t)nc * p, *vq = V + (size_t)nc * q;
#pragma unroll
        for (int k = 0; k < R; ++k) {
          const int row = lane + 32 * k;
          if (row < nc) {
            const float2 x = vp[row], y = vq[row];
            const float2 yy = make_float2(er * y.x - ei * y.y, er * y.y + ei * y.x);
            vp[row] = make_float2(c * x.x - s * yy.x, c * x.y - s * yy.y);
            vq[row] = make_float2(s * x.x + c * yy.x, s * x.y + c * yy.y);
          }
        }
        n_rot += 1;
        if (lane == 0) s_rot = 1;
      }
      __syncthreads();
    }
    sweeps = sweep;
    converged = (s_rot == 0);
    __syncthreads();
  }

  // g_i = max(1 - t / sigma_i, 0); the sigma-vs-t decision is taken in FP64.
  for (int i = warp; i < nc; i += nwarps) {
    const float2 *wi = W + (size_t)nr * i;
    float n2 = 0.f;
    for (int row = lane; row < nr; row += 32) n2 = fmaf(wi[row].x, wi[row].x, fmaf(wi[row].y, wi[row].y, n2));
    n2 = warp_sum(n2);
    const double sigma = sqrt((double)n2);
    const float g = t < 0.0f ? 1.0f : (sigma > (double)t ? (float)(1.0 - (double)t / sigma) : 0.0f);
    float2 *vi = V + (size_t)nc * i;
    for (int row = lane; row < nc; row += 32) vi[row] = make_float2(vi[row].x * g, vi[row].y * g);
  }
  if (tid == 0) sweeps_out[blockIdx.x] = converged ? sweeps : -max_sweeps;
  if (work && lane == 0) {
    atomicAdd(work + 0, n_pairs);
    atomicAdd(work + 1, n_rot);
  }
}

// ---------------------------------------------------------------------------
// Shared pieces of the packed kernel: panel width, rotation formula.
// Panel width (columns) of the packed kernels: 32 with 16-warp CTAs, or 16
// with 8-warp CTAs, two of which share an SM (a warp per pair of columns of
// a panel: PW / 2 warps, PW half-warps).
constexpr int kPW = 32;

struct Rot {
  float c, s, er, ei;
  float d;  // |a'|^2 = |a|^2 - d and |b'|^2 = |b|^2 + d (d = t |g|, the 2x2 Schur rotation's shift)
};

// Rotation of the 2x2 Hermitian [[al, g], [conj g, be]], or false when the
// pair is orthogonal to tolerance or a column is negligible.
// 1/sqrt(x) to about an ulp: the MUFU estimate refined by one Newton step.
__device__ __forceinline__ float rsqrt_nr(float x) {
  const float y = rsqrtf(x);
  return y * fmaf(-0.5f * x * y, y, 1.5f);
}

// Rotation of the 2x2 Hermitian [[al, g], [conj g, be]], or false when the
// pair is orthogonal to tolerance (|g|^2 <= tol^2 al be) or a column is
// negligible.  Unitarity rests on c = 1/sqrt(1 + t^2), s = c t and |e| = 1,
// which take the Newton-refined reciprocal square root; the angle itself
// (zeta, t) may carry a few ulps of error without affecting unitarity.
__device__ __forceinline__ bool make_rot(float al, float be, float gr, float gi, float tol,
                                         float negl, Rot &r) {
  if (!(al > negl && be > negl)) return false;
  const float g2 = fmaf(gr, gr, gi * gi);
  if (!(g2 > (tol * tol) * (al * be))) return false;
  const float inv_ag = rsqrt_nr(g2);
  const float zeta = 0.5f * (be - al) * inv_ag;
  const float az = fabsf(zeta);
  const float q = fmaf(az, az, 1.0f);
  const float tn = az > 1e18f ? __fdividef(0.5f, az) : __fdividef(1.0f, az + q * rsqrtf(q));
  const float tt = zeta >= 0.0f ? tn : -tn;
  r.c = rsqrt_nr(fmaf(tt, tt, 1.0f));
  r.s = r.c * tt;
  r.er = gr * inv_ag;
  r.ei = -gi * inv_ag;
  r.d = tt * (g2 * inv_ag);
  return true;
}


constexpr int kHW = kPW / 2;  // warps per CTA of the 32-column packed kernel

__device__ __forceinline__ float half_sum(float v) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// Packed kernel (nr <= 224): the half-warp panel scheme with Blackwell's
// paired FP32 instructions (__ffma2_rn / __fmul2_rn: two FP32 FMAs per lane
// per instruction).  Staged columns use a split row-pair layout: row pair m is
// one float4 (re_2m, re_2m+1, im_2m, im_2m+1), so a 128-bit load gives the two
// packed operands (re, re) and (im, im) directly and complex arithmetic needs
// no register shuffles: a dot-product step costs 4 paired instructions per two
// rows and a rotation 12 (against 16 and 24 scalar FMAs).  Panel a's W columns
// live in registers (one per half-warp); V columns of panel a and of the
// streamed panel b stay in shared memory.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 dup(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 lo2(const float4 &v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4 &v) { return make_float2(v.z, v.w); }

// A rotation as broadcast pairs: a' = c a - (s e) b, b' = s a + (c e) b.
struct PRot {
  float2 C, S, NSEX, SEY, NSEY, CEX, CEY, NCEY;
};

__device__ __forceinline__ PRot packed(const Rot &r) {
  const float sex = r.s * r.er, sey = r.s * r.ei, cex = r.c * r.er, cey = r.c * r.ei;
  PRot q;
  q.C = dup(r.c);
  q.S = dup(r.s);
  q.NSEX = dup(-sex);
  q.SEY = dup(sey);
  q.NSEY = dup(-sey);
  q.CEX = dup(cex);
  q.CEY = dup(cey);
  q.NCEY = dup(-cey);
  return q;
}

__device__ __forceinline__ void pk_rot(float4 &a, float4 &b, const PRot &q) {
  const float2 Ra = lo2(a), Ia = hi2(a), Rb = lo2(b), Ib = hi2(b);
  const float2 aR = fma2(q.SEY, Ib, fma2(q.NSEX, Rb, mul2(q.C, Ra)));
  const float2 aI = fma2(q.NSEY, Rb, fma2(q.NSEX, Ib, mul2(q.C, Ia)));
  const float2 bR = fma2(q.NCEY, Ib, fma2(q.CEX, Rb, mul2(q.S, Ra)));
  const float2 bI = fma2(q.CEY, Rb, fma2(q.CEX, Ib, mul2(q.S, Ia)));
  a = make_float4(aR.x, aR.y, aI.x, aI.y);
  b = make_float4(bR.x, bR.y, bI.x, bI.y);
}

// lane partial sums of |a|^2, |b|^2, re(a^H b), im(a^H b) over K row pairs,
// in two interleaved chains (even / odd k) to halve the dependent FMA depth
template <int K>
__device__ __forceinline__ void pk_dots(const float4 (&a)[K], const float4 (&b)[K], float &al,
                                        float &be, float &gr, float &gi) {
  const float2 z = make_float2(0.f, 0.f);
  float2 aa[2] = {z, z}, bb[2] = {z, z}, rr[2] = {z, z}, i1[2] = {z, z}, i2[2] = {z, z};
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int c = k & 1;
    const float2 Ra = lo2(a[k]), Ia = hi2(a[k]), Rb = lo2(b[k]), Ib = hi2(b[k]);
    aa[c] = fma2(Ia, Ia, fma2(Ra, Ra, aa[c]));
    bb[c] = fma2(Ib, Ib, fma2(Rb, Rb, bb[c]));
    rr[c] = fma2(Ia, Ib, fma2(Ra, Rb, rr[c]));
    i1[c] = fma2(Ra, Ib, i1[c]);
    i2[c] = fma2(Ia, Rb, i2[c]);
  }
  al = (aa[0].x + aa[1].x) + (aa[0].y + aa[1].y);
  be = (bb[0].x + bb[1].x) + (bb[0].y + bb[1].y);
  gr = (rr[0].x + rr[1].x) + (rr[0].y + rr[1].y);
  gi = ((i1[0].x + i1[1].x) + (i1[0].y + i1[1].y)) - ((i2[0].x + i2[1].x) + (i2[0].y + i2[1].y));
}

// lane partial sums of re(a^H b), im(a^H b) only (pk_dots without the norms,
// in the same order, so the inner product is bit-identical to pk_dots')
template <int K>
__device__ __forceinline__ void pk_cross(const float4 (&a)[K], const float4 (&b)[K], float &gr,
                                         float &gi) {
  const float2 z = make_float2(0.f, 0.f);
  float2 rr[2] = {z, z}, i1[2] = {z, z}, i2[2] = {z, z};
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int c = k & 1;
    const float2 Ra = lo2(a[k]), Ia = hi2(a[k]), Rb = lo2(b[k]), Ib = hi2(b[k]);
    rr[c] = fma2(Ia, Ib, fma2(Ra, Rb, rr[c]));
    i1[c] = fma2(Ra, Ib, i1[c]);
    i2[c] = fma2(Ia, Rb, i2[c]);
  }
  gr = (rr[0].x + rr[1].x) + (rr[0].y + rr[1].y);
  gi = ((i1[0].x + i1[1].x) + (i1[0].y + i1[1].y)) - ((i2[0].x + i2[1].x) + (i2[0].y + i2[1].y));
}

// lane partial sum of |a|^2 over K row pairs
template <int K>
__device__ __forceinline__ float pk_norm(const float4 (&a)[K]) {
  const float2 z = make_float2(0.f, 0.f);
  float2 aa[2] = {z, z};
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int c = k & 1;
    const float2 Ra = lo2(a[k]), Ia = hi2(a[k]);
    aa[c] = fma2(Ia, Ia, fma2(Ra, Ra, aa[c]));
  }
  return (aa[0].x + aa[1].x) + (aa[0].y + aa[1].y);
}

// A tracked squared norm that fell below this fraction of its value before
// the rotation is marked for recomputation from the column itself (when the
// column is next read): the update |a|^2 - d cancels there, and its absolute
// rounding (about eps |a|^2) would become a large relative error.
constexpr float kNormDrop = 0.0625f;

// rotates two shared-memory columns (row-pair layout), lane stride `step`
template <int K, int STEP>
__device__ __forceinline__ void pk_rot_smem(float4 *ca, float4 *cb, const PRot &q, int l) {
#pragma unroll
  for (int k = 0; k < K; k += 2) {
    float4 x0 = ca[l + STEP * k], y0 = cb[l + STEP * k];
    float4 x1, y1;
    if (k + 1 < K) {
      x1 = ca[l + STEP * (k + 1)];
      y1 = cb[l + STEP * (k + 1)];
    }
    pk_rot(x0, y0, q);
    ca[l + STEP * k] = x0;
    cb[l + STEP * k] = y0;
    if (k + 1 < K) {
      pk_rot(x1, y1, q);
      ca[l + STEP * (k + 1)] = x1;
      cb[l + STEP * (k + 1)] = y1;
    }
  }
}

// rotates the register column a against shared-memory column col (row-pair
// layout, half-warp lane stride), two row pairs at a time
template <int K>
__device__ __forceinline__ void pk_rot_stream(float4 (&a)[K], float4 *col, const PRot &q, int ul) {
  // loads run one row pair ahead of the rotate-and-store
  float4 y = col[ul];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    float4 ynext;
    if (k + 1 < K) ynext = col[ul + 16 * (k + 1)];
    pk_rot(a[k], y, q);
    col[ul + 16 * k] = y;
    if (k + 1 < K) y = ynext;
  }
}

// Loads of W and V that another SM may have written during the same launch
// (the task-graph schedule below) bypass L1, which is not coherent across SMs.
template <bool CG>
__device__ __forceinline__ float2 ldw(const float2 *p) {
  return CG ? __ldcg(p) : *p;
}

// Staging of panels into shared memory: a shared panel holds ld2 row pairs
// per column in the split layout, zero padded, of wcols columns of n rows;
// warp w copies columns w, w + PW / 2.  A lane's row pairs of one column:
// ld2 <= kStageIt * 32 for every packed shape (PkShape: at most 128).
constexpr int kStageIt = 4;

// One column of n rows into registers (the lane's row pairs m = lane + 32 it,
// zeros past n or for a padding column), and from there into a shared panel
// column in the split row-pair layout, returning the lane's part of its
// squared norm.
template <bool CG>
__device__ __forceinline__ void col_load(float2 (&x0)[kStageIt], float2 (&x1)[kStageIt],
                                         const float2 *s, int n, int ld2, bool real) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int it = 0; it < kStageIt; ++it) {
    const int m = lane + 32 * it, r0 = 2 * m, r1 = 2 * m + 1;
    x0[it] = (real && m < ld2 && r0 < n) ? ldw<CG>(s + r0) : make_float2(0.f, 0.f);
    x1[it] = (real && m < ld2 && r1 < n) ? ldw<CG>(s + r1) : make_float2(0.f, 0.f);
  }
}

__device__ __forceinline__ float col_store(float4 *d, const float2 (&x0)[kStageIt],
                                           const float2 (&x1)[kStageIt], int ld2) {
  const int lane = threadIdx.x & 31;
  float part = 0.0f;
#pragma unroll
  for (int it = 0; it < kStageIt; ++it) {
    const int m = lane + 32 * it;
    if (m < ld2) {
      d[m] = make_float4(x0[it].x, x1[it].x, x0[it].y, x1[it].y);
      part = fmaf(x0[it].x, x0[it].x,
                  fmaf(x0[it].y, x0[it].y, fmaf(x1[it].x, x1[it].x, fmaf(x1[it].y, x1[it].y, part))));
    }
  }
  return part;
}

// A panel's W (nr rows, squared column norms into nrm) and V (nc rows)
// staged together: a warp issues the loads of its W and V columns (NCOL of
// each) before its first shared store, so that 16 NCOL loads a lane are in
// flight.  NCOL = 2 holds 32 float2 a lane, for stagings with no register
// panel live.
// With a column map (cols, shared memory: the panel's wcols column indices),
// sW and sV are the slice's first columns and panel column c is column
// cols[c]; without one the panel's columns are contiguous from sW and sV.
template <int PW, bool CG, int NCOL>
__device__ __forceinline__ void pk_stage_wv(float4 *dW, const float2 *sW, int nr, float *nrm,
                                            float4 *dV, const float2 *sV, int nc, int ld2,
                                            int wcols, const int *cols = nullptr) {
  constexpr int HW = PW / 2;
  const int lane = threadIdx.x & 31;
  for (int c0 = threadIdx.x >> 5; c0 < PW; c0 += NCOL * HW) {
    float2 w0[NCOL][kStageIt], w1[NCOL][kStageIt], v0[NCOL][kStageIt], v1[NCOL][kStageIt];
#pragma unroll
    for (int k = 0; k < NCOL; ++k) {
      const int c = c0 + k * HW;
      const bool real = c < PW && c < wcols;
      const int g = cols ? (real ? cols[c] : 0) : c;
      col_load<CG>(w0[k], w1[k], sW + (size_t)nr * g, nr, ld2, real);
      col_load<CG>(v0[k], v1[k], sV + (size_t)nc * g, nc, ld2, real);
    }
#pragma unroll
    for (int k = 0; k < NCOL; ++k) {
      const int c = c0 + k * HW;
      if (c >= PW) break;
      const float part = warp_sum(col_store(dW + ld2 * c, w0[k], w1[k], ld2));
      if (lane == 0) nrm[c] = part;
      col_store(dV + ld2 * c, v0[k], v1[k], ld2);
    }
  }
}

template <int PW>
__device__ __forceinline__ void pk_stage_out(float2 *dst, const float4 *src, int ld2, int n,
                                             int wcols, const int *cols = nullptr) {
  const int lane = threadIdx.x & 31;
  for (int c = threadIdx.x >> 5; c < wcols; c += PW / 2) {
    float2 *d = dst + (size_t)n * (cols ? cols[c] : c);
    const float4 *s = src + ld2 * c;
    for (int m = lane; 2 * m < n; m += 32) {
      const float4 v = s[m];
      d[2 * m] = make_float2(v.x, v.z);
      if (2 * m + 1 < n) d[2 * m + 1] = make_float2(v.y, v.w);
    }
  }
}

template <int KP>
struct PkShape {
  static constexpr int KPF = (KP + 1) / 2;  // row pairs per lane, full warp
  static constexpr int LD2 = (16 * KP > 32 * KPF) ? 16 * KP : 32 * KPF;  // row pairs per column
  static_assert(LD2 <= 32 * kStageIt, "col_load covers a column in kStageIt loads a lane");
};

// This thread's share of sum |x_e|^2 over n complex values (e = thread,
// thread + blockDim.x, ...), in four chains so that four loads are in flight.
template <bool CG>
__device__ __forceinline__ float sumsq4(const float2 *x, size_t n) {
  const size_t T = blockDim.x;
  float p0 = 0.0f, p1 = 0.0f, p2 = 0.0f, p3 = 0.0f;
  size_t e = threadIdx.x;
  for (; e + 3 * T < n; e += 4 * T) {
    const float2 a = ldw<CG>(x + e), b = ldw<CG>(x + e + T), c = ldw<CG>(x + e + 2 * T),
                 d = ldw<CG>(x + e + 3 * T);
    p0 = fmaf(a.x, a.x, fmaf(a.y, a.y, p0));
    p1 = fmaf(b.x, b.x, fmaf(b.y, b.y, p1));
    p2 = fmaf(c.x, c.x, fmaf(c.y, c.y, p2));
    p3 = fmaf(d.x, d.x, fmaf(d.y, d.y, p3));
  }
  for (; e < n; e += T) {
    const float2 a = ldw<CG>(x + e);
    p0 = fmaf(a.x, a.x, fmaf(a.y, a.y, p0));
  }
  return (p0 + p1) + (p2 + p3);
}

// Per-slice set-up of a packed Jacobi run by the whole CTA: V := I unless warm
// (warm: V holds the basis W was multiplied by), then ||W||_F^2, returned to
// every thread (s_red: 32 floats of shared memory).
template <bool CG>
__device__ __forceinline__ float pk_setup(int nr, int nc, const float2 *W, float2 *V, int warm,
                                          float *s_red) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (!warm)
    for (int e = tid; e < nc * nc; e += blockDim.x)
      V[e] = make_float2((e % nc) == (e / nc) ? 1.0f : 0.0f, 0.0f);
  float part = sumsq4<CG>(W, (size_t)nr * nc);
  part = warp_sum(part);
  if (lane == 0) s_red[warp] = part;
  __syncthreads();
  if (warp == 0) {
    float v = lane < (int)(blockDim.x >> 5) ? s_red[lane] : 0.0f;
    v = warp_sum(v);
    if (lane == 0) s_red[0] = v;
  }
  __syncthreads();
  const float fro2 = s_red[0];
  __syncthreads();
  return fro2;
}

// A pair left with relative inner product g moves the SVT result by at most
// about t g (both values kept: t g s_p / (s_p + s_q); one kept: g s_cut <= t g;
// both cut: nothing), so with the threshold t below the columns' RMS norm the
// relative tolerance is raised to tol rms / t: the absolute error stays at
// the level tol rms that a threshold near the RMS norm already allows.  The
// RMS norm is the largest over the slices of one tensor when it is given
// (ms2 >= 0): the inverse DFT mixes the slices, so all of them are resolved to
// the same absolute precision.
__device__ __forceinline__ float pk_tolerance(float tol, float fro2, int nc, float skip_t,
                                              float gms2) {
  if (skip_t > 0.0f && nc > 0) {
    const float ms2 = gms2 >= 0.0f ? gms2 : fro2 / (float)nc;
    tol = fmaxf(tol, tol * (sqrtf(ms2) / skip_t));
  }
  return tol;
}

// The pairs inside one staged panel (W in sW with squared norms s_na, V in
// sVa; wa real columns): 31 rounds of 16 disjoint pairs, one per warp.
template <int KP, int PW>
__device__ __forceinline__ void pk_intra(float4 *sW, float4 *sVa, float *s_na, int wa, float tol,
                                         float negl, unsigned &n_pairs, unsigned &n_rot,
                                         int &rotated) {
  constexpr int KPF = PkShape<KP>::KPF;
  constexpr int LD2 = PkShape<KP>::LD2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = 0; r < PW - 1; ++r) {
    int p, q;
    pair_of(r, warp, PW, p, q);
    if (p < wa && q < wa) {
      float4 xa[KPF], xb[KPF];
#pragma unroll
      for (int k = 0; k < KPF; ++k) {
        xa[k] = sW[LD2 * p + lane + 32 * k];
        xb[k] = sW[LD2 * q + lane + 32 * k];
      }
      float gr, gi;
      pk_cross<KPF>(xa, xb, gr, gi);
      gr = warp_sum(gr);
      gi = warp_sum(gi);
      // a norm marked negative after a rotation that cancelled it is
      // recomputed from the column (warp-uniform: p, q are the warp's)
      float al = s_na[p], be = s_na[q];
      if (al < 0.0f) al = warp_sum(pk_norm<KPF>(xa));
      if (be < 0.0f) be = warp_sum(pk_norm<KPF>(xb));
      if (lane == 0) n_pairs += 1;
      Rot rt;
      if (make_rot(al, be, gr, gi, tol, negl, rt)) {
        const PRot pq = packed(rt);
#pragma unroll
        for (int k = 0; k < KPF; ++k) {
          pk_rot(xa[k], xb[k], pq);
          sW[LD2 * p + lane + 32 * k] = xa[k];
          sW[LD2 * q + lane + 32 * k] = xb[k];
        }
        pk_rot_smem<KPF, 32>(sVa + LD2 * p, sVa + LD2 * q, pq, lane);
        const float na = al - rt.d, nb = be + rt.d;
        if (lane == 0) {
          s_na[p] = na < kNormDrop * al ? -1.0f : na;
          s_na[q] = nb < kNormDrop * be ? -1.0f : nb;
          n_rot += 1;
        }
        rotated = 1;
      }
    }
    __syncthreads();
  }
}

// Panel a's columns (one per half-warp, `unit`; W in aW, V in aV, both in
// registers; mine = the column is real) against the streamed panel b (W in
// sW with squared norms s_nb, V in sVb; wb real columns): 16 double rounds in
// which warp w owns streamed columns 2c, 2c+1 (c = (w + R) mod 16) and its
// half-warps rotate them in swapped order, so only the warp synchronises
// between the two sub-steps and the block once per double round.
template <int KP, int PW>
__device__ __forceinline__ void pk_cross_pass(float4 (&aW)[KP], float4 (&aV)[KP], bool mine,
                                              float4 *sW, float4 *sVb, float *s_nb, int wb,
                                              float tol, float negl, unsigned &n_pairs,
                                              unsigned &n_rot, int &rotated,
                                              float *al_out = nullptr) {
  constexpr int LD2 = PkShape<KP>::LD2;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int unit = tid >> 4, ul = tid & 15;
  float4 bW[KP];
  // the register column's squared norm, exact at the start of each streamed
  // panel (the whole warp shuffles: both halves compute theirs)
  float al_reg = half_sum(pk_norm<KP>(aW));
  __syncthreads();
  for (int r = 0; r < PW; ++r) {
    const int sub = r & 1;
    const int cpi = (warp + (r >> 1)) & (PW / 2 - 1);
    const int j = 2 * cpi + ((unit & 1) ^ sub);
    const bool real = mine && j < wb;
#pragma unroll
    for (int k = 0; k < KP; ++k) bW[k] = sW[LD2 * j + ul + 16 * k];
    float gr, gi;
    pk_cross<KP>(aW, bW, gr, gi);
    gr = half_sum(gr);
    gi = half_sum(gi);
    // norms marked negative after a rotation that cancelled them are
    // recomputed here, where both columns are in registers; the decision is
    // made per warp so that both halves take part in the shuffles
    float be = s_nb[j];
    if (__any_sync(0xffffffffu, be < 0.0f || al_reg < 0.0f)) {
      const float xa = half_sum(pk_norm<KP>(aW));
      const float xb = half_sum(pk_norm<KP>(bW));
      if (al_reg < 0.0f) al_reg = xa;
      if (be < 0.0f) be = xb;
    }
    Rot rt;
    const bool go = real && make_rot(al_reg, be, gr, gi, tol, negl, rt);
    if (ul == 0 && real) n_pairs += 1;
    if (__any_sync(0xffffffffu, go)) {
      // the other half-warp may rotate: this half applies the identity, which
      // rewrites its columns unchanged
      if (!go) {
        rt.c = 1.0f;
        rt.s = 0.0f;
        rt.er = 1.0f;
        rt.ei = 0.0f;
        rt.d = 0.0f;
      }
      const PRot pq = packed(rt);
#pragma unroll
      for (int k = 0; k < KP; ++k) {
        pk_rot(aW[k], bW[k], pq);
        sW[LD2 * j + ul + 16 * k] = bW[k];
      }
      pk_rot_stream<KP>(aV, sVb + LD2 * j, pq, ul);
      if (go) {
        const float na = al_reg - rt.d, nb = be + rt.d;
        al_reg = na < kNormDrop * al_reg ? -1.0f : na;
        if (ul == 0) {
          s_nb[j] = nb < kNormDrop * be ? -1.0f : nb;
          n_rot += 1;
        }
        rotated = 1;
      }
    }
    if (sub == 0)
      __syncwarp();
    else
      __syncthreads();
  }
  if (al_out) *al_out = al_reg;
}

// Panel a's W column `unit` of the staged panel moves to registers, with its V.
template <int KP>
__device__ __forceinline__ void pk_to_registers(const float4 *sW, const float4 *sVa,
                                                float4 (&aW)[KP], float4 (&aV)[KP]) {
  constexpr int LD2 = PkShape<KP>::LD2;
  const int unit = threadIdx.x >> 4, ul = threadIdx.x & 15;
#pragma unroll
  for (int k = 0; k < KP; ++k) {
    aW[k] = sW[LD2 * unit + ul + 16 * k];
    aV[k] = sVa[LD2 * unit + ul + 16 * k];
  }
}

// Panel a back to global memory from the registers (W) and, through sVa, V.
template <int KP, int PW>
__device__ __forceinline__ void pk_from_registers(const float4 (&aW)[KP], const float4 (&aV)[KP],
                                                  bool mine, float4 *sVa, float2 *Wa,
                                                  float2 *Va, int nr, int nc, int wa,
                                                  const int *cols = nullptr) {
  constexpr int LD2 = PkShape<KP>::LD2;
  const int unit = threadIdx.x >> 4, ul = threadIdx.x & 15;
#pragma unroll
  for (int k = 0; k < KP; ++k) sVa[LD2 * unit + ul + 16 * k] = aV[k];
  __syncthreads();
  if (mine) {
    float2 *wcol = Wa + (size_t)nr * (cols ? cols[unit] : unit);
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      const int m = ul + 16 * k;
      if (2 * m < nr) wcol[2 * m] = make_float2(aW[k].x, aW[k].z);
      if (2 * m + 1 < nr) wcol[2 * m + 1] = make_float2(aW[k].y, aW[k].w);
    }
  }
  pk_stage_out<PW>(Va, sVa, LD2, nc, wa, cols);
}

// g_i = max(1 - t / sigma_i, 0) applied to V's columns (t < 0: V unscaled),
// sigma_i = |w_i|; the sigma-vs-t decision is taken in FP64.
template <bool CG>
__device__ __forceinline__ void pk_epilogue(int nr, int nc, const float2 *W, float2 *V, float t) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (t < 0.0f) return;
  for (int i = warp; i < nc; i += (int)(blockDim.x >> 5)) {
    const float2 *wi = W + (size_t)nr * i;
    float n2 = 0.f;
    for (int row = lane; row < nr; row += 32) {
      const float2 x = ldw<CG>(wi + row);
      n2 = fmaf(x.x, x.x, fmaf(x.y, x.y, n2));
    }
    n2 = warp_sum(n2);
    const double sigma = sqrt((double)n2);
    const float g = sigma > (double)t ? (float)(1.0 - (double)t / sigma) : 0.0f;
    float2 *vi = V + (size_t)nc * i;
    for (int row = lane; row < nc; row += 32) {
      const float2 v = ldw<CG>(vi + row);
      vi[row] = make_float2(v.x * g, v.y * g);
    }
  }
}

// Columns of a slice of the packed kernels at most (nc <= nr <= 256).
constexpr int kSortCols = 256;

// Squared norms of a slice's nc columns of nr <= 256 rows into key (shared
// memory), by the whole CTA: two columns a warp at a time, every lane's loads
// of both issued together.  W was written by an earlier launch.
__device__ void col_norms(int nr, int nc, const float2 *W, float *key) {
  const int lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  for (int c = threadIdx.x >> 5; c < nc; c += 2 * nwarp) {
    const int c2 = c + nwarp;
    const float2 *w0 = W + (size_t)nr * c, *w1 = W + (size_t)nr * (c2 < nc ? c2 : c);
    float2 x[8], y[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int r = lane + 32 * k;
      x[k] = r < nr ? w0[r] : make_float2(0.f, 0.f);
      y[k] = r < nr ? w1[r] : make_float2(0.f, 0.f);
    }
    float a = 0.f, b = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      a = fmaf(x[k].x, x[k].x, fmaf(x[k].y, x[k].y, a));
      b = fmaf(y[k].x, y[k].x, fmaf(y[k].y, y[k].y, b));
    }
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) {
      key[c] = a;
      if (c2 < nc) key[c2] = b;
    }
  }
}

// The order of a slice's columns for its next sweep, by the whole CTA: by
// decreasing squared norm, ties by index (the norm-sorted ordering that de
// Rijk proposed for one-sided Jacobi, 1989: sweeps that pair the large
// columns first converge in fewer sweeps).  key: nc squared norms in shared
// memory (a NaN or a negative value sorts as 0); perm[rank] = column.  The
// ranks are counted, not sorted, so ties and the result are deterministic.
__device__ void order_columns(int nc, float *key, int *perm) {
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    const float v = key[i];
    key[i] = v > 0.0f ? v : 0.0f;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    const float ki = key[i];
    int rank = 0;
    for (int j = 0; j < nc; ++j) {
      const float kj = key[j];
      rank += (kj > ki) || (kj == ki && j < i);
    }
    perm[rank] = i;
  }
}

// The packed Jacobi SVT of one slice by the whole CTA (kHW warps): W (nr x nc)
// and V (nc x nc) in global memory, `smem` the CTA's dynamic shared memory
// (3 kPW LD2 float4).  Panel by panel: panel a's own pairs, then panel a (in
// registers) against every later panel b streamed through shared memory.
// Writes the sweep count (negative at the cap) to *sweeps_slot.  Shared by the
// one-slice-per-CTA kernel and the persistent batch kernel, so both compute
// bit-identical results.
template <int KP, int PW>
__device__ __forceinline__ void jacobi_pk_slice(int nr, int nc, float2 *W, float2 *V, float t,
                                                int max_sweeps, float tol, float negl_rel,
                                                int *sweeps_slot, unsigned long long *work,
                                                float4 *smem, int warm, float skip_t,
                                                float gms2, bool preconv = false,
                                                bool sort = false) {
  constexpr int LD2 = PkShape<KP>::LD2;
  float4 *sW = smem;              // panel a (own pairs), then panel b: W
  float4 *sVa = sW + PW * LD2;    // panel a: V
  float4 *sVb = sVa + PW * LD2;   // panel b: V
  const int tid = threadIdx.x, ul = tid & 15, unit = tid >> 4;
  __shared__ float s_red[32];
  __shared__ int s_rot;
  // squared column norms of panel a and of the streamed panel b: exact when
  // a panel is staged, then carried through each rotation by the 2x2 update
  // (|a|^2 - d, |b|^2 + d), so that a pair's test needs only its inner product
  __shared__ float s_na[PW], s_nb[PW];
  // with `sort`: the sweep's column order (position -> column; panel a holds
  // positions a PW ...) and each column's squared norm as the sweep left it
  __shared__ int s_perm[kSortCols];
  __shared__ float s_key[kSortCols];

  const float fro2 = pk_setup<false>(nr, nc, W, V, warm, s_red);
  const float negl = negl_rel * fro2;
  const int npan = (nc + PW - 1) / PW;
  unsigned n_pairs = 0, n_rot = 0;  // lane 0 (own pairs) and ul 0 (cross pairs) count
  int sweeps = (nc < 2) ? 1 : 0;
  bool converged = (nc < 2);
  // every singular value is at most ||W||_F: at or below the threshold the SVT
  // is zero whatever the sweeps would find, so none is run
  if (skip_t >= 0.0f && fro2 <= skip_t * skip_t) {
    sweeps = 0;
    converged = true;
  }
  // the tensor-core Gram check showed that a sweep would rotate no pair: the
  // one sweep it would take changes nothing
  if (!converged && preconv) {
    sweeps = 1;
    converged = true;
  }
  tol = pk_tolerance(tol, fro2, nc, skip_t, gms2);
  float4 aW[KP], aV[KP];
  if (!converged) {  // the first sweep's order: by the columns' norms, or as stored
    if (sort) {
      col_norms(nr, nc, W, s_key);
      __syncthreads();
      order_columns(nc, s_key, s_perm);
    } else {
      for (int c = tid; c < nc; c += blockDim.x) s_perm[c] = c;
    }
  }
  for (int sweep = 1; sweep <= max_sweeps && !converged; ++sweep) {
    if (tid == 0) s_rot = 0;
    int rotated = 0;
    for (int a = 0; a < npan; ++a) {
      const int ca = a * PW, wa = min(PW, nc - ca);
      const int *cola = s_perm + ca;  // panel a: positions ca ... of the sweep's order
      __syncthreads();
      pk_stage_wv<PW, false, 2>(sW, W, nr, s_na, sVa, V, nc, LD2, wa, cola);
      __syncthreads();
      pk_intra<KP, PW>(sW, sVa, s_na, wa, tol, negl, n_pairs, n_rot, rotated);
      if (sort && tid < wa) s_key[cola[tid]] = s_na[tid];
      const bool mine = unit < wa;
      pk_to_registers<KP>(sW, sVa, aW, aV);
      for (int b = a + 1; b < npan; ++b) {
        const int cb = b * PW, wb = min(PW, nc - cb);
        const int *colb = s_perm + cb;
        __syncthreads();
        pk_stage_wv<PW, false, 1>(sW, W, nr, s_nb, sVb, V, nc, LD2, wb, colb);
        float al = 0.0f;
        pk_cross_pass<KP, PW>(aW, aV, mine, sW, sVb, s_nb, wb, tol, negl, n_pairs, n_rot, rotated,
                              &al);
        if (sort) {
          if (mine && ul == 0) s_key[cola[unit]] = al;
          if (tid < wb) s_key[colb[tid]] = s_nb[tid];
        }
        pk_stage_out<PW>(W, sW, LD2, nr, wb, colb);
        pk_stage_out<PW>(V, sVb, LD2, nc, wb, colb);
      }
      pk_from_registers<KP, PW>(aW, aV, mine, sVa, W, V, nr, nc, wa, cola);
    }
    if (rotated) s_rot = 1;
    __syncthreads();
    sweeps = sweep;
    converged = (s_rot == 0);
    // the next sweep's order, from the norms this one left
    if (sort && !converged) order_columns(nc, s_key, s_perm);
    __syncthreads();
  }
  pk_epilogue<false>(nr, nc, W, V, t);
  if (tid == 0) *sweeps_slot = converged ? sweeps : -max_sweeps;
  if (work && ul == 0) {
    atomicAdd(work + 0, (unsigned long long)n_pairs);
    atomicAdd(work + 1, (unsigned long long)n_rot);
  }
}

// Slices of up to 64 rows fit in 64 registers a thread, and 16-column panels
// take 8-warp CTAs: two CTAs share an SM.
template <int KP, int PW>
__global__ void __launch_bounds__(PW * 16, (KP <= 2 || PW == 16) ? 2 : 1)
    k_jacobi_pk(int nr, int nc, size_t wstride, size_t vstride, float2 *W_all, float2 *V_all,
                float t, int max_sweeps, float tol, float negl_rel, int *__restrict__ sweeps_out,
                unsigned long long *__restrict__ work, JacOpt o, const int *__restrict__ order) {
  extern __shared__ float4 smem_f4[];
  // CTAs start in launch order: with `order`, the slices that took the most
  // sweeps in the previous E-step come first
  const int s = order ? order[blockIdx.x] : (int)blockIdx.x;
  jacobi_pk_slice<KP, PW>(nr, nc, W_all + (size_t)s * wstride, V_all + (size_t)s * vstride, t,
                          max_sweeps, tol, negl_rel, sweeps_out + s, work, smem_f4, o.warm,
                          o.t_svt, o.ms2 ? o.ms2[s / o.group] : -1.0f,
                          o.conv ? o.conv[s] != 0 : false, o.sort != 0);
}

// order[0..n) = the slices by the sweeps |sweeps[s]| of their previous run,
// most first, equal counts in slice order (a stable counting sort by one
// CTA; counts above 63 share the first bucket).
__global__ void __launch_bounds__(1024) k_slice_order(const int *__restrict__ sweeps, int n,
                                                      int *__restrict__ order) {
  __shared__ int s_cnt[64], s_start[64];
  const int tid = threadIdx.x;
  if (tid < 64) s_cnt[tid] = 0;
  __syncthreads();
  auto key = [&](int i) {
    const int a = abs(sweeps[i]);
    return 63 - (a < 63 ? a : 63);  // bucket 0: the most sweeps
  };
  for (int i = tid; i < n; i += blockDim.x) atomicAdd(&s_cnt[key(i)], 1);
  __syncthreads();
  if (tid == 0) {
    int run = 0;
    for (int k = 0; k < 64; ++k) {
      s_start[k] = run;
      run += s_cnt[k];
    }
  }
  __syncthreads();
  // stable placement: warp 0 walks the slices in order, a 32-slice chunk at
  // a time, ranking each lane within its bucket by the lanes before it
  if (tid < 32) {
    for (int base = 0; base < n; base += 32) {
      const int i = base + tid;
      const int k = i < n ? key(i) : -1;
      int rank = 0;
      for (int j = 0; j < 32; ++j) {
        const int kj = __shfl_sync(0xffffffffu, k, j);
        if (j < tid && kj == k) ++rank;
      }
      if (i < n) order[s_start[k] + rank] = i;
      __syncwarp();
      for (int j = 0; j < 32; ++j) {
        const int kj = __shfl_sync(0xffffffffu, k, j);
        if (tid == 0 && kj >= 0) s_start[kj] += 1;
      }
      __syncwarp();
    }
  }
}

// ---------------------------------------------------------------------------
// Task-graph schedule of the packed Jacobi (nr <= 256).  In a sweep the
// column panels of a slice are paired by a round-robin tournament (pair_of
// over P + 1 players for an odd number P of panels, P + 2 for an even one,
// the extra players being empty): in each round a slice's pairs are disjoint,
// a panel paired with an empty player runs its own pairs, and every pair of
// panels meets once per sweep, so every column pair is still visited once per
// sweep.  Each (slice, round, pair) is a task: one cross pass (pk_cross_pass)
// or one panel's own pairs (pk_intra), with the panels read from and written
// back to global memory.  A persistent grid takes tasks from a queue in global
// memory; the task that completes a slice's round queues the slice's next
// round (or, at the end of a sweep, ends the slice when no pair rotated, or at
// the cap), so slices advance independently and every SM works on whichever
// slice has work: at 200 x 200 x 80 the 123 slices' work spreads over all 152
// SMs, and slices that converge early leave their share to the others.  The
// rotation formula, tolerances and convergence test are the one-CTA-per-slice
// kernel's; the order of the pairs within a sweep differs.
//
// Scratch (ints, zeroed by the host before each launch; jacobi_task_ints):
// [0] queue head, [1] queue tail, [2] finished slices, [3] error flag;
// per slice: sweep, round in progress, tasks left in the round,
// rotated-in-this-sweep; per slice (floats): tolerance, negligible squared
// norm; the queue: cap 64-bit slots, each a task (its slice, round and pair)
// and the mark of its position (slot i's mark is i + 1); per slice,
// kSortCols ints (the column order of its current sweep: panel p holds the
// columns at positions p PW ...) and kSortCols floats (each column's squared
// norm as the last task that rotated it left it).
constexpr unsigned long long kTaskWaitNs = 2000000000ull;  // a wait for work gives up after 2 s

__device__ __forceinline__ int ld_relaxed(const int *p) { return *(const volatile int *)p; }

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// The rounds of one sweep.  An odd number of panels plays a round-robin
// tournament with one empty player (npan + 1 players, npan rounds): the panel
// paired with it runs its own pairs.  An even number first runs every
// panel's own pairs in one round (round 0), then the npan - 1 rounds of the
// tournament among the panels themselves.
__device__ __forceinline__ int tour_players(int npan) { return npan + (npan & 1); }
__device__ __forceinline__ int tour_rounds(int npan) { return npan; }
// pair i of round r: panels p, q (q >= npan: p's own pairs); false if empty
__device__ __forceinline__ bool tour_pair(int npan, int r, int i, int &p, int &q) {
  if (!(npan & 1)) {
    if (r == 0) {
      p = i;
      q = npan;  // own pairs
      return i < npan;
    }
    r -= 1;
  }
  const int np = tour_players(npan);
  if (i >= np / 2) return false;
  pair_of(r, i, np, p, q);
  if (p >= npan) {
    const int x = p;
    p = q;
    q = x;
  }
  return p < npan;
}
// tasks per round at most: npan (even npan, round 0) or (npan + 1) / 2
__device__ __forceinline__ int tour_width(int npan) { return (npan & 1) ? (npan + 1) / 2 : npan; }
// task ids per slice: tour_width of 512 columns in 16-column panels (32);
// rounds of a sweep: tour_rounds of up to 32 panels
constexpr int kTaskIds = 32;
constexpr int kTaskRounds = 32;

__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long *p) {
  return *(const volatile unsigned long long *)p;
}

struct TaskView {
  int *head, *tail, *finished, *err;
  int *sweep, *round, *left, *rot;
  float *tol, *negl;
  // the queue: slot i holds (mark << 32) | task, the mark of the i-th task
  // queued being i + 1, written in one 64-bit exchange so that a reader sees
  // the task and its mark together
  unsigned long long *qslot;
  int *perm;     // per slice, kSortCols: position -> column
  float *norm;   // per slice, kSortCols: column -> squared norm
  int cap;
  __device__ TaskView(int *sched, int ns, int cap_) : cap(cap_) {
    head = sched;
    tail = sched + 1;
    finished = sched + 2;
    err = sched + 3;
    sweep = sched + 4;
    round = sweep + ns;
    left = round + ns;
    rot = left + ns;
    tol = (float *)(rot + ns);
    negl = tol + ns;
    qslot = (unsigned long long *)(negl + ns);  // 4 + 6 ns ints before it: 8-byte aligned
    perm = (int *)(qslot + cap);
    norm = (float *)(perm + (size_t)kSortCols * ns);
  }
  // queues the tasks of round r of slice s (one thread); a task is
  // (s kTaskRounds + r) kTaskIds + its pair index in the round
  __device__ void push_round(int s, int r, int npan) {
    int ids[kTaskIds], c = 0;
    for (int i = 0; i < tour_width(npan); ++i) {
      int p, q;
      if (tour_pair(npan, r, i, p, q)) ids[c++] = i;
    }
    round[s] = r;
    left[s] = c;
    __threadfence();
    for (int k = 0; k < c; ++k) {
      const int idx = atomicAdd(tail, 1);
      const unsigned task = (unsigned)((s * kTaskRounds + r) * kTaskIds + ids[k]);
      atomicExch(qslot + (idx & (cap - 1)),
                 ((unsigned long long)(unsigned)(idx + 1) << 32) | task);
    }
  }
};

// Set-up of the task-graph run, one CTA per slice: V := I unless warm,
// ||W||_F^2, the slice's tolerance and negligible squared norm; a slice whose
// singular values are all cut (||W||_F <= t) ends here with 0 sweeps, the
// others queue their first round.
__global__ void __launch_bounds__(kHW * 32)
    k_jacobi_task_setup(int nr, int nc, int nslices, size_t wstride, size_t vstride,
                        float2 *W_all, float2 *V_all, float t, int max_sweeps, float tol0,
                        float negl_rel, int *__restrict__ sweeps_out, JacOpt o, int *sched,
                        int cap, int pw) {
  __shared__ float s_red[32];
  __shared__ float s_key[kSortCols];
  const int s = blockIdx.x;
  TaskView tv(sched, nslices, cap);
  float2 *W = W_all + (size_t)s * wstride, *V = V_all + (size_t)s * vstride;
  const float fro2 = pk_setup<false>(nr, nc, W, V, o.warm, s_red);
  const float skip_t = o.t_svt;
  const bool cut = skip_t >= 0.0f && fro2 <= skip_t * skip_t;
  // the tensor-core Gram check showed that a sweep would rotate no pair
  const bool pre = !cut && o.conv && o.conv[s];
  if (cut || pre) pk_epilogue<false>(nr, nc, W, V, t);  // cut: every g_i is 0 (t >= 0), or V is kept
  // the first sweep's column order: by the columns' squared norms, or as stored
  int *perm = tv.perm + (size_t)kSortCols * s;
  if (!(cut || pre)) {
    if (o.sort) {
      col_norms(nr, nc, W, s_key);
      __syncthreads();
      order_columns(nc, s_key, perm);
    } else {
      for (int c = threadIdx.x; c < nc; c += blockDim.x) perm[c] = c;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    tv.tol[s] = pk_tolerance(tol0, fro2, nc, skip_t, o.ms2 ? o.ms2[s / o.group] : -1.0f);
    tv.negl[s] = negl_rel * fro2;
    tv.sweep[s] = 0;
    tv.rot[s] = 0;
    if (cut || pre) {
      sweeps_out[s] = cut ? 0 : 1;
      __threadfence();
      atomicAdd(tv.finished, 1);
    } else {
      sweeps_out[s] = -max_sweeps;  // until the slice ends: a run that stops early reports it
      tv.push_round(s, 0, (nc + pw - 1) / pw);
    }
  }
}

// The persistent worker grid: every CTA takes tasks until every slice has
// ended (or a wait for work runs out, after kTaskWaitNs; the slices still
// open then stay reported as capped).
template <int KP, int PW>
__global__ void __launch_bounds__(PW * 16, (KP <= 2 || PW == 16) ? 2 : 1)
    k_jacobi_tasks(int nr, int nc, int nslices, size_t wstride, size_t vstride, float2 *W_all,
                   float2 *V_all, float t, int max_sweeps, int *__restrict__ sweeps_out,
                   unsigned long long *__restrict__ work, int *sched, int cap, int sort) {
  extern __shared__ float4 smem_f4[];
  constexpr int LD2 = PkShape<KP>::LD2;
  float4 *sW = smem_f4, *sVa = sW + PW * LD2, *sVb = sVa + PW * LD2;
  __shared__ float s_na[PW], s_nb[PW];
  __shared__ int s_cola[PW], s_colb[PW];  // the panels' columns (the sweep's column order)
  __shared__ int s_task, s_last, s_end, s_next;
  const int tid = threadIdx.x, ul = tid & 15, unit = tid >> 4;
  TaskView tv(sched, nslices, cap);
  const int npan = (nc + PW - 1) / PW, nrounds = tour_rounds(npan);
  unsigned n_pairs = 0, n_rot = 0;
  float4 aW[KP], aV[KP];
  int claim = -1;  // thread 0: a queue slot claimed ahead
  for (;;) {
    // one thread claims the next queue slot (unless it claimed it while the
    // previous task wrote its panels back) and waits (bounded) until it is
    // filled or every slice has ended
    if (tid == 0) {
      const int idx = claim >= 0 ? claim : atomicAdd(tv.head, 1);
      claim = -1;
      const int slot = idx & (cap - 1);
      const unsigned long long t0 = gtimer();
      int task = -1;
      for (;;) {
        const unsigned long long v = ld_relaxed64(tv.qslot + slot);
        if ((unsigned)(v >> 32) == (unsigned)(idx + 1)) {
          __threadfence();
          task = (int)(unsigned)v;
          break;
        }
        if (ld_relaxed(tv.finished) >= nslices) break;
        if (gtimer() - t0 > kTaskWaitNs) {
          atomicExch(tv.err, 1);
          break;
        }
        __nanosleep(128);
      }
      s_task = task;
    }
    __syncthreads();
    const int task = s_task;
    if (task < 0) break;
    const int s = task / (kTaskIds * kTaskRounds), pi = task % kTaskIds;
    const int r = (task / kTaskIds) % kTaskRounds;
    float2 *W = W_all + (size_t)s * wstride, *V = V_all + (size_t)s * vstride;
    const float tol = ((const volatile float *)tv.tol)[s];
    const float negl = ((const volatile float *)tv.negl)[s];
    int pa, pb;
    tour_pair(npan, r, pi, pa, pb);  // pa is a real panel; pb >= npan: pa's own pairs
    int rotated = 0;
    const int ca = pa * PW, wa = min(PW, nc - ca);
    const int cb = pb < npan ? pb * PW : 0, wb = pb < npan ? min(PW, nc - cb) : 0;
    // the panels' columns in this sweep's order (written by the task that
    // started the sweep, on another SM: read past L1)
    int *perm = tv.perm + (size_t)kSortCols * s;
    float *gnorm = tv.norm + (size_t)kSortCols * s;
    if (tid < wa) s_cola[tid] = __ldcg(perm + ca + tid);
    if (tid >= PW && tid - PW < wb) s_colb[tid - PW] = __ldcg(perm + cb + tid - PW);
    __syncthreads();
    pk_stage_wv<PW, true, 2>(sW, W, nr, s_na, sVa, V, nc, LD2, wa, s_cola);
    __syncthreads();
    if (pb >= npan) {  // panel pa's own pairs
      pk_intra<KP, PW>(sW, sVa, s_na, wa, tol, negl, n_pairs, n_rot, rotated);
      if (tid == 0) claim = atomicAdd(tv.head, 1);  // its latency hides behind the write-back
      if (sort && tid < wa) gnorm[s_cola[tid]] = s_na[tid];
      pk_stage_out<PW>(W, sW, LD2, nr, wa, s_cola);
      pk_stage_out<PW>(V, sVa, LD2, nc, wa, s_cola);
    } else {  // panel pa (registers) against panel pb (streamed)
      const bool mine = unit < wa;
      pk_to_registers<KP>(sW, sVa, aW, aV);
      __syncthreads();
      pk_stage_wv<PW, true, 1>(sW, W, nr, s_nb, sVb, V, nc, LD2, wb, s_colb);
      float al = 0.0f;
      pk_cross_pass<KP, PW>(aW, aV, mine, sW, sVb, s_nb, wb, tol, negl, n_pairs, n_rot, rotated,
                            &al);
      if (tid == 0) claim = atomicAdd(tv.head, 1);  // its latency hides behind the write-back
      if (sort) {
        if (mine && ul == 0) gnorm[s_cola[unit]] = al;
        if (tid < wb) gnorm[s_colb[tid]] = s_nb[tid];
      }
      pk_stage_out<PW>(W, sW, LD2, nr, wb, s_colb);
      pk_stage_out<PW>(V, sVb, LD2, nc, wb, s_colb);
      pk_from_registers<KP, PW>(aW, aV, mine, sVa, W, V, nr, nc, wa, s_cola);
    }
    // the panels are written (every thread fences its own stores); then the
    // task counts off its slice's round
    __threadfence();
    rotated = __syncthreads_or(rotated);
    if (tid == 0) {
      if (rotated) atomicOr(tv.rot + s, 1);
      __threadfence();
      s_last = atomicSub(tv.left + s, 1) == 1;
      s_end = 0;
      s_next = -1;
      if (s_last) {  // this task completed the round: queue the next, or end the slice
        __threadfence();
        int next = r + 1;
        if (next == nrounds) {  // the sweep is complete
          const int sw = ld_relaxed(tv.sweep + s) + 1;
          const int any = atomicExch(tv.rot + s, 0);
          if (!any)
            s_end = sw;  // converged: a sweep without a rotation
          else if (sw >= max_sweeps)
            s_end = -max_sweeps;
          else {
            tv.sweep[s] = sw;
            next = 0;
          }
        }
        if (!s_end) s_next = next;
      }
    }
    __syncthreads();
    if (s_next == 0 && sort) {
      // a new sweep: its column order from the norms the sweep's tasks left
      // (every one of them fenced its stores before counting off its round)
      float *key = (float *)smem_f4;
      for (int c = tid; c < nc; c += blockDim.x) key[c] = __ldcg(gnorm + c);
      __syncthreads();
      order_columns(nc, key, perm);
      __threadfence();
      __syncthreads();
    }
    if (tid == 0 && s_next >= 0) tv.push_round(s, s_next, npan);
    if (s_end) {  // the slice ended: this CTA applies its epilogue and counts it
      pk_epilogue<true>(nr, nc, W, V, t);
      __threadfence();
      __syncthreads();
      if (tid == 0) {
        sweeps_out[s] = s_end;
        __threadfence();
        atomicAdd(tv.finished, 1);
      }
    }
    __syncthreads();
  }
  if (work && ul == 0) {
    atomicAdd(work + 0, (unsigned long long)n_pairs);
    atomicAdd(work + 1, (unsigned long long)n_rot);
  }
}

// Persistent kernel for a batch of cubes: each CTA takes the next slice from
// an atomic counter (tasks sorted largest first) until the list is empty, and
// runs the same jacobi_pk_slice as the one-slice kernel on it.  Threshold and
// tolerances are formed exactly as the per-cube launch forms them, so the two
// paths agree bit for bit.
// KPMAX: the tallest slice's row pairs per lane.  Slices of 225-256 rows (KP 8)
// make the kernel spill some 380 bytes a thread, so only batches that hold
// such slices take that instance.
template <int KPMAX>
__global__ void __launch_bounds__(kHW * 32, 1)
    k_jacobi_batch(const SliceTask *__restrict__ tasks, int ntasks, int *counter, double mu,
                   int max_sweeps, unsigned long long *work, int warm, int keep, int sort) {
  extern __shared__ float4 smem_f4[];
  __shared__ int s_item;
  const float eps = FLT_EPSILON * 0.5f;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= ntasks) return;
    const SliceTask tk = tasks[item];
    const float tt = (float)((double)tk.alpha / mu);
    const float t = keep ? -1.0f : tt;
    const float tol = 8.0f * sqrtf((float)tk.nr) * eps;
    const float negl = ((float)tk.nr * eps) * ((float)tk.nr * eps);
    const int KP = (tk.nr + 31) / 32;
    if (KP <= 1)
      jacobi_pk_slice<1, kPW>(tk.nr, tk.nc, tk.W, tk.V, t, max_sweeps, tol, negl, tk.sweeps, work, smem_f4, warm, tt, tk.ms2 ? *tk.ms2 : -1.0f, tk.conv ? *tk.conv != 0 : false, sort != 0);
    else if (KP <= 2)
      jacobi_pk_slice<2, kPW>(tk.nr, tk.nc, tk.W, tk.V, t, max_sweeps, tol, negl, tk.sweeps, work, smem_f4, warm, tt, tk.ms2 ? *tk.ms2 : -1.0f, tk.conv ? *tk.conv != 0 : false, sort != 0);
    else if (KP <= 4)
      jacobi_pk_slice<4, kPW>(tk.nr, tk.nc, tk.W, tk.V, t, max_sweeps, tol, negl, tk.sweeps, work, smem_f4, warm, tt, tk.ms2 ? *tk.ms2 : -1.0f, tk.conv ? *tk.conv != 0 : false, sort != 0);
    else if (KP <= 5)
      jacobi_pk_slice<5, kPW>(tk.nr, tk.nc, tk.W, tk.V, t, max_sweeps, tol, negl, tk.sweeps, work, smem_f4, warm, tt, tk.ms2 ? *tk.ms2 : -1.0f, tk.conv ? *tk.conv != 0 : false, sort != 0);
    else if (KPMAX <= 7 || KP <= 7)
      jacobi_pk_slice<7, kPW>(tk.nr, tk.nc, tk.W, tk.V, t, max_sweeps, tol, negl, tk.sweeps, work, smem_f4, warm, tt, tk.ms2 ? *tk.ms2 : -1.0f, tk.conv ? *tk.conv != 0 : false, sort != 0);
    else
      jacobi_pk_slice<KPMAX, kPW>(tk.nr, tk.nc, tk.W, tk.V, t, max_sweeps, tol, negl, tk.sweeps, work, smem_f4, warm, tt, tk.ms2 ? *tk.ms2 : -1.0f, tk.conv ? *tk.conv != 0 : false, sort != 0);
  }
}

int task_cap(int nslices) {
  // a slot is reused only after the ring has wrapped: queued-but-untaken
  // tasks stay below one round (at most kTaskIds) per live slice and
  // claimed-but-unfilled slots below one per worker CTA, under the capacity
  int cap = 4096;
  while (cap < kTaskIds * nslices + 4096) cap <<= 1;
  return cap;
}

template <int KP, int PW>
cudaError_t launch_tasks(int nslices, int nr, int nc, size_t ws, size_t vs, float2 *W, float2 *V,
                         float t, int max_sweeps, float tol, float negl, int *sweeps,
                         unsigned long long *work, const JacOpt &o, cudaStream_t st) {
  const size_t smem = sizeof(float4) * 3 * (size_t)PW * PkShape<KP>::LD2;
  cudaError_t e = cudaFuncSetAttribute(k_jacobi_tasks<KP, PW>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int dev = 0, nsm = 0, occ = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_jacobi_tasks<KP, PW>, PW * 16,
                                                      smem);
  if (e != cudaSuccess) return e;
  const int cap = task_cap(nslices);
  const int npan = (nc + PW - 1) / PW;
  const int width = (npan & 1) ? (npan + 1) / 2 : npan;
  // workers: the resident CTAs of every SM but the spare ones, and no more
  // than the tasks a round offers
  const int per_sm = occ > 0 ? occ : 1;
  long long grid = (long long)per_sm * (nsm - (o.spare_sms < nsm ? o.spare_sms : 0));
  const long long most = (long long)nslices * width;
  if (grid > most) grid = most;
  if (grid < 1) grid = 1;
  e = cudaMemsetAsync(o.sched, 0, sizeof(int) * jacobi_task_ints(nslices), st);
  if (e != cudaSuccess) return e;
  k_jacobi_task_setup<<<nslices, kHW * 32, 0, st>>>(nr, nc, nslices, ws, vs, W, V, t, max_sweeps,
                                                     tol, negl, sweeps, o, o.sched, cap, PW);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_jacobi_tasks<KP, PW><<<(unsigned)grid, PW * 16, smem, st>>>(nr, nc, nslices, ws, vs, W, V, t,
                                                                  max_sweeps, sweeps, work,
                                                                  o.sched, cap, o.sort ? 1 : 0);
  return cudaGetLastError();
}

template <int KP, int PW>
cudaError_t launch_pk(int nslices, int nr, int nc, size_t ws, size_t vs, float2 *W, float2 *V,
                      float t, int max_sweeps, float tol, float negl, int *sweeps,
                      unsigned long long *work, const JacOpt &o, cudaStream_t st) {
  const size_t smem = sizeof(float4) * 3 * (size_t)PW * PkShape<KP>::LD2;
  cudaError_t e = cudaFuncSetAttribute(k_jacobi_pk<KP, PW>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // the order matters only when the slices take more than one wave of CTAs
  const int *order = (o.order && !tasks_pay(nslices, nr, PW)) ? o.order : nullptr;
  if (order) {
    k_slice_order<<<1, 1024, 0, st>>>(sweeps, nslices, o.order);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  k_jacobi_pk<KP, PW><<<nslices, PW * 16, smem, st>>>(nr, nc, ws, vs, W, V, t, max_sweeps, tol,
                                                      negl, sweeps, work, o, order);
  return cudaGetLastError();
}

// the packed kernel of a slice height (KP row pairs per lane) and panel width
template <int PW>
cudaError_t launch_packed(bool tasks, int nslices, int nr, int nc, size_t ws, size_t vs,
                          float2 *W, float2 *V, float t, int max_sweeps, float tol, float negl,
                          int *sweeps, unsigned long long *work, const JacOpt &o,
                          cudaStream_t st) {
  const int KP = (nr + 31) / 32;
#define LRSTV_PK(K)                                                                            \
  return tasks ? launch_tasks<K, PW>(nslices, nr, nc, ws, vs, W, V, t, max_sweeps, tol, negl,  \
                                     sweeps, work, o, st)                                      \
               : launch_pk<K, PW>(nslices, nr, nc, ws, vs, W, V, t, max_sweeps, tol, negl,     \
                                  sweeps, work, o, st)
  if (KP <= 1) LRSTV_PK(1);
  if (KP <= 2) LRSTV_PK(2);
  if (KP <= 4) LRSTV_PK(4);
  if (KP <= 5) LRSTV_PK(5);  // 129-160 rows (the 145-pixel Indian Pines shape)
  if (KP <= 7) LRSTV_PK(7);
  LRSTV_PK(8);
#undef LRSTV_PK
}

// sigma_i = |w_i| and V_s = V diag(g), g = max(1 - t / sigma, 0), with the same
// arithmetic and summation order as the Jacobi kernels' epilogue (so a Jacobi
// run with t < 0 followed by this kernel equals a run with threshold t).
__global__ void __launch_bounds__(512)
    k_sigma_scale(int nr, int nc, size_t wstride, const float2 *__restrict__ W,
                  const float2 *__restrict__ V, float t, double *__restrict__ sig,
                  float2 *__restrict__ Vs) {
  // slice blockIdx.x, one column a warp: blockIdx.y takes columns
  // blockDim.x / 32 blockIdx.y .. + blockDim.x / 32 - 1
  const int s = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  const float2 *Ws = W + (size_t)s * wstride;
  const size_t vs = (size_t)nc * nc;
  const int i = blockIdx.y * nwarps + warp;
  if (i < nc) {
    const float2 *wi = Ws + (size_t)nr * i;
    float n2 = 0.f;
#pragma unroll 4
    for (int row = lane; row < nr; row += 32)
      n2 = fmaf(wi[row].x, wi[row].x, fmaf(wi[row].y, wi[row].y, n2));
    n2 = warp_sum(n2);
    const double sigma = sqrt((double)n2);
    const float g = sigma > (double)t ? (float)(1.0 - (double)t / sigma) : 0.0f;
    if (sig && lane == 0) sig[(size_t)s * nc + i] = sigma;
    const float2 *vi = V + s * vs + (size_t)nc * i;
    float2 *oi = Vs + s * vs + (size_t)nc * i;
#pragma unroll 4
    for (int row = lane; row < nc; row += 32) oi[row] = make_float2(vi[row].x * g, vi[row].y * g);
  }
}

// Mean-square column norm ||W_s||_F^2 / nc of every slice, reduced to the
// largest over each group of `group` consecutive slices (atomic max on the
// bits of non-negative floats; the group slots start at zero).
__global__ void __launch_bounds__(1024)
    k_group_ms2(int nr, int nc, size_t wstride, const float2 *__restrict__ W, int group,
                unsigned *__restrict__ gmax) {
  __shared__ float s_red[32];
  const float2 *Ws = W + (size_t)blockIdx.x * wstride;
  float part = sumsq4<false>(Ws, (size_t)nr * nc);
  part = warp_sum(part);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    float v = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += s_red[w];
    atomicMax(gmax + blockIdx.x / group, __float_as_uint(v / (float)nc));
  }
}

// cand[s] = 1 when slice s's previous Jacobi run took one sweep (not none:
// a slice whose singular values were all cut, or that has not run yet, is
// left to the Jacobi's own cheap all-cut test or to its sweeps).
__global__ void k_gram_gate(const int *__restrict__ sweeps, int n, int *__restrict__ cand) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) cand[s] = sweeps[s] == 1 ? 1 : 0;
}

// conv[s] for the Gram matrix G_s (nc x nc, column-major) of a candidate slice:
// 1 when every pair p < q passes |G_pq| <= (tol (1 - 1e-3) - kappa) sqrt(G_pp G_qq).
// The sweep rotates a pair when |g|^2 > tol^2 |w_p|^2 |w_q|^2 with g its own FP32
// inner product; G_pq carries at most about (nr eps + 2^-20) |w_p| |w_q| of
// rounding (3xTF32 products, FP32 sums) and g about nr eps |w_p| |w_q|, so
// kappa = 4 nr eps + 4e-6 keeps every passing pair below the sweep's test, and
// the (1 - 1e-3) covers the sweep's own squared norms and this test's FP32
// squares.  tol: the Jacobi's threshold-aware tolerance (pk_tolerance with the
// tensor's ms2).  One CTA a slice.
__global__ void __launch_bounds__(256)
    k_gram_check(const float2 *__restrict__ G, int nr, int nc, const int *__restrict__ cand,
                 float tol0, float skip_t, const float *__restrict__ ms2, int group,
                 int *__restrict__ conv) {
  const int s = blockIdx.x;
  if (!cand[s]) {
    if (threadIdx.x == 0) conv[s] = 0;
    return;
  }
  const float2 *Gs = G + (size_t)s * nc * nc;
  __shared__ float s_d[512];
  __shared__ float s_red[8];
  float part = 0.0f;
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    const float di = Gs[(size_t)i * nc + i].x;
    s_d[i] = fmaxf(di, 0.0f);
    part += di;
  }
  part = warp_sum(part);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = part;
  __syncthreads();
  float fro2 = 0.0f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) fro2 += s_red[w];
  const float tol = pk_tolerance(tol0, fro2, nc, skip_t, ms2 ? ms2[s / group] : -1.0f);
  const double eps = (double)FLT_EPSILON * 0.5;
  const double lim = (double)tol * (1.0 - 1e-3) - (4.0 * nr * eps + 4e-6);
  const float lim2 = (float)(lim * lim);
  int ok = lim > 0.0;
  for (size_t e = threadIdx.x; ok && e < (size_t)nc * nc; e += blockDim.x) {
    const int p = (int)(e % nc), q = (int)(e / nc);
    if (p >= q) continue;
    const float2 g = Gs[e];
    if (!(fmaf(g.x, g.x, g.y * g.y) <= lim2 * (s_d[p] * s_d[q]))) ok = 0;
  }
  ok = __syncthreads_and(ok);
  if (threadIdx.x == 0) conv[s] = ok;
}

// One Newton-Schulz step towards the nearest unitary matrix:
// V := V (3 I - V^H V) / 2 = 1.5 V - 0.5 D with D = (V V^H) V given.
__global__ void k_ns_update(int nc, int nslices, size_t dstride, float2 *__restrict__ V,
                            const float2 *__restrict__ D) {
  const size_t per = (size_t)nc * nc, total = per * nslices;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t s = e / per, r = e - s * per;
    const float2 v = V[e], d = D[s * dstride + r];
    V[e] = make_float2(1.5f * v.x - 0.5f * d.x, 1.5f * v.y - 0.5f * d.y);
  }
}

}  // namespace

cudaError_t launch_sigma_scale(const Dims &d, int nslices, const float2 *W, const float2 *V,
                               float t, double *sig, float2 *Vs, cudaStream_t st) {
  if (nslices <= 0) return cudaSuccess;
  // 16 columns a CTA: about a dozen CTAs a slice, so every SM streams
  k_sigma_scale<<<dim3(nslices, (d.nc + 15) / 16), 512, 0, st>>>(d.nr, d.nc, d.P, W, V, t, sig,
                                                                   Vs);
  return cudaGetLastError();
}

cudaError_t launch_group_ms2(const Dims &d, int nslices, const float2 *W, int group, float *ms2,
                             cudaStream_t st) {
  if (nslices <= 0) return cudaSuccess;
  const int ngroups = (nslices + group - 1) / group;
  cudaError_t e = cudaMemsetAsync(ms2, 0, sizeof(float) * ngroups, st);
  if (e != cudaSuccess) return e;
  k_group_ms2<<<nslices, 1024, 0, st>>>(d.nr, d.nc, d.P, W, group, (unsigned *)ms2);
  return cudaGetLastError();
}

float jacobi_tol0(int nr) { return 8.0f * sqrtf((float)nr) * (FLT_EPSILON * 0.5f); }

cudaError_t launch_gram_check(const Dims &d, int nslices, const float2 *W, float2 *G,
                              const int *sweeps, int *cand, int *conv, float t_svt,
                              const float *ms2, int group, int *gemm_err, cudaStream_t st) {
  if (nslices <= 0) return cudaSuccess;
  if (d.nc > 512) return cudaErrorInvalidValue;  // s_d holds the diagonal
  k_gram_gate<<<(nslices + 255) / 256, 256, 0, st>>>(sweeps, nslices, cand);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  CGemm g{};
  g.A = W; g.sA = (long long)d.P; g.lda = d.nr; g.opA = 1;
  g.B = W; g.sB = (long long)d.P; g.ldb = d.nr; g.opB = 0;
  g.C = G; g.sC = (long long)d.nc * d.nc; g.ldc = d.nc;
  g.M = d.nc; g.N = d.nc; g.K = d.nr; g.batch = nslices;
  g.gate = cand;
  if ((e = launch_cgemm_tc(g, gemm_err, st, 0)) != cudaSuccess) return e;
  k_gram_check<<<nslices, 256, 0, st>>>(G, d.nr, d.nc, cand, jacobi_tol0(d.nr), t_svt, ms2, group,
                                        conv);
  return cudaGetLastError();
}

cudaError_t launch_ns_update(int nc, int nslices, size_t dstride, float2 *V, const float2 *D,
                             cudaStream_t st) {
  const size_t total = (size_t)nc * nc * nslices;
  if (total == 0) return cudaSuccess;
  size_t blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_ns_update<<<(unsigned)blocks, 256, 0, st>>>(nc, nslices, dstride, V, D);
  return cudaGetLastError();
}

// The task graph pays when one CTA per slice would leave SMs idle for a
// whole wave (fewer slices than resident CTAs): it spreads the slices' work
// over every SM.  With more slices than that the per-slice kernel keeps its
// panel in registers across the streamed panels and reads each slice's data
// fewer times, and the task graph's extra panel traffic costs more than its
// balance gains (measured at 256 x 256 x 191: 288 slices, 17.1 against 13.3 ms).
bool tasks_pay(int nslices, int nr, int pw) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const int per_sm = (nr <= 64 || pw == 16) ? 2 : 1;  // the packed kernel's CTAs per SM
  return nslices < nsm * per_sm;
}

size_t jacobi_task_ints(int nslices) {
  return 4 + 6 * (size_t)nslices + 2 * (size_t)task_cap(nslices) +
         2 * (size_t)kSortCols * nslices;
}

size_t jacobi_batch_smem(int max_nr) {
  const int KP = (max_nr + 31) / 32;
  const int LD2 = KP <= 1 ? PkShape<1>::LD2
                  : KP <= 2 ? PkShape<2>::LD2
                  : KP <= 4 ? PkShape<4>::LD2
                  : KP <= 5 ? PkShape<5>::LD2
                  : KP <= 7 ? PkShape<7>::LD2
                            : PkShape<8>::LD2;
  return sizeof(float4) * 3 * (size_t)kPW * LD2;
}

cudaError_t launch_jacobi_batch(const SliceTask *tasks, int ntasks, int *counter, double mu,
                                int max_sweeps, unsigned long long *work, int grid, size_t smem,
                                cudaStream_t st, int warm, int keep, int max_nr, int sort) {
  if (ntasks <= 0) return cudaSuccess;
  const bool tall = max_nr > 224;
  cudaError_t e = cudaFuncSetAttribute(tall ? k_jacobi_batch<8> : k_jacobi_batch<7>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (tall)
    k_jacobi_batch<8><<<grid, kHW * 32, smem, st>>>(tasks, ntasks, counter, mu, max_sweeps, work,
                                                     warm, keep, sort);
  else
    k_jacobi_batch<7><<<grid, kHW * 32, smem, st>>>(tasks, ntasks, counter, mu, max_sweeps, work,
                                                     warm, keep, sort);
  return cudaGetLastError();
}

cudaError_t launch_jacobi(const Dims &d, int nslices, float2 *W, float2 *V, float t,
                          int max_sweeps, int *sweeps, unsigned long long *work,
                          cudaStream_t st, const JacOpt &o) {
  const int nr = d.nr, nc = d.nc;
  if (nslices <= 0) return cudaSuccess;
  const int np = nc + (nc & 1);
  const int R = (nr + 31) / 32;
  int pairs = np / 2 < 1 ? 1 : np / 2;
  const int maxw = R <= 8 ? 32 : 16;
  const int nw = pairs < maxw ? pairs : maxw;
  // FP32 dot products of nr terms carry about sqrt(nr) eps relative noise;
  // pairs are rotated only above a few times that.
  const float eps = FLT_EPSILON * 0.5f;
  const float tol = jacobi_tol0(nr);
  const float negl = o.negl_rel >= 0.0f ? o.negl_rel : ((float)nr * eps) * ((float)nr * eps);
  const size_t ws = d.P, vs = (size_t)nc * nc;
  if (nr <= 256 && nc >= 2) {
    // the task graph when one CTA per slice would leave SMs idle
    const bool tasks = o.sched && tasks_pay(nslices, nr, o.pw);
    if (o.pw == 16)
      return launch_packed<16>(tasks, nslices, nr, nc, ws, vs, W, V, t, max_sweeps, tol, negl,
                               sweeps, work, o, st);
    return launch_packed<32>(tasks, nslices, nr, nc, ws, vs, W, V, t, max_sweeps, tol, negl,
                             sweeps, work, o, st);
  }
  dim3 grid(nslices), block(32 * nw);
  if (R <= 1) k_jacobi<1><<<grid, block, 0, st>>>(nr, nc, ws, vs, W, V, t, max_sweeps, tol, negl, sweeps, work, o);
  else if (R <= 2) k_jacobi<2><<<grid, block, 0, st>>>(nr, nc, ws, vs, W, V, t, max_sweeps, tol, negl, sweeps, work, o);
  else if (R <= 4) k_jacobi<4><<<grid, block, 0, st>>>(nr, nc, ws, vs, W, V, t, max_sweeps, tol, negl, sweeps, work, o);
  else if (R <= 8) k_jacobi<8><<<grid, block, 0, st>>>(nr, nc, ws, vs, W, V, t, max_sweeps, tol, negl, sweeps, work, o);
  else if (R <= 16) k_jacobi<16><<<grid, block, 0, st>>>(nr, nc, ws, vs, W, V, t, max_sweeps, tol, negl, sweeps, work, o);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace lrstv
