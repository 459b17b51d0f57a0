// svt.cu -- singular value thresholding of the Fourier frontal slices in the
// t-SVT of the E-update (arXiv 2204.12879, eq. E_solution; the slice-wise
// form follows Theorem 4.2's t-SVD).
//
// Each slice's working matrix W (nr x nc complex, nr >= nc) is orthogonalised
// by one-sided (Hestenes) Jacobi: column pairs (p, q) are rotated until
// |w_p^H w_q| <= tol |w_p| |w_q|.  The rotations accumulate in V, so W = A V
// has orthogonal columns sigma_i u_i and SVT_t(A) = W diag(g) V^H with
// g_i = max(1 - t / sigma_i, 0).  U is never formed; the reconstruction
// W (V diag g)^H is a batched complex GEMM (dft.cu).
//
// One CTA per slice.  A sweep visits all nc(nc-1)/2 pairs in np-1 rounds of
// np/2 disjoint pairs (round-robin "circle" ordering, np = nc rounded up to
// even; an odd nc gets a phantom column).  Each warp owns one pair of a
// round at a time and keeps both columns in registers (R rows per lane) for
// the dot products and the rotation.  Columns live in global memory (the
// slices are L2-resident between rounds); __syncthreads separates rounds.
// The sweep loop is capped; a slice that reaches the cap reports it.
#include <float.h>

#include "lrstv_internal.cuh"

namespace lrstv {

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
             unsigned long long *__restrict__ work) {
  float2 *W = W_all + (size_t)blockIdx.x * wstride;
  float2 *V = V_all + (size_t)blockIdx.x * vstride;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  __shared__ float s_red[32];
  __shared__ int s_rot;

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
    const float g = sigma > (double)t ? (float)(1.0 - (double)t / sigma) : 0.0f;
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
// Panel kernel (nr <= 256).  Same one-sided Jacobi and rotation formula, with
// the columns visited panel by panel: the 32 columns of panel a are first
// rotated among themselves in shared memory (round-robin, 16 disjoint pairs per
// round), then held in registers, two per warp, while every later panel b is
// staged in shared memory and swept past them: in round r warp w rotates
// panel-b column (w + r) mod 32 against both of its own columns, so one staged
// column serves two rotations.  Every pair is visited once per sweep (a block
// row-cyclic ordering), and between rounds each column is touched by a single
// warp.
constexpr int kPW = 32;      // panel width (columns)
constexpr int kPWarps = 16;  // warps per CTA; warp w holds panel columns 2w, 2w+1

struct Rot {
  float c, s, er, ei;
};

// Rotation of the 2x2 Hermitian [[al, g], [conj g, be]], or false when the
// pair is orthogonal to tolerance or a column is negligible.
__device__ __forceinline__ bool make_rot(float al, float be, float gr, float gi, float tol,
                                         float negl, Rot &r) {
  if (!(al > negl && be > negl)) return false;
  const float ag = hypotf(gr, gi);
  if (!(ag > tol * sqrtf(al) * sqrtf(be))) return false;
  const float zeta = (be - al) / (2.0f * ag);
  const float az = fabsf(zeta);
  const float tn = (az > 1e18f ? 0.5f / az : 1.0f / (az + sqrtf(fmaf(az, az, 1.0f))));
  const float tt = zeta >= 0.0f ? tn : -tn;
  r.c = 1.0f / sqrtf(fmaf(tt, tt, 1.0f));
  r.s = r.c * tt;
  r.er = gr / ag;
  r.ei = -gi / ag;
  return true;
}

template <int R>
__device__ __forceinline__ void pair_dots(const float2 (&a)[R], const float2 (&b)[R], float &al,
                                          float &be, float &gr, float &gi) {
  al = be = gr = gi = 0.f;
#pragma unroll
  for (int k = 0; k < R; ++k) {
    al = fmaf(a[k].x, a[k].x, fmaf(a[k].y, a[k].y, al));
    be = fmaf(b[k].x, b[k].x, fmaf(b[k].y, b[k].y, be));
    gr = fmaf(a[k].x, b[k].x, fmaf(a[k].y, b[k].y, gr));
    gi = fmaf(a[k].x, b[k].y, fmaf(-a[k].y, b[k].x, gi));
  }
  al = warp_sum(al);
  be = warp_sum(be);
  gr = warp_sum(gr);
  gi = warp_sum(gi);
}

// (a, b) <- (c a - s e b, s a + c e b), e = er + i ei; padded rows stay 0.
template <int R>
__device__ __forceinline__ void pair_apply(float2 (&a)[R], float2 (&b)[R], const Rot &r) {
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const float2 bb = make_float2(r.er * b[k].x - r.ei * b[k].y, r.er * b[k].y + r.ei * b[k].x);
    const float2 x = a[k];
    a[k] = make_float2(r.c * x.x - r.s * bb.x, r.c * x.y - r.s * bb.y);
    b[k] = make_float2(r.s * x.x + r.c * bb.x, r.s * x.y + r.c * bb.y);
  }
}

template <int R>
__device__ __forceinline__ void col_load(float2 (&x)[R], const float2 *src, int n, int lane) {
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const int row = lane + 32 * k;
    x[k] = row < n ? src[row] : make_float2(0.f, 0.f);
  }
}

template <int R>
__device__ __forceinline__ void col_store(const float2 (&x)[R], float2 *dst, int n, int lane) {
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const int row = lane + 32 * k;
    if (row < n) dst[row] = x[k];
  }
}

__device__ __forceinline__ void block_copy(float2 *dst, const float2 *src, size_t n) {
  for (size_t e = threadIdx.x; e < n; e += blockDim.x) dst[e] = src[e];
}

template <int R>
__global__ void __launch_bounds__(kPWarps * 32, 1)
    k_jacobi_panel(int nr, int nc, size_t wstride, size_t vstride, float2 *W_all, float2 *V_all,
                   float t, int max_sweeps, float tol, float negl_rel,
                   int *__restrict__ sweeps_out, unsigned long long *__restrict__ work) {
  extern __shared__ float4 smem_f4[];
  float2 *sW = reinterpret_cast<float2 *>(smem_f4);  // kPW columns of nr rows
  float2 *sV = sW + (size_t)kPW * nr;                // kPW columns of nc rows
  float2 *W = W_all + (size_t)blockIdx.x * wstride;
  float2 *V = V_all + (size_t)blockIdx.x * vstride;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __shared__ float s_red[32];
  __shared__ int s_rot;

  for (int e = tid; e < nc * nc; e += blockDim.x)
    V[e] = make_float2((e % nc) == (e / nc) ? 1.0f : 0.0f, 0.0f);
  float part = 0.0f;
  for (size_t e = tid; e < (size_t)nr * nc; e += blockDim.x) {
    const float2 x = W[e];
    part = fmaf(x.x, x.x, fmaf(x.y, x.y, part));
  }
  part = warp_sum(part);
  if (lane == 0) s_red[warp] = part;
  __syncthreads();
  if (warp == 0) {
    float v = lane < kPWarps ? s_red[lane] : 0.0f;
    v = warp_sum(v);
    if (lane == 0) s_red[0] = v;
  }
  __syncthreads();
  const float negl = negl_rel * s_red[0];

  const int npan = (nc + kPW - 1) / kPW;
  unsigned long long n_pairs = 0, n_rot = 0;
  int sweeps = (nc < 2) ? 1 : 0;
  bool converged = (nc < 2);
  float2 aW0[R], aV0[R], aW1[R], aV1[R], bW[R], bV[R];
  for (int sweep = 1; sweep <= max_sweeps && !converged; ++sweep) {
    if (tid == 0) s_rot = 0;
    int rotated = 0;
    for (int a = 0; a < npan; ++a) {
      const int ca = a * kPW, wa = min(kPW, nc - ca);
      __syncthreads();
      block_copy(sW, W + (size_t)nr * ca, (size_t)nr * wa);
      block_copy(sV, V + (size_t)nc * ca, (size_t)nc * wa);
      __syncthreads();
      // pairs inside panel a
      for (int r = 0; r < kPW - 1; ++r) {
        int p, q;
        pair_of(r, warp, kPW, p, q);
        if (p < wa && q < wa) {
          col_load<R>(aW0, sW + (size_t)nr * p, nr, lane);
          col_load<R>(bW, sW + (size_t)nr * q, nr, lane);
          float al, be, gr, gi;
          pair_dots<R>(aW0, bW, al, be, gr, gi);
          n_pairs += 1;
          Rot rt;
          if (make_rot(al, be, gr, gi, tol, negl, rt)) {
            pair_apply<R>(aW0, bW, rt);
            col_store<R>(aW0, sW + (size_t)nr * p, nr, lane);
            col_store<R>(bW, sW + (size_t)nr * q, nr, lane);
            col_load<R>(aV0, sV + (size_t)nc * p, nc, lane);
            col_load<R>(bV, sV + (size_t)nc * q, nc, lane);
            pair_apply<R>(aV0, bV, rt);
            col_store<R>(aV0, sV + (size_t)nc * p, nc, lane);
            col_store<R>(bV, sV + (size_t)nc * q, nc, lane);
            n_rot += 1;
            rotated = 1;
          }
        }
        __syncthreads();
      }
      // panel a's columns 2w, 2w+1 move to registers
      const int i0 = 2 * warp, i1 = 2 * warp + 1;
      const bool h0 = i0 < wa, h1 = i1 < wa;
      if (h0) {
        col_load<R>(aW0, sW + (size_t)nr * i0, nr, lane);
        col_load<R>(aV0, sV + (size_t)nc * i0, nc, lane);
      }
      if (h1) {
        col_load<R>(aW1, sW + (size_t)nr * i1, nr, lane);
        col_load<R>(aV1, sV + (size_t)nc * i1, nc, lane);
      }
      for (int b = a + 1; b < npan; ++b) {
        const int cb = b * kPW, wb = min(kPW, nc - cb);
        __syncthreads();
        block_copy(sW, W + (size_t)nr * cb, (size_t)nr * wb);
        block_copy(sV, V + (size_t)nc * cb, (size_t)nc * wb);
        __syncthreads();
        for (int r = 0; r < kPW; ++r) {
          const int j = (warp + r) & (kPW - 1);
          if (j < wb && (h0 || h1)) {
            col_load<R>(bW, sW + (size_t)nr * j, nr, lane);
            col_load<R>(bV, sV + (size_t)nc * j, nc, lane);
            bool dirty = false;
            if (h0) {
              float al, be, gr, gi;
              pair_dots<R>(aW0, bW, al, be, gr, gi);
              n_pairs += 1;
              Rot rt;
              if (make_rot(al, be, gr, gi, tol, negl, rt)) {
                pair_apply<R>(aW0, bW, rt);
                pair_apply<R>(aV0, bV, rt);
                n_rot += 1;
                dirty = true;
              }
            }
            if (h1) {
              float al, be, gr, gi;
              pair_dots<R>(aW1, bW, al, be, gr, gi);
              n_pairs += 1;
              Rot rt;
              if (make_rot(al, be, gr, gi, tol, negl, rt)) {
                pair_apply<R>(aW1, bW, rt);
                pair_apply<R>(aV1, bV, rt);
                n_rot += 1;
                dirty = true;
              }
            }
            if (dirty) {
              col_store<R>(bW, sW + (size_t)nr * j, nr, lane);
              col_store<R>(bV, sV + (size_t)nc * j, nc, lane);
              rotated = 1;
            }
          }
          __syncthreads();
        }
        block_copy(W + (size_t)nr * cb, sW, (size_t)nr * wb);
        block_copy(V + (size_t)nc * cb, sV, (size_t)nc * wb);
      }
      if (h0) {
        col_store<R>(aW0, W + (size_t)nr * (ca + i0), nr, lane);
        col_store<R>(aV0, V + (size_t)nc * (ca + i0), nc, lane);
      }
      if (h1) {
        col_store<R>(aW1, W + (size_t)nr * (ca + i1), nr, lane);
        col_store<R>(aV1, V + (size_t)nc * (ca + i1), nc, lane);
      }
    }
    if (rotated && lane == 0) s_rot = 1;
    __syncthreads();
    sweeps = sweep;
    converged = (s_rot == 0);
    __syncthreads();
  }

  for (int i = warp; i < nc; i += kPWarps) {
    const float2 *wi = W + (size_t)nr * i;
    float n2 = 0.f;
    for (int row = lane; row < nr; row += 32) n2 = fmaf(wi[row].x, wi[row].x, fmaf(wi[row].y, wi[row].y, n2));
    n2 = warp_sum(n2);
    const double sigma = sqrt((double)n2);
    const float g = sigma > (double)t ? (float)(1.0 - (double)t / sigma) : 0.0f;
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
// Half-warp kernel (nr <= 208).  The panel scheme above with one column pair
// per half-warp (16 lanes, R2 rows per lane), so each warp instruction works on
// two independent pairs, reductions take four shuffle levels, and the 32
// columns of panel a map to the 32 half-warps.  Panels are staged in shared
// memory with rows padded to 16 R2 (zeros, which rotations keep at zero), so
// no row needs a bounds check.  A half-warp whose pair is phantom, negligible
// or already orthogonal applies the identity rotation (c = 1, s = 0, e = 1),
// which leaves its columns bit-for-bit unchanged.
constexpr int kHW = 16;  // warps per CTA (32 half-warps)

__device__ __forceinline__ float half_sum(float v) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int R2>
__device__ __forceinline__ void hw_dots(const float2 (&a)[R2], const float2 (&b)[R2], float &al,
                                        float &be, float &gr, float &gi) {
  al = be = gr = gi = 0.f;
#pragma unroll
  for (int k = 0; k < R2; ++k) {
    al = fmaf(a[k].x, a[k].x, fmaf(a[k].y, a[k].y, al));
    be = fmaf(b[k].x, b[k].x, fmaf(b[k].y, b[k].y, be));
    gr = fmaf(a[k].x, b[k].x, fmaf(a[k].y, b[k].y, gr));
    gi = fmaf(a[k].x, b[k].y, fmaf(-a[k].y, b[k].x, gi));
  }
  al = half_sum(al);
  be = half_sum(be);
  gr = half_sum(gr);
  gi = half_sum(gi);
}

template <int R2>
__device__ __forceinline__ void hw_load(float2 (&x)[R2], const float2 *col, int ul) {
#pragma unroll
  for (int k = 0; k < R2; ++k) x[k] = col[ul + kHW * k];
}

template <int R2>
__device__ __forceinline__ void hw_store(const float2 (&x)[R2], float2 *col, int ul) {
#pragma unroll
  for (int k = 0; k < R2; ++k) col[ul + kHW * k] = x[k];
}

// Rotates the register column a against the shared-memory column col,
// streaming col through registers C rows at a time (keeps few registers live).
template <int R2, int C>
__device__ __forceinline__ void hw_rot_stream(float2 (&a)[R2], float2 *col, const Rot &r, int ul) {
#pragma unroll
  for (int k0 = 0; k0 < R2; k0 += C) {
    float2 b[C];
#pragma unroll
    for (int k = 0; k < C; ++k)
      if (k0 + k < R2) b[k] = col[ul + kHW * (k0 + k)];
#pragma unroll
    for (int k = 0; k < C; ++k) {
      if (k0 + k < R2) {
        const float2 bb = make_float2(r.er * b[k].x - r.ei * b[k].y, r.er * b[k].y + r.ei * b[k].x);
        const float2 x = a[k0 + k];
        a[k0 + k] = make_float2(r.c * x.x - r.s * bb.x, r.c * x.y - r.s * bb.y);
        b[k] = make_float2(r.s * x.x + r.c * bb.x, r.s * x.y + r.c * bb.y);
      }
    }
#pragma unroll
    for (int k = 0; k < C; ++k)
      if (k0 + k < R2) col[ul + kHW * (k0 + k)] = b[k];
  }
}

// shared panel (ld rows per column, zero padded) <- wcols columns of n rows
__device__ __forceinline__ void stage_in(float2 *dst, int ld, const float2 *src, int n, int wcols) {
  const float2 z = make_float2(0.f, 0.f);
  for (int e = threadIdx.x; e < kPW * ld; e += blockDim.x) {
    const int c = e / ld, r = e - c * ld;
    dst[e] = (c < wcols && r < n) ? src[(size_t)n * c + r] : z;
  }
}

__device__ __forceinline__ void stage_out(float2 *dst, const float2 *src, int ld, int n, int wcols) {
  for (int e = threadIdx.x; e < wcols * n; e += blockDim.x) {
    const int c = e / n, r = e - c * n;
    dst[e] = src[c * ld + r];
  }
}

template <int R2>
__global__ void __launch_bounds__(kHW * 32, 1)
    k_jacobi_hw(int nr, int nc, size_t wstride, size_t vstride, float2 *W_all, float2 *V_all,
                float t, int max_sweeps, float tol, float negl_rel, int *__restrict__ sweeps_out,
                unsigned long long *__restrict__ work) {
  constexpr int LD = kHW * R2;  // padded rows of a staged column
  extern __shared__ float4 smem_f4[];
  float2 *sW = reinterpret_cast<float2 *>(smem_f4);  // kPW x LD
  float2 *sV = sW + kPW * LD;                          // kPW x LD
  float2 *W = W_all + (size_t)blockIdx.x * wstride;
  float2 *V = V_all + (size_t)blockIdx.x * vstride;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int unit = tid >> 4, ul = tid & 15;  // half-warp and its lane
  __shared__ float s_red[32];
  __shared__ int s_rot;

  for (int e = tid; e < nc * nc; e += blockDim.x)
    V[e] = make_float2((e % nc) == (e / nc) ? 1.0f : 0.0f, 0.0f);
  float part = 0.0f;
  for (size_t e = tid; e < (size_t)nr * nc; e += blockDim.x) {
    const float2 x = W[e];
    part = fmaf(x.x, x.x, fmaf(x.y, x.y, part));
  }
  part = warp_sum(part);
  if (lane == 0) s_red[warp] = part;
  __syncthreads();
  if (warp == 0) {
    float v = lane < kHW ? s_red[lane] : 0.0f;
    v = warp_sum(v);
    if (lane == 0) s_red[0] = v;
  }
  __syncthreads();
  const float negl = negl_rel * s_red[0];

  const int npan = (nc + kPW - 1) / kPW;
  unsigned long long n_pairs = 0, n_rot = 0;  // counted by lane 0 of each half-warp
  int sweeps = (nc < 2) ? 1 : 0;
  bool converged = (nc < 2);
  float2 aW[R2], aV[R2], bW[R2];
  for (int sweep = 1; sweep <= max_sweeps && !converged; ++sweep) {
    if (tid == 0) s_rot = 0;
    int rotated = 0;
    for (int a = 0; a < npan; ++a) {
      const int ca = a * kPW, wa = min(kPW, nc - ca);
      __syncthreads();
      stage_in(sW, LD, W + (size_t)nr * ca, nr, wa);
      stage_in(sV, LD, V + (size_t)nc * ca, nc, wa);
      __syncthreads();
      // pairs inside panel a: 16 disjoint pairs per round on half-warps 0..15
      for (int r = 0; r < kPW - 1; ++r) {
        if (unit < kPW / 2) {
          int p, q;
          pair_of(r, unit, kPW, p, q);
          const bool real = p < wa && q < wa;
          hw_load<R2>(aW, sW + LD * p, ul);
          hw_load<R2>(bW, sW + LD * q, ul);
          float al, be, gr, gi;
          hw_dots<R2>(aW, bW, al, be, gr, gi);
          Rot rt;
          const bool go = real && make_rot(al, be, gr, gi, tol, negl, rt);
          if (ul == 0 && real) n_pairs += 1;
          if (go) {
            pair_apply<R2>(aW, bW, rt);
            hw_store<R2>(aW, sW + LD * p, ul);
            hw_store<R2>(bW, sW + LD * q, ul);
            hw_load<R2>(aV, sV + LD * p, ul);
            hw_rot_stream<R2, 4>(aV, sV + LD * q, rt, ul);
            hw_store<R2>(aV, sV + LD * p, ul);
            if (ul == 0) n_rot += 1;
            rotated = 1;
          }
        }
        __syncthreads();
      }
      // panel a's column `unit` moves to registers
      const bool mine = unit < wa;
      hw_load<R2>(aW, sW + LD * unit, ul);
      hw_load<R2>(aV, sV + LD * unit, ul);
      for (int b = a + 1; b < npan; ++b) {
        const int cb = b * kPW, wb = min(kPW, nc - cb);
        __syncthreads();
        stage_in(sW, LD, W + (size_t)nr * cb, nr, wb);
        stage_in(sV, LD, V + (size_t)nc * cb, nc, wb);
        __syncthreads();
        for (int r = 0; r < kPW; ++r) {
          const int j = (unit + r) & (kPW - 1);
          const bool real = mine && j < wb;
          hw_load<R2>(bW, sW + LD * j, ul);
          float al, be, gr, gi;
          hw_dots<R2>(aW, bW, al, be, gr, gi);
          Rot rt;
          const bool go = real && make_rot(al, be, gr, gi, tol, negl, rt);
          if (ul == 0 && real) n_pairs += 1;
          if (__any_sync(0xffffffffu, go)) {
            // the other half-warp of this warp may rotate: this half applies
            // the identity, which rewrites its columns unchanged
            if (!go) {
              rt.c = 1.0f;
              rt.s = 0.0f;
              rt.er = 1.0f;
              rt.ei = 0.0f;
            }
            pair_apply<R2>(aW, bW, rt);
            hw_store<R2>(bW, sW + LD * j, ul);
            hw_rot_stream<R2, 4>(aV, sV + LD * j, rt, ul);
            if (go) {
              if (ul == 0) n_rot += 1;
              rotated = 1;
            }
          }
          __syncthreads();
        }
        stage_out(W + (size_t)nr * cb, sW, LD, nr, wb);
        stage_out(V + (size_t)nc * cb, sV, LD, nc, wb);
      }
      if (mine) {
        float2 *wcol = W + (size_t)nr * (ca + unit);
        float2 *vcol = V + (size_t)nc * (ca + unit);
#pragma unroll
        for (int k = 0; k < R2; ++k) {
          const int row = ul + kHW * k;
          if (row < nr) wcol[row] = aW[k];
          if (row < nc) vcol[row] = aV[k];
        }
      }
    }
    if (rotated) s_rot = 1;
    __syncthreads();
    sweeps = sweep;
    converged = (s_rot == 0);
    __syncthreads();
  }

  for (int i = warp; i < nc; i += kHW) {
    const float2 *wi = W + (size_t)nr * i;
    float n2 = 0.f;
    for (int row = lane; row < nr; row += 32) n2 = fmaf(wi[row].x, wi[row].x, fmaf(wi[row].y, wi[row].y, n2));
    n2 = warp_sum(n2);
    const double sigma = sqrt((double)n2);
    const float g = sigma > (double)t ? (float)(1.0 - (double)t / sigma) : 0.0f;
    float2 *vi = V + (size_t)nc * i;
    for (int row = lane; row < nc; row += 32) vi[row] = make_float2(vi[row].x * g, vi[row].y * g);
  }
  if (tid == 0) sweeps_out[blockIdx.x] = converged ? sweeps : -max_sweeps;
  if (work && ul == 0) {
    atomicAdd(work + 0, n_pairs);
    atomicAdd(work + 1, n_rot);
  }
}

template <int R2>
cudaError_t launch_hw(int nslices, int nr, int nc, size_t ws, size_t vs, float2 *W, float2 *V,
                      float t, int max_sweeps, float tol, float negl, int *sweeps,
                      unsigned long long *work, cudaStream_t st) {
  const size_t smem = sizeof(float2) * 2 * (size_t)kPW * kHW * R2;
  cudaError_t e = cudaFuncSetAttribute(k_jacobi_hw<R2>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_jacobi_hw<R2><<<nslices, kHW * 32, smem, st>>>(nr, nc, ws, vs, W, V, t, max_sweeps, tol, negl,
                                                   sweeps, work);
  return cudaGetLastError();
}

template <int R>
cudaError_t launch_panel(int nslices, int nr, int nc, size_t ws, size_t vs, float2 *W, float2 *V,
                         float t, int max_sweeps, float tol, float negl, int *sweeps,
                         unsigned long long *work, cudaStream_t st) {
  const size_t smem = sizeof(float2) * (size_t)kPW * (nr + nc);
  cudaError_t e = cudaFuncSetAttribute(k_jacobi_panel<R>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_jacobi_panel<R><<<nslices, kPWarps * 32, smem, st>>>(nr, nc, ws, vs, W, V, t, max_sweeps, tol,
                                                         negl, sweeps, work);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_jacobi(const Dims &d, int nslices, float2 *W, float2 *V, float t,
                          int max_sweeps, int *sweeps, unsigned long long *work,
                          cudaStream_t st) {
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
  const float tol = 8.0f * sqrtf((float)nr) * eps;
  const float negl = ((float)nr * eps) * ((float)nr * eps);
  const size_t ws = d.P, vs = (size_t)nc * nc;
  if (nr <= 208 && nc >= 2) {
    const int R2 = (nr + 15) / 16;
    if (R2 <= 2) return launch_hw<2>(nslices, nr, nc, ws, vs, W, V, t, max_sweeps, tol, negl, sweeps, work, st);
    if (R2 <= 4) return launch_hw<4>(nslices, nr, nc, ws, vs, W, V, t, max_sweeps, tol, negl, sweeps, work, st);
    if (R2 <= 8) return launch_hw<8>(nslices, nr, nc, ws, vs, W, V, t, max_sweeps, tol, negl, sweeps, work, st);
    return launch_hw<13>(nslices, nr, nc, ws, vs, W, V, t, max_sweeps, tol, negl, sweeps, work, st);
  }
  if (R <= 8 && nc >= 2) {
    if (R <= 1) return launch_panel<1>(nslices, nr, nc, ws, vs, W, V, t, max_sweeps, tol, negl, sweeps, work, st);
    if (R <= 2) return launch_panel<2>(nslices, nr, nc, ws, vs, W, V, t, max_sweeps, tol, negl, sweeps, work, st);
    if (R <= 4) return launch_panel<4>(nslices, nr, nc, ws, vs, W, V, t, max_sweeps, tol, negl, sweeps, work, st);
    return launch_panel<8>(nslices, nr, nc, ws, vs, W, V, t, max_sweeps, tol, negl, sweeps, work, st);
  }
  dim3 grid(nslices), block(32 * nw);
  if (R <= 1) k_jacobi<1><<<grid, block, 0, st>>>(nr, nc, ws, vs, W, V, t, max_sweeps, tol, negl, sweeps, work);
  else if (R <= 2) k_jacobi<2><<<grid, block, 0, st>>>(nr, nc, ws, vs, W, V, t, max_sweeps, tol, negl, sweeps, work);
  else if (R <= 4) k_jacobi<4><<<grid, block, 0, st>>>(nr, nc, ws, vs, W, V, t, max_sweeps, tol, negl, sweeps, work);
  else if (R <= 8) k_jacobi<8><<<grid, block, 0, st>>>(nr, nc, ws, vs, W, V, t, max_sweeps, tol, negl, sweeps, work);
  else if (R <= 16) k_jacobi<16><<<grid, block, 0, st>>>(nr, nc, ws, vs, W, V, t, max_sweeps, tol, negl, sweeps, work);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace lrstv
