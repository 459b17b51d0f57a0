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
