// tcgemm.cu -- batched complex GEMM on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory) for the dense contractions of
// the iteration: the spatial DFT passes of the Z-solve (eq. Z_solution) and
// the SVT reconstruction W (V diag g)^H of the E-update (eq. E_solution).
//
// Same contract as k_cgemm (dft.cu): C_b = A_b op(B_b), column-major complex,
// op(B) = B or B^H, optional spectral-division epilogue.
//
// Precision: FP32-accurate "3xTF32".  Each FP32 operand x is split into
// x_hi = tf32(x) and x_lo = x - x_hi, and a product is formed as
// hi*hi + hi*lo + lo*hi with FP32 accumulation (the lo*lo term is below FP32
// resolution), so the result carries about 2^-21 relative error per term
// instead of TF32's 2^-11.  The tensor core accumulates with truncation, so
// each K chunk (32 real terms) goes into a fresh TMEM tile that the threads
// drain into FP32 register accumulators: accumulation error then grows over
// 32 terms, not over the whole K.
//
// Complex arithmetic as real GEMMs with K doubled: for a K chunk,
//   Re C += [Re A | Im A] . [Re B | -Im B]^T,   Im C += [Re A | Im A] . [Im B | Re B]^T.
//
// Tile: 128 rows of C (M = 128 MMA), 64 complex columns (two N = 64 MMAs
// into 128 TMEM columns), 16 complex K per chunk (four K = 8 MMA steps per
// product).  Operands are staged by the CTA's threads into shared memory in
// the canonical K-major layout without swizzle: 8-row x 16-byte core matrices,
// K-adjacent core matrices 128 B apart (LBO), 8-row groups 1024 B apart (SBO).
// One thread issues the MMAs and commits them to an mbarrier; every wait on
// that barrier is bounded and, if it runs out, the CTA records an error flag,
// skips its epilogue and still frees its tensor memory.
#include <stdint.h>

#include "lrstv_internal.cuh"

namespace lrstv {

namespace {

constexpr int TM = 128;       // rows of C per CTA
constexpr int TN = 64;        // complex columns of C per CTA
constexpr int TK = 16;        // complex K per chunk (32 real K)
constexpr int KR = 2 * TK;    // real K per chunk
constexpr int kThreads = 128; // four warps: TMEM lanes 0..127
constexpr uint32_t kLBO = 128, kSBO = (KR / 4) * 128;  // bytes
constexpr int kTileA = TM * KR;  // floats per A tile (one split)
constexpr int kTileB = TN * KR;  // floats per B tile (one split, one of re/im)
constexpr long long kWaitLimit = 20000000;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((kLBO >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((kSBO >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of tcgen05; no swizzle, base offset 0
  return d;
}

// byte offset of element (row r, real k kk) in a K-major no-swizzle tile
__device__ __forceinline__ int koff(int r, int kk) {
  return (r >> 3) * (int)kSBO + (kk >> 2) * (int)kLBO + (r & 7) * 16 + (kk & 3) * 4;
}

__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void put_split(float *hi, float *lo, int off, float x) {
  const float h = tf32_hi(x);
  hi[off >> 2] = h;
  lo[off >> 2] = x - h;
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  for (long long it = 0; it < kWaitLimit && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity));
  }
  return done != 0;
}

template <int OPB, int EPI>
__global__ void __launch_bounds__(kThreads, 1) k_cgemm_tc(CGemm g, int *err) {
  extern __shared__ __align__(1024) float smem[];
  float *aHi = smem, *aLo = aHi + kTileA;
  float *bReHi = aLo + kTileA, *bReLo = bReHi + kTileB;
  float *bImHi = bReLo + kTileB, *bImLo = bImHi + kTileB;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  __shared__ int s_ok;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = blockIdx.z;
  const float2 *A = g.A + (size_t)b * g.sA;
  const float2 *B = g.B + (size_t)b * g.sB;
  float2 *C = g.C + (size_t)b * g.sC;
  const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_ok = 1;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(
        smem_u32(&tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tslot;
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TN >> 3) << 17) |
                         ((uint32_t)(TM >> 4) << 24);
  const uint32_t bar = smem_u32(&mbar);

  uint32_t phase = 0;
  bool ok = true;
  const int row = 32 * warp + lane;  // TMEM lane = row of the tile this thread drains
  const uint32_t tl = tmem + ((uint32_t)(32 * warp) << 16);
  float accRe[TN], accIm[TN];
#pragma unroll
  for (int c = 0; c < TN; ++c) {
    accRe[c] = 0.f;
    accIm[c] = 0.f;
  }
  const int nchunks = (g.K + TK - 1) / TK;
  for (int ch = 0; ch < nchunks && ok; ++ch) {
    const int k0 = ch * TK;
    // A tile: rows m0..m0+127, complex k0..k0+15 -> real kk = k (re), k + 16 (im).
    // A warp covers 8 rows x 4 k: its 32 stores hit 32 distinct banks of a core
    // matrix row group, and its loads are four 64-byte runs of a column.
    for (int e = tid; e < TM * TK; e += kThreads) {
      const int rest = e >> 5;
      const int r = ((rest % (TM / 8)) << 3) | ((e >> 2) & 7);
      const int kc = ((rest / (TM / 8)) << 2) | (e & 3);
      const int gm = m0 + r, gk = k0 + kc;
      const float2 v = (gm < g.M && gk < g.K) ? A[gm + (size_t)g.lda * gk] : make_float2(0.f, 0.f);
      put_split(aHi, aLo, koff(r, kc), v.x);
      put_split(aHi, aLo, koff(r, kc + TK), v.y);
    }
    // B tiles for output columns n0..n0+63: row n holds op(B)(k, n) over k
    // (8 rows n x 4 k per warp, as for A: conflict-free stores; loads are runs
    // of 4 k (B(k, n) at k + ldb n) or of 8 n (B(n, k) at n + ldb k))
    for (int e = tid; e < TN * TK; e += kThreads) {
      const int rest = e >> 5;
      const int n = ((rest % (TN / 8)) << 3) | ((e >> 2) & 7);
      const int kc = ((rest / (TN / 8)) << 2) | (e & 3);
      const int gn = n0 + n, gk = k0 + kc;
      float2 v = make_float2(0.f, 0.f);
      if (gn < g.N && gk < g.K) {
        v = OPB == 0 ? B[gk + (size_t)g.ldb * gn] : B[gn + (size_t)g.ldb * gk];
        if (OPB == 1) v.y = -v.y;
      }
      put_split(bReHi, bReLo, koff(n, kc), v.x);        // [Re B | -Im B]
      put_split(bReHi, bReLo, koff(n, kc + TK), -v.y);
      put_split(bImHi, bImLo, koff(n, kc), v.y);        // [Im B | Re B]
      put_split(bImHi, bImLo, koff(n, kc + TK), v.x);
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0) {
      const uint32_t a_hi = smem_u32(aHi), a_lo = smem_u32(aLo);
      const uint32_t br_hi = smem_u32(bReHi), br_lo = smem_u32(bReLo);
      const uint32_t bi_hi = smem_u32(bImHi), bi_lo = smem_u32(bImLo);
#pragma unroll
      for (int j = 0; j < KR / 8; ++j) {  // K = 8 per instruction = two core matrices
        const uint32_t ko = (uint32_t)j * 2 * kLBO;
        const uint32_t acc0 = j > 0 ? 1u : 0u;  // a fresh tile per chunk
        // Re C (TMEM columns 0..63), Im C (64..127); 3xTF32 per product
        mma_tf32(tmem, sdesc(a_hi + ko), sdesc(br_hi + ko), idesc, acc0);
        mma_tf32(tmem, sdesc(a_hi + ko), sdesc(br_lo + ko), idesc, 1u);
        mma_tf32(tmem, sdesc(a_lo + ko), sdesc(br_hi + ko), idesc, 1u);
        mma_tf32(tmem + TN, sdesc(a_hi + ko), sdesc(bi_hi + ko), idesc, acc0);
        mma_tf32(tmem + TN, sdesc(a_hi + ko), sdesc(bi_lo + ko), idesc, 1u);
        mma_tf32(tmem + TN, sdesc(a_lo + ko), sdesc(bi_hi + ko), idesc, 1u);
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar));
    }
    // the MMAs must finish reading the tiles before they are restaged
    if (!mbar_wait(bar, phase)) {
      ok = false;
      if (tid == 0) s_ok = 0;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    __syncthreads();
    ok = ok && s_ok;
    if (ok) {  // drain this chunk's tile into the register accumulators
#pragma unroll
      for (int c0 = 0; c0 < TN; c0 += 16) {
        uint32_t re[16], im[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(re[0]), "=r"(re[1]), "=r"(re[2]), "=r"(re[3]), "=r"(re[4]), "=r"(re[5]),
              "=r"(re[6]), "=r"(re[7]), "=r"(re[8]), "=r"(re[9]), "=r"(re[10]), "=r"(re[11]),
              "=r"(re[12]), "=r"(re[13]), "=r"(re[14]), "=r"(re[15])
            : "r"(tl + c0));
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(im[0]), "=r"(im[1]), "=r"(im[2]), "=r"(im[3]), "=r"(im[4]), "=r"(im[5]),
              "=r"(im[6]), "=r"(im[7]), "=r"(im[8]), "=r"(im[9]), "=r"(im[10]), "=r"(im[11]),
              "=r"(im[12]), "=r"(im[13]), "=r"(im[14]), "=r"(im[15])
            : "r"(tl + TN + c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          accRe[c0 + c] += __uint_as_float(re[c]);
          accIm[c0 + c] += __uint_as_float(im[c]);
        }
      }
      // the next chunk's MMAs overwrite the tile only after every thread's reads
      asm volatile("tcgen05.fence::before_thread_sync;");
    }
  }
  if (!ok) {
    if (tid == 0 && err) atomicExch(err, 1);
    // give MMAs still in flight a last bounded chance to land before the free
    mbar_wait(bar, phase ^ 1u);
  } else if (nchunks > 0) {
    // epilogue: thread (warp w, lane l) owns row m0 + 32 w + l of the tile
    const int gm = m0 + row;
    const int lb = g.lam3_period > 0 ? b % g.lam3_period : b;
    if (gm < g.M) {
#pragma unroll
      for (int c = 0; c < TN; ++c) {
        const int n = n0 + c;
        if (n >= g.N) break;
        float2 v = make_float2(accRe[c], accIm[c]);
        if (EPI == 1) {
          const float den = g.mu * (1.0f + g.lam1[gm] + g.lam2[n] + g.lam3[lb]);
          const float q = g.scale / den;
          v.x *= q;
          v.y *= q;
        }
        C[gm + (size_t)g.ldc * n] = v;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
}

}  // namespace

size_t cgemm_tc_smem() { return sizeof(float) * (2 * (size_t)kTileA + 4 * (size_t)kTileB); }

cudaError_t launch_cgemm_tc(const CGemm &g, int *err, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  if (g.opA != 0 || g.epi == 2) return cudaErrorInvalidValue;  // SIMT kernel only
  const size_t smem = cgemm_tc_smem();
  dim3 grid((g.M + TM - 1) / TM, (g.N + TN - 1) / TN, g.batch);
  cudaError_t e;
#define LRSTV_TC_LAUNCH(OPB, EPI)                                                              \
  e = cudaFuncSetAttribute(k_cgemm_tc<OPB, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                           (int)smem);                                                        \
  if (e != cudaSuccess) return e;                                                             \
  k_cgemm_tc<OPB, EPI><<<grid, kThreads, smem, st>>>(g, err);
  if (g.opB == 0 && g.epi == 0) {
    LRSTV_TC_LAUNCH(0, 0)
  } else if (g.opB == 0 && g.epi == 1) {
    LRSTV_TC_LAUNCH(0, 1)
  } else if (g.opB == 1 && g.epi == 0) {
    LRSTV_TC_LAUNCH(1, 0)
  } else {
    return cudaErrorInvalidValue;
  }
#undef LRSTV_TC_LAUNCH
  return cudaGetLastError();
}

}  // namespace lrstv
