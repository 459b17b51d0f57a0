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
// each K chunk (16 real terms) goes into a fresh TMEM tile that the threads
// drain into FP32 register accumulators: accumulation error then grows over
// 16 terms, not over the whole K.
//
// Complex arithmetic as real GEMMs with K doubled: for a K chunk,
//   Re C += [Re A | Im A] . [Re B | -Im B]^T,   Im C += [Re A | Im A] . [Im B | Re B]^T.
//
// Mixed precision (prec = 1, "3xBF16"): the same split with bf16 halves,
// x_hi = bf16(x), x_lo = bf16(x - x_hi), and the three products on the BF16
// tensor-core path (kind::f16, both operands bf16, FP32 accumulation): about
// 2^-17 relative error per term, half the shared-memory bytes and half the
// MMA instructions of 3xTF32 (K = 16 per instruction instead of 8).
//
// Tile: 128 rows of C (M = 128 MMA), 64 complex columns (one N = 128 MMA over
// the adjacent Re and Im B tiles into 128 TMEM columns, which reads the A tile
// once for both parts), 8 (3xTF32) or 16 (3xBF16) complex K per chunk: two
// K = 8 TF32 or two K = 16 BF16 MMA steps per product, a 32 KB stage either
// way.  Operands are staged by the CTA's threads into shared memory in the
// canonical K-major layout without swizzle: 8-row x 16-byte core matrices,
// K-adjacent core matrices 128 B apart (LBO), 8-row groups one chunk row
// (KR elements) apart (SBO).  Two stages and two TMEM tiles pipeline the
// chunks: chunk k is loaded and staged while chunk k - 1's MMAs run, and
// chunk k - 1's tile is drained while chunk k's MMAs run.
// One thread issues the MMAs and commits them to the stage's mbarrier; every
// wait on a barrier is bounded and, if it runs out, the CTA records an error
// flag, skips its epilogue and still frees its tensor memory.
#include <cuda_bf16.h>
#include <stdint.h>

#include "lrstv_internal.cuh"

namespace lrstv {

namespace {

constexpr int TM = 128;       // rows of C per CTA
constexpr int TN = 64;        // complex columns of C per CTA
// eight warps: warp w reads TMEM lanes 32 (w mod 4) .. + 31 (rows of the tile)
// and, by warpgroup, columns 0..31 or 32..63 of each Re / Im tile
constexpr int kThreads = 256;
constexpr uint32_t kLBO = 128;  // bytes
// tries of a bounded barrier wait: one mbarrier.try_wait that finds the
// phase incomplete suspends the thread for about 3.8 us on GB300 (measured
// by the wait probe below), so the bound is about a second, against the
// microseconds one chunk's MMAs take
constexpr long long kWaitLimit = 250000;

// Per precision: element bytes, elements per 16-byte core-matrix row, the
// 8-row group stride, tile sizes and the instruction descriptor's operand
// format (kind::tf32: TF32 = 2; kind::f16: BF16 = 1).
template <int PREC>
struct Prec {
  static constexpr int kBytes = PREC ? 2 : 4;
  // complex K per chunk: 8 for 3xTF32 (16 real terms per TMEM tile), 16 for
  // 3xBF16; either way a stage is 32 KB and two stages fit two CTAs per SM
  static constexpr int kTK = PREC ? 16 : 8;
  static constexpr int kKR = 2 * kTK;                             // real K per chunk
  static constexpr int kPerCore = 16 / kBytes;                    // along K
  static constexpr uint32_t kSBO = (kKR / kPerCore) * 128;        // bytes
  static constexpr int kMmaK = PREC ? 16 : 8;                     // K per instruction
  static constexpr uint32_t kFmt = PREC ? 1u : 2u;
  static constexpr size_t kTileA = (size_t)TM * kKR * kBytes;     // bytes, one split
  static constexpr size_t kTileB = (size_t)TN * kKR * kBytes;     // bytes, one split, re or im
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

template <int PREC>
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((kLBO >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((Prec<PREC>::kSBO >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of tcgen05; no swizzle, base offset 0
  return d;
}

// byte offset of element (row r, real k kk) in a K-major no-swizzle tile
template <int PREC>
__device__ __forceinline__ int koff(int r, int kk) {
  constexpr int pc = Prec<PREC>::kPerCore;
  return (r >> 3) * (int)Prec<PREC>::kSBO + (kk / pc) * (int)kLBO + (r & 7) * 16 +
         (kk % pc) * Prec<PREC>::kBytes;
}

__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// x = hi + lo at byte offset off of the hi and lo tiles
template <int PREC>
__device__ __forceinline__ void put_split(char *hi, char *lo, int off, float x) {
  if (PREC == 0) {
    const float h = tf32_hi(x);
    *(float *)(hi + off) = h;
    *(float *)(lo + off) = x - h;
  } else {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    *(__nv_bfloat16 *)(hi + off) = h;
    *(__nv_bfloat16 *)(lo + off) = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}

// Two consecutive-k values as BF16 hi and lo halves, one 4-byte word each
// (off 4-byte aligned: k even).
__device__ __forceinline__ void put_split2(char *hi, char *lo, int off, float x0, float x1) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
  const float2 hf = __bfloat1622float2(h);
  *(__nv_bfloat162 *)(hi + off) = h;
  *(__nv_bfloat162 *)(lo + off) = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
}

template <int PREC>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t accumulate) {
  if (PREC == 0)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          long long tries = kWaitLimit) {
  uint32_t done = 0;
  for (long long it = 0; it < tries && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
  }
  return done != 0;
}

// KIND 0: the complex GEMM C = A op(B) of CGemm (OPB 0: B, 1: B^H), or, with
// OPB 2, C = A^H B (the Gram products W^H W).  KIND 1 and 2: the mode-3
// DFTs of the cubes of Dft3 as GEMMs over the pixels (M = n1 n2):
//  KIND 1 (real -> half spectrum): C(p, k) = sum_c x(p, c) exp(-2 pi i k c / n3),
//    k < h, a real A (x, or x - ycoef y) against the twiddles; a K chunk holds
//    KR real bands in the A tile, and the B tiles hold the real and the
//    imaginary twiddle parts of those bands, so that the MMAs form Re C and
//    Im C directly.  Written at the working orientation's pixel (conjugated
//    when transposed).
//  KIND 2 (half spectrum -> real): x(p, c) = (1/n3) sum_{k<h} w_k Re(X_k(p)
//    exp(2 pi i k c / n3)) with w_k = 1 at k = 0 and k = n3/2, else 2: the
//    complex GEMM's Re C alone, B(k, c) = w_k exp(2 pi i k c / n3); the
//    epilogue scales by 1/n3 and, in mode 1, updates Gamma4 += mu (x - F).
// The DFT kinds take their tile indices from blockIdx.x with the N tiles of
// one M tile adjacent in launch order, so the M tile's inputs come from DRAM
// once and from L2 for the other N tiles.
template <int OPB, int EPI, int PREC, int KIND = 0>
// The forward DFT kind holds both cubes' next chunk in registers (152 of them
// with 3xTF32) and runs one CTA per SM without spills; the others fit two.
__global__ void __launch_bounds__(kThreads, KIND == 1 ? 1 : 2) k_cgemm_tc(CGemm g, Dft3 f, int *err) {
  extern __shared__ __align__(1024) char smem[];
  using P = Prec<PREC>;
  // two shared-memory stages, so that a chunk is staged while the previous
  // chunk's MMAs run, and two TMEM tiles (one per stage)
  constexpr uint32_t kCols = 256;
  constexpr size_t kStageBytes = 2 * P::kTileA + 4 * P::kTileB;
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tslot;
  __shared__ int s_ok;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = blockIdx.z;
  if (KIND == 0 && g.gate && !g.gate[b]) return;  // a gated-off batch entry (CTA-uniform)
  const float2 *A = g.A + (size_t)b * g.sA;
  const float2 *B = g.B + (size_t)b * g.sB;
  float2 *C = g.C + (size_t)b * g.sC;
  int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
  // the DFT kinds: problem size, this batch entry's cubes
  int gM = g.M, gN = g.N, gK = g.K;
  const float *xb = nullptr, *yb = nullptr;
  const float2 *specb = nullptr;
  if (KIND != 0) {
    const int nt = ((KIND == 1 ? f.h : f.n3) + TN - 1) / TN;
    m0 = (blockIdx.x / nt) * TM;
    n0 = (blockIdx.x % nt) * TN;
    gM = (int)f.P;
    gN = KIND == 1 ? f.h : f.n3;
    gK = KIND == 1 ? f.n3 : f.h;
    if (KIND == 1) {
      xb = f.x + (size_t)b * f.N;
      if (f.y) yb = f.y + (size_t)b * f.N;
    } else {
      specb = f.spec + (size_t)b * f.h * f.P;
    }
  }
  // pixel p of the cube -> its index in the working orientation's slice
  auto wpos = [&](int p) -> size_t {
    if (!f.trans) return (size_t)p;
    const int i = p % f.n1, j = p / f.n1;
    return (size_t)j + (size_t)f.n2 * i;
  };

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_ok = 1;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tslot)),
                 "n"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tslot;
  // D format F32, A and B in the precision's format, both K-major, N, M
  const uint32_t idesc = (1u << 4) | (P::kFmt << 7) | (P::kFmt << 10) |
                         ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
  const uint32_t idesc2 = (1u << 4) | (P::kFmt << 7) | (P::kFmt << 10) |
                          ((uint32_t)((2 * TN) >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
  const uint32_t bar0 = smem_u32(&mbar[0]), bar1 = smem_u32(&mbar[1]);
  // per stage: the parity of its next MMA commit, and whether a commit is
  // outstanding (issued, not yet seen complete)
  uint32_t ph0 = 0u, ph1 = 0u;
  bool out0 = false, out1 = false;
  bool ok = true;
  const int row = 32 * (warp & 3) + lane;  // TMEM lane = row of the tile this thread drains
  const int colh = (warp >> 2) * (TN / 2);  // first of the 32 columns it drains
  const uint32_t tl = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)colh;
  float accRe[TN / 2], accIm[TN / 2];
#pragma unroll
  for (int c = 0; c < TN / 2; ++c) {
    accRe[c] = 0.f;
    accIm[c] = 0.f;
  }
  constexpr int TK = P::kTK, KR = P::kKR;
  // a chunk is TK complex K (KIND 0, 2) or KR real bands (KIND 1)
  const int nchunks = KIND == 1 ? (gK + KR - 1) / KR : (gK + TK - 1) / TK;
  // Staging is software-pipelined: chunk ch + 1's operands are loaded from
  // global memory into registers while chunk ch's MMAs run, then split and
  // stored to shared memory once those MMAs are done with the tiles.
  // A tile: rows m0..m0+127, complex k0..k0+TK-1 -> real kk = k (re), k + TK
  // (im).  Element e of a tile: a warp covers 8 rows x 4 k, so its 32 stores
  // hit 32 distinct banks of a core-matrix row group and its loads are four
  // 64-byte runs of a column.  B tiles (output columns n0..n0+63): row n holds
  // op(B)(k, n) over k, 8 rows n x 4 k per warp (loads are runs of 4 k,
  // B(k, n) at k + ldb n, or of 8 n, B(n, k) at n + ldb k).
  constexpr int kPa = TM * TK / kThreads, kPb = TN * TK / kThreads;
  float2 ra[kPa], rb[kPb] = {};
  // KIND 1 with a second cube: its raw values, combined (x - ycoef y) only when
  // the chunk is stored, so that the loads stay in flight meanwhile.  The DFT
  // kinds' B operand (twiddles from a table of n3 entries that stays in L1) is
  // read when the chunk is stored, not held in registers across the pipeline.
  float2 ry[KIND == 1 ? kPa : 1] = {};
  // 3xBF16: a thread takes two consecutive k of one row (items i, i + 1 with
  // i even), so that each hi or lo store is one 4-byte word of two halves and
  // a warp's 32 words (8 rows x 4 k pairs) again fall in 32 distinct banks
  auto a_pos = [&](int i, int &r, int &kc) {
    const int e = tid + kThreads * (PREC ? i >> 1 : i), rest = e >> 5;
    r = ((rest % (TM / 8)) << 3) | ((e >> 2) & 7);
    kc = ((rest / (TM / 8)) << 2) | (e & 3);
    if (PREC) kc = (kc << 1) | (i & 1);
  };
  auto b_pos = [&](int i, int &n, int &kc) {
    const int e = tid + kThreads * (PREC ? i >> 1 : i), rest = e >> 5;
    n = ((rest % (TN / 8)) << 3) | ((e >> 2) & 7);
    kc = ((rest / (TN / 8)) << 2) | (e & 3);
    if (PREC) kc = (kc << 1) | (i & 1);
  };
  // the raw value of cube q at pixel gm, band c (0 outside the cube)
  auto cval = [&](const float *q, int gm, int c) -> float {
    return (gm < gM && c < gK) ? q[(size_t)gm + f.P * c] : 0.0f;
  };
  // exp(-2 pi i k c / n3) (0 outside the half spectrum or the bands)
  auto twid = [&](int k, int c) -> float2 {
    if (k >= f.h || c >= f.n3) return make_float2(0.f, 0.f);
    return f.tw3[(unsigned)(k * c) % (unsigned)f.n3];
  };
  auto load_chunk = [&](int k0) {
    if constexpr (KIND == 1) {
#pragma unroll
      for (int i = 0; i < kPa; ++i) {
        int r, kc;
        a_pos(i, r, kc);
        ra[i] = make_float2(cval(xb, m0 + r, k0 + kc), cval(xb, m0 + r, k0 + TK + kc));
        if (yb)
          ry[KIND == 1 ? i : 0] =
              make_float2(cval(yb, m0 + r, k0 + kc), cval(yb, m0 + r, k0 + TK + kc));
      }
    } else {
#pragma unroll
      for (int i = 0; i < kPa; ++i) {
        int r, kc;
        a_pos(i, r, kc);
        const int gm = m0 + r, gk = k0 + kc;
        if (KIND == 2) {  // raw; conjugated (transposed slices) when stored
          ra[i] = (gm < gM && gk < gK) ? specb[wpos(gm) + f.P * gk] : make_float2(0.f, 0.f);
        } else if (OPB == 2) {  // A^H(m, k) = conj A(k, m)
          float2 v = make_float2(0.f, 0.f);
          if (gm < g.M && gk < g.K) {
            v = A[gk + (size_t)g.lda * gm];
            v.y = -v.y;
          }
          ra[i] = v;
        } else {
          ra[i] = (gm < g.M && gk < g.K) ? A[gm + (size_t)g.lda * gk] : make_float2(0.f, 0.f);
        }
      }
      if (KIND == 0) {
#pragma unroll
        for (int i = 0; i < kPb; ++i) {
          int n, kc;
          b_pos(i, n, kc);
          const int gn = n0 + n, gk = k0 + kc;
          float2 v = make_float2(0.f, 0.f);
          if (gn < g.N && gk < g.K) {
            v = OPB != 1 ? B[gk + (size_t)g.ldb * gn] : B[gn + (size_t)g.ldb * gk];
            if (OPB == 1) v.y = -v.y;
          }
          rb[i] = v;
        }
      }
    }
  };
  // B item i of the chunk at k0: (v, w) = KIND 0 the loaded op(B) value (w
  // unused); KIND 1 the twiddles of bands k0 + kc and k0 + TK + kc; KIND 2
  // w_k exp(+2 pi i k c / n3) of frequency k0 + kc (w unused)
  auto bval = [&](int i, int k0, float2 &v, float2 &w) {
    int n, kc;
    b_pos(i, n, kc);
    if (KIND == 0) {
      v = rb[i];
    } else if (KIND == 1) {
      v = twid(n0 + n, k0 + kc);
      w = twid(n0 + n, k0 + TK + kc);
    } else {
      const int gn = n0 + n, gk = k0 + kc;
      v = make_float2(0.f, 0.f);
      if (gn < gN && gk < gK) {
        const float2 t = f.tw3[(unsigned)(gk * gn) % (unsigned)f.n3];
        const float wk = (gk == 0 || 2 * gk == f.n3) ? 1.0f : 2.0f;
        v = make_float2(wk * t.x, -wk * t.y);
      }
    }
  };
  // split the registers' chunk into the hi / lo tiles of stage `st`
  auto store_chunk = [&](int st, int k0) {
    char *aHi = smem + st * kStageBytes, *aLo = aHi + P::kTileA;
    // [Re | Im] B tiles of each split adjacent: one 128-row B operand
    char *bReHi = aLo + P::kTileA, *bImHi = bReHi + P::kTileB;
    char *bReLo = bImHi + P::kTileB, *bImLo = bReLo + P::kTileB;
    // the A values as the MMAs take them: KIND 1 x - ycoef y, KIND 2 the
    // conjugate on transposed slices
    auto aval = [&](int i) -> float2 {
      float2 v = ra[i];
      if (KIND == 1 && yb) {
        const float2 w = ry[KIND == 1 ? i : 0];
        v = make_float2(v.x - f.ycoef * w.x, v.y - f.ycoef * w.y);
      }
      if (KIND == 2 && f.trans) v.y = -v.y;
      return v;
    };
    if (PREC == 0) {
#pragma unroll
      for (int i = 0; i < kPa; ++i) {
        int r, kc;
        a_pos(i, r, kc);
        const float2 v = aval(i);
        put_split<PREC>(aHi, aLo, koff<PREC>(r, kc), v.x);
        put_split<PREC>(aHi, aLo, koff<PREC>(r, kc + TK), v.y);
      }
#pragma unroll
      for (int i = 0; i < kPb; ++i) {
        int n, kc;
        b_pos(i, n, kc);
        float2 v, w;
        bval(i, k0, v, w);
        if (KIND == 1) {  // real and imaginary twiddle parts of the chunk's bands
          put_split<PREC>(bReHi, bReLo, koff<PREC>(n, kc), v.x);
          put_split<PREC>(bReHi, bReLo, koff<PREC>(n, kc + TK), w.x);
          put_split<PREC>(bImHi, bImLo, koff<PREC>(n, kc), v.y);
          put_split<PREC>(bImHi, bImLo, koff<PREC>(n, kc + TK), w.y);
          continue;
        }
        put_split<PREC>(bReHi, bReLo, koff<PREC>(n, kc), v.x);  // [Re B | -Im B]
        put_split<PREC>(bReHi, bReLo, koff<PREC>(n, kc + TK), -v.y);
        if (KIND == 2) continue;  // Re C only
        put_split<PREC>(bImHi, bImLo, koff<PREC>(n, kc), v.y);  // [Im B | Re B]
        put_split<PREC>(bImHi, bImLo, koff<PREC>(n, kc + TK), v.x);
      }
    } else {
#pragma unroll
      for (int i = 0; i < kPa; i += 2) {  // k pairs (kc even, kc + 1)
        int r, kc;
        a_pos(i, r, kc);
        const float2 v0 = aval(i), v1 = aval(i + 1);
        put_split2(aHi, aLo, koff<PREC>(r, kc), v0.x, v1.x);
        put_split2(aHi, aLo, koff<PREC>(r, kc + TK), v0.y, v1.y);
      }
#pragma unroll
      for (int i = 0; i < kPb; i += 2) {
        int n, kc;
        b_pos(i, n, kc);
        float2 v0, v1, w0, w1;
        bval(i, k0, v0, w0);
        bval(i + 1, k0, v1, w1);
        if (KIND == 1) {
          put_split2(bReHi, bReLo, koff<PREC>(n, kc), v0.x, v1.x);
          put_split2(bReHi, bReLo, koff<PREC>(n, kc + TK), w0.x, w1.x);
          put_split2(bImHi, bImLo, koff<PREC>(n, kc), v0.y, v1.y);
          put_split2(bImHi, bImLo, koff<PREC>(n, kc + TK), w0.y, w1.y);
          continue;
        }
        put_split2(bReHi, bReLo, koff<PREC>(n, kc), v0.x, v1.x);  // [Re B | -Im B]
        put_split2(bReHi, bReLo, koff<PREC>(n, kc + TK), -v0.y, -v1.y);
        if (KIND == 2) continue;  // Re C only
        put_split2(bImHi, bImLo, koff<PREC>(n, kc), v0.y, v1.y);  // [Im B | Re B]
        put_split2(bImHi, bImLo, koff<PREC>(n, kc + TK), v0.x, v1.x);
      }
    }
  };
  // one thread: the chunk's MMAs on stage `st` into a fresh TMEM tile `st`,
  // committed to barrier `st`
  auto issue = [&](int st) {
    const char *base = smem + st * kStageBytes;
    const uint32_t a_hi = smem_u32(base), a_lo = a_hi + (uint32_t)P::kTileA;
    const uint32_t b_hi = a_lo + (uint32_t)P::kTileA, b_lo = b_hi + 2 * (uint32_t)P::kTileB;
    const uint32_t dt = tmem + (uint32_t)st * (2 * TN);
#pragma unroll
    for (int j = 0; j < KR / P::kMmaK; ++j) {  // one instruction spans two core matrices
      const uint32_t ko = (uint32_t)j * 2 * kLBO;
      const uint32_t acc0 = j > 0 ? 1u : 0u;  // a fresh tile per chunk
      // Re C (tile columns 0..63) and Im C (64..127) from one N = 128 MMA over
      // the adjacent [Re | Im] B tiles, so that A is read once for both; the
      // real part alone (KIND 2) from N = 64.  Three split products each.
      const uint32_t id = KIND == 2 ? idesc : idesc2;
      mma<PREC>(dt, sdesc<PREC>(a_hi + ko), sdesc<PREC>(b_hi + ko), id, acc0);
      mma<PREC>(dt, sdesc<PREC>(a_hi + ko), sdesc<PREC>(b_lo + ko), id, 1u);
      mma<PREC>(dt, sdesc<PREC>(a_lo + ko), sdesc<PREC>(b_hi + ko), id, 1u);
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            st ? bar1 : bar0));
  };
  auto mark_issued = [&](int st) {
    if (st) out1 = true;
    else out0 = true;
  };
  // add TMEM tile `st` into the FP32 register accumulators
  auto drain = [&](int st) {
    const uint32_t tile = (uint32_t)st * (2 * TN);
#pragma unroll
    for (int c0 = 0; c0 < TN / 2; c0 += 16) {
      uint32_t re[16], im[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(re[0]), "=r"(re[1]), "=r"(re[2]), "=r"(re[3]), "=r"(re[4]), "=r"(re[5]),
            "=r"(re[6]), "=r"(re[7]), "=r"(re[8]), "=r"(re[9]), "=r"(re[10]), "=r"(re[11]),
            "=r"(re[12]), "=r"(re[13]), "=r"(re[14]), "=r"(re[15])
          : "r"(tl + tile + c0));
      if (KIND == 1) {
        // the real parts first: half the destination registers live at once,
        // which leaves room for the next chunk's loads of both cubes
        asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
        for (int c = 0; c < 16; ++c) accRe[c0 + c] += __uint_as_float(re[c]);
      }
      if (KIND != 2)
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(im[0]), "=r"(im[1]), "=r"(im[2]), "=r"(im[3]), "=r"(im[4]), "=r"(im[5]),
              "=r"(im[6]), "=r"(im[7]), "=r"(im[8]), "=r"(im[9]), "=r"(im[10]), "=r"(im[11]),
              "=r"(im[12]), "=r"(im[13]), "=r"(im[14]), "=r"(im[15])
            : "r"(tl + tile + TN + c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        if (KIND != 1) accRe[c0 + c] += __uint_as_float(re[c]);
        if (KIND != 2) accIm[c0 + c] += __uint_as_float(im[c]);
      }
    }
    // the tile is rewritten only after every thread's reads
    asm volatile("tcgen05.fence::before_thread_sync;");
  };
  // every thread waits for the MMAs committed to barrier `st`; on a timeout
  // the commit stays outstanding for the last bounded wait before the free
  auto wait_mmas = [&](int st) {
    const bool done = mbar_wait(st ? bar1 : bar0, st ? ph1 : ph0);
    if (done) {
      if (st) {
        ph1 ^= 1u;
        out1 = false;
      } else {
        ph0 ^= 1u;
        out0 = false;
      }
    } else {
      ok = false;
      if (tid == 0) s_ok = 0;
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
  };
  auto stage_barrier = [&]() {
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
  };
  if (nchunks > 0) load_chunk(0);
  // chunk ch: stage s = ch & 1 is written while chunk ch - 1's MMAs (stage
  // s ^ 1) run; once those are done, chunk ch's MMAs are issued and chunk
  // ch - 1's tile is drained while they run
  for (int ch = 0; ch < nchunks && ok; ++ch) {
    const int st = ch & 1;
    store_chunk(st, ch * (KIND == 1 ? KR : TK));  // stage st was last read by chunk ch - 2
    if (ch + 1 < nchunks) load_chunk((ch + 1) * (KIND == 1 ? KR : TK));
    stage_barrier();
    if (ch > 0) {
      wait_mmas(st ^ 1);
      __syncthreads();
      ok = ok && s_ok;
      if (!ok) break;
    }
    if (tid == 0) issue(st);
    mark_issued(st);
    if (ch > 0) drain(st ^ 1);
  }
  if (ok && nchunks > 0) {
    const int last = (nchunks - 1) & 1;
    wait_mmas(last);
    __syncthreads();
    ok = ok && s_ok;
    if (ok) drain(last);
  }
  if (!ok) {
    if (tid == 0 && err) atomicExch(err, 1);
    // give MMAs still in flight a last bounded chance to land before the free
    if (out0) mbar_wait(bar0, ph0);
    if (out1) mbar_wait(bar1, ph1);
  } else if (nchunks > 0) {
    // epilogue: thread (warp w, lane l) owns row m0 + 32 (w mod 4) + l of the
    // tile, columns colh .. colh + 31
    const int gm = m0 + row;
    const int lb = g.lam3_period > 0 ? b % g.lam3_period : b;
    if (KIND == 1 && gm < gM) {
      float2 *ob = f.spec_out + (size_t)b * f.h * f.P + wpos(gm);
#pragma unroll
      for (int c = 0; c < TN / 2; ++c) {
        const int n = n0 + colh + c;
        if (n >= gN) break;
        ob[f.P * n] = make_float2(accRe[c], f.trans ? -accIm[c] : accIm[c]);
      }
    } else if (KIND == 2 && gm < gM) {
      const float inv = 1.0f / (float)f.n3;
      const size_t base = (size_t)b * f.N + gm;
      const bool g4 = f.mode == 1 && f.gamma4;
      // eight columns at a time: their Gamma4 and F loads are issued together
      // before any is used
#pragma unroll
      for (int c0 = 0; c0 < TN / 2; c0 += 8) {
        float g[8], fv[8];
        if (g4) {
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const int n = n0 + colh + c0 + c;
            const bool in = n < gN;
            const size_t v = base + f.P * (in ? n : 0);
            g[c] = in ? f.G4[v] : 0.0f;
            fv[c] = in ? f.F[v] : 0.0f;
          }
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int n = n0 + colh + c0 + c;
          if (n >= gN) break;
          const size_t v = base + f.P * n;
          const float r = accRe[c0 + c] * inv;
          f.out[v] = r;
          if (g4) f.G4[v] = g[c] + f.mu * (r - fv[c]);
        }
      }
    } else if (KIND == 0 && gm < g.M) {
#pragma unroll
      for (int c = 0; c < TN / 2; ++c) {
        const int n = n0 + colh + c;
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(kCols));
}

// Checks the GEMM's bounded barrier wait and its timeout path: one warp
// allocates tensor memory as the GEMM does, then waits on an mbarrier with
// the wait cut to `tries` tries.  With `arrive`, lane 0 arrives first and the
// phase completes; without, nothing arrives and the wait runs out.  A timeout
// is recorded in out[0]; the tensor memory is freed on both paths, and
// out[1] counts the lanes that got past the free.
__global__ void __launch_bounds__(32) k_wait_probe(long long tries, int arrive, int *out) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t slot;
  const uint32_t b = smem_u32(&bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(
                   smem_u32(&slot)));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = slot;
  if (arrive && threadIdx.x == 0)
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(b)
                 : "memory");
  __syncwarp();
  if (!mbar_wait(b, 0u, tries)) atomicOr(out, 1);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem));
  atomicAdd(out + 1, 1);
}

// Tensor-pipe throughput probe: one CTA per SM, one thread issuing n_mma
// MMAs of M = 128, N = 256 (K = 8 TF32 or 16 BF16 per instruction) from
// shared-memory tiles into two alternating TMEM accumulators, then one
// commit and a bounded wait.  The tiles hold a fixed non-zero pattern (the
// tensor core's power, and so its clock under the power cap, depends on the
// data).  A wait that runs out sets *err; tensor memory is freed either way.
constexpr int kProbeN = 256;
constexpr size_t kProbeSmem = 120 * 1024;  // more than half the SM's shared memory: one CTA per SM

template <int PREC>
__global__ void __launch_bounds__(128, 1) k_mma_peak(long long n_mma, int *err) {
  extern __shared__ __align__(1024) char smem[];
  using P = Prec<PREC>;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const size_t tile_bytes = (size_t)(TM + kProbeN) * P::kKR * P::kBytes;
  for (size_t e = tid; e < tile_bytes / 4; e += blockDim.x) {
    const uint32_t h = (uint32_t)e * 2654435761u;
    const float x = 0.25f + (float)(h >> 9) * (1.0f / 16777216.0f);  // in [0.25, 1.25)
    if (PREC == 0) {
      ((float *)smem)[e] = tf32_hi(x);
    } else {
      __nv_bfloat162 v = __floats2bfloat162_rn(x, 1.5f - x);
      ((__nv_bfloat162 *)smem)[e] = v;
    }
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
        smem_u32(&tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tslot;
  const uint32_t idesc = (1u << 4) | (P::kFmt << 7) | (P::kFmt << 10) |
                         ((uint32_t)(kProbeN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
  const uint32_t bar = smem_u32(&mbar);
  if (tid == 0) {
    const uint64_t a = sdesc<PREC>(smem_u32(smem));
    const uint64_t b = sdesc<PREC>(smem_u32(smem + (size_t)TM * P::kKR * P::kBytes));
    for (long long i = 0; i < n_mma; ++i)
      mma<PREC>(tmem + (uint32_t)(i & 1) * kProbeN, a, b, idesc, i > 1 ? 1u : 0u);
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar));
  }
  __syncwarp();
  if (!mbar_wait(bar, 0u) && tid == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

template <int PREC>
size_t smem_bytes() {
  return 2 * (2 * Prec<PREC>::kTileA + 4 * Prec<PREC>::kTileB);
}

template <int OPB, int EPI, int PREC>
cudaError_t launch_one(const CGemm &g, int *err, cudaStream_t st) {
  const size_t smem = smem_bytes<PREC>();
  cudaError_t e = cudaFuncSetAttribute(k_cgemm_tc<OPB, EPI, PREC>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((g.M + TM - 1) / TM, (g.N + TN - 1) / TN, g.batch);
  k_cgemm_tc<OPB, EPI, PREC><<<grid, kThreads, smem, st>>>(g, Dft3{}, err);
  return cudaGetLastError();
}

template <int KIND, int PREC>
cudaError_t launch_dft(const Dft3 &f, int nb, int *err, cudaStream_t st) {
  const size_t smem = smem_bytes<PREC>();
  cudaError_t e = cudaFuncSetAttribute(k_cgemm_tc<0, 0, PREC, KIND>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const size_t mt = (f.P + TM - 1) / TM;
  const size_t nt = ((KIND == 1 ? f.h : f.n3) + TN - 1) / TN;
  dim3 grid((unsigned)(mt * nt), 1, nb);
  k_cgemm_tc<0, 0, PREC, KIND><<<grid, kThreads, smem, st>>>(CGemm{}, f, err);
  return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_prec(const CGemm &g, int *err, cudaStream_t st) {
  if (g.opA == 1) {  // A^H B only
    if (g.opB == 0 && g.epi == 0) return launch_one<2, 0, PREC>(g, err, st);
    return cudaErrorInvalidValue;
  }
  if (g.opB == 0 && g.epi == 0) return launch_one<0, 0, PREC>(g, err, st);
  if (g.opB == 0 && g.epi == 1) return launch_one<0, 1, PREC>(g, err, st);
  if (g.opB == 1 && g.epi == 0) return launch_one<1, 0, PREC>(g, err, st);
  return cudaErrorInvalidValue;
}

}  // namespace

size_t cgemm_tc_smem() { return smem_bytes<0>(); }

long long cgemm_tc_wait_limit() { return kWaitLimit; }

cudaError_t launch_wait_probe(long long tries, int arrive, int *out, cudaStream_t st) {
  k_wait_probe<<<1, 32, 0, st>>>(tries, arrive, out);
  return cudaGetLastError();
}

cudaError_t launch_mma_peak(int prec, int nsm, long long n_mma, int *err, cudaStream_t st,
                            double *flops) {
  const double per = 2.0 * TM * kProbeN * (prec ? 16 : 8);
  *flops = per * (double)n_mma * nsm;
  if (prec == 0) {
    cudaError_t e = cudaFuncSetAttribute(k_mma_peak<0>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kProbeSmem);
    if (e != cudaSuccess) return e;
    k_mma_peak<0><<<nsm, 128, kProbeSmem, st>>>(n_mma, err);
  } else {
    cudaError_t e = cudaFuncSetAttribute(k_mma_peak<1>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kProbeSmem);
    if (e != cudaSuccess) return e;
    k_mma_peak<1><<<nsm, 128, kProbeSmem, st>>>(n_mma, err);
  }
  return cudaGetLastError();
}

cudaError_t launch_dft3_tc(int kind, const Dft3 &f, int nb, int *err, cudaStream_t st, int prec) {
  if (f.P == 0 || nb <= 0) return cudaSuccess;
  if (f.P > (size_t)TM * 0x7fffffff / 4) return cudaErrorInvalidValue;
  if (kind == 1) return prec ? launch_dft<1, 1>(f, nb, err, st) : launch_dft<1, 0>(f, nb, err, st);
  if (kind == 2) return prec ? launch_dft<2, 1>(f, nb, err, st) : launch_dft<2, 0>(f, nb, err, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_cgemm_tc(const CGemm &g, int *err, cudaStream_t st, int prec) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  if (g.epi == 2) return cudaErrorInvalidValue;  // SIMT kernel only
  if (prec == 0) return launch_prec<0>(g, err, st);
  if (prec == 1) return launch_prec<1>(g, err, st);
  return cudaErrorInvalidValue;
}

}  // namespace lrstv
