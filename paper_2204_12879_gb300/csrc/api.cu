// api.cu -- the C ABI of include/lrstv.h: plans, the ADMM iteration of
// arXiv 2204.12879 (Algorithm 1 with the full-rank L-update) as a sequence of
// stream-ordered kernel launches, optional CUDA-graph replay of whole runs,
// state import/export, and the standalone operators.
#include <math.h>
#include <new>
#include <stdlib.h>
#include <string.h>

#include "lrstv.h"
#include "lrstv_internal.cuh"

namespace lrstv {

Dims make_dims(int n1, int n2, int n3) {
  Dims d;
  d.n1 = n1;
  d.n2 = n2;
  d.n3 = n3;
  d.P = (size_t)n1 * n2;
  d.N = d.P * n3;
  d.h = n3 / 2 + 1;
  d.trans = n1 < n2 ? 1 : 0;
  d.nr = n1 >= n2 ? n1 : n2;
  d.nc = n1 >= n2 ? n2 : n1;
  return d;
}

void carve_tables(Carver &c, const Dims &d, Tables &t) {
  t.tw3 = c.take<float2>(d.n3);
  t.F1 = c.take<float2>((size_t)d.n1 * d.n1);
  t.G1 = c.take<float2>((size_t)d.n1 * d.n1);
  t.F2 = c.take<float2>((size_t)d.n2 * d.n2);
  t.G2 = c.take<float2>((size_t)d.n2 * d.n2);
  t.lam1 = c.take<float>(d.n1);
  t.lam2 = c.take<float>(d.n2);
  t.lam3 = c.take<float>(d.n3);
}

int check_shape(int n1, int n2, int n3) {
  if (n1 < 1 || n2 < 1 || n3 < 1) return LRSTV_ERR_ARG;
  if (n1 > kMaxSpatial || n2 > kMaxSpatial) return LRSTV_ERR_SHAPE;
  if (n3 > kMaxBands) return LRSTV_ERR_SHAPE;  // the mode-3 DFTs' twiddle indices k c < 2^24
  if ((double)n1 * n2 * n3 * 3.0 > 2.0e9) return LRSTV_ERR_SHAPE;  // 3N fits a 32-bit grid walk
  return LRSTV_OK;
}

namespace {

constexpr int kResRing = 4096;     // per-iteration residual history
// SMs a plan's task-graph Jacobi leaves to the side stream, which runs the
// next iteration's L-update and Z-solve while the E-step's Jacobi runs.  The
// Jacobi's time follows the SMs it has (200 x 200 x 80: 5.05 ms on 152 SMs,
// 5.52 on 136), while the side stream's work, once the Jacobi's CTAs have
// left, takes a fraction of a millisecond on the whole GPU: 16 spare SMs gave
// 155.4 iterations/s against 163.9 with none, so none are kept.
constexpr int kJacobiSpareSMs = 0;

int check_params(const lrstv_params *p) {
  if (!p) return LRSTV_ERR_ARG;
  const float v[] = {p->tau, p->alpha, p->lambda, p->w[0], p->w[1], p->w[2], p->mu0, p->rho,
                     p->mu_max};
  for (float x : v)
    if (!isfinite(x) || x < 0.0f) return LRSTV_ERR_ARG;
  if (!(p->mu0 > 0.0f) || !(p->mu_max >= p->mu0) || p->max_iter < 0) return LRSTV_ERR_ARG;
  if (p->flags & ~(unsigned)(LRSTV_FLAG_F_THRESH_EXACT | LRSTV_FLAG_NO_GAMMA4 | LRSTV_FLAG_GRAPH |
                             LRSTV_FLAG_STRICT | LRSTV_FLAG_SIMT_GEMM | LRSTV_FLAG_WARM_START |
                             LRSTV_FLAG_SIMT_DFT | LRSTV_FLAG_JACOBI_PER_SLICE |
                             LRSTV_FLAG_ISO_TV | LRSTV_FLAG_BF16X3 | LRSTV_FLAG_JACOBI_PANEL16 |
                             LRSTV_FLAG_JACOBI_FIXED_ORDER))
    return LRSTV_ERR_ARG;
  // the split-BF16 products exist on the tensor-core path only
  if ((p->flags & LRSTV_FLAG_BF16X3) && (p->flags & LRSTV_FLAG_SIMT_GEMM)) return LRSTV_ERR_ARG;
  return LRSTV_OK;
}

}  // namespace

// Per-launch CUDA-event bracketing for lrstv_profile_* (off unless enabled).
struct Prof {
  static constexpr int kCap = 4096;
  int on = 0;
  int n = 0;
  cudaEvent_t *ev = nullptr;  // 2 kCap events, created on first enable
  unsigned char cls[kCap];
  unsigned long long *d_work = nullptr;  // Jacobi [pairs, rotations], in the plan arena
};

// Records a begin event now and an end event when it goes out of scope,
// around exactly one launch; skipped while `st` is being captured.
struct Span {
  Prof *p = nullptr;
  int idx = -1;
  cudaStream_t st;
  Span(Prof *prof, int cls, cudaStream_t s) : st(s) {
    if (!prof || !prof->on || prof->n >= Prof::kCap) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
      cudaGetLastError();
      return;
    }
    p = prof;
    idx = p->n++;
    p->cls[idx] = (unsigned char)cls;
    cudaEventRecord(p->ev[2 * idx], s);
  }
  ~Span() {
    if (p) cudaEventRecord(p->ev[2 * idx + 1], st);
  }
};

namespace {

cudaError_t gemm_z(const CGemm &g, cudaStream_t st, Prof *prof, GemmSel gs) {
  Span sp(prof, LRSTV_K_CGEMM_Z, st);
  return gemm(g, gs, st);
}

}  // namespace

cudaError_t gemm(const CGemm &g, GemmSel gs, cudaStream_t st) {
  return gs.tc ? launch_cgemm_tc(g, gs.err, st, gs.prec) : launch_cgemm(g, st);
}

// Z-solve of nb cubes on their h half-spectrum slices each: specA <- fftn(T)
// / (mu (1 + P_z)) -> ifftn -> Z.  specA, specB: nb h P complex each.
cudaError_t zsolve_core(const Dims &d, int nb, const Tables &tb, const float *T, float mu,
                        float *Z, float2 *specA, float2 *specB, cudaStream_t st, Prof *prof,
                        GemmSel gs) {
  cudaError_t e;
  {
    Span sp(prof, LRSTV_K_R2C_Z, st);
    e = launch_r2c3(d, nb, T, nullptr, 0.0f, specA, 0, tb.tw3, st, gs);
  }
  if (e != cudaSuccess) return e;
  CGemm g{};
  g.M = d.n1;
  g.N = d.n2;
  g.batch = nb * d.h;
  g.lam3_period = d.h;
  g.lda = d.n1;
  g.ldc = d.n1;
  g.sC = (long long)d.P;
  // mode 1: specB_k = F1 specA_k
  g.A = tb.F1; g.sA = 0; g.B = specA; g.sB = (long long)d.P; g.ldb = d.n1; g.K = d.n1;
  g.C = specB; g.opB = 0; g.epi = 0;
  if ((e = gemm_z(g, st, prof, gs)) != cudaSuccess) return e;
  // mode 2 + spectral division: specA_k = (specB_k F2) / (mu (1 + P_z)) / (n1 n2)
  g.A = specB; g.sA = (long long)d.P; g.B = tb.F2; g.sB = 0; g.ldb = d.n2; g.K = d.n2;
  g.C = specA; g.epi = 1; g.lam1 = tb.lam1; g.lam2 = tb.lam2; g.lam3 = tb.lam3; g.mu = mu;
  g.scale = (float)(1.0 / ((double)d.n1 * (double)d.n2));
  if ((e = gemm_z(g, st, prof, gs)) != cudaSuccess) return e;
  // inverse mode 1 and mode 2
  g.epi = 0;
  g.A = tb.G1; g.sA = 0; g.B = specA; g.sB = (long long)d.P; g.ldb = d.n1; g.K = d.n1; g.C = specB;
  if ((e = gemm_z(g, st, prof, gs)) != cudaSuccess) return e;
  g.A = specB; g.sA = (long long)d.P; g.B = tb.G2; g.sB = 0; g.ldb = d.n2; g.K = d.n2; g.C = specA;
  if ((e = gemm_z(g, st, prof, gs)) != cudaSuccess) return e;
  Span sp(prof, LRSTV_K_C2R_Z, st);
  return launch_c2r3(d, nb, specA, 0, tb.tw3, Z, 0, nullptr, nullptr, 0.0f, 0, st, gs);
}

namespace {

// t-SVT of nb cubes x_b - ycoef y_b with threshold t, in three phases:
// DFT along mode 3 into the working orientation (tsvt_pre), Jacobi + g-scaling
// (tsvt_jac), W V^H and the inverse DFT (tsvt_post).
cudaError_t tsvt_pre(const Dims &d, int nb, const float *x, const float *y, float ycoef,
                     const float2 *tw3, float2 *specA, cudaStream_t st, Prof *prof,
                     GemmSel gs = kSimt) {
  Span sp(prof, LRSTV_K_R2C_E, st);
  return launch_r2c3(d, nb, x, y, ycoef, specA, 1, tw3, st, gs);
}

// ms2 (may be null): nb floats for the tensors' largest mean-square column
// norms, which then set the threshold-aware tolerance tensor by tensor.
cudaError_t tsvt_jac(const Dims &d, int nb, float t, float2 *specA, float2 *V, int *sweeps,
                     cudaStream_t st, Prof *prof, float *ms2 = nullptr, int *sched = nullptr,
                     int pw = 32, int *order = nullptr, int sort = 1) {
  if (ms2) {
    cudaError_t e = launch_group_ms2(d, nb * d.h, specA, d.h, ms2, st);
    if (e != cudaSuccess) return e;
  }
  JacOpt o;
  o.t_svt = t;
  o.ms2 = ms2;
  o.group = d.h;
  o.sched = sched;
  o.spare_sms = sched ? kJacobiSpareSMs : 0;
  o.pw = pw;
  o.order = order;
  o.sort = sort;
  Span sp(prof, LRSTV_K_JACOBI, st);
  return launch_jacobi(d, nb * d.h, specA, V, t, kMaxSweeps, sweeps, prof ? prof->d_work : nullptr,
                       st, o);
}

cudaError_t tsvt_post(const Dims &d, int nb, float *out, int mode, float *G4, const float *F,
                      float mu, int gamma4, const float2 *tw3, float2 *specA, float2 *specB,
                      float2 *V, cudaStream_t st, Prof *prof, GemmSel gs = kSimt) {
  const int ns = nb * d.h;
  CGemm g{};
  g.A = specA; g.sA = (long long)d.P; g.lda = d.nr;
  g.B = V; g.sB = (long long)d.nc * d.nc; g.ldb = d.nc; g.opB = 1;
  g.C = specB; g.sC = (long long)d.P; g.ldc = d.nr;
  g.M = d.nr; g.N = d.nc; g.K = d.nc; g.batch = ns; g.epi = 0;
  cudaError_t e;
  {
    Span sp(prof, LRSTV_K_CGEMM_E, st);
    e = gemm(g, gs, st);
  }
  if (e != cudaSuccess) return e;
  Span sp(prof, LRSTV_K_C2R_E, st);
  return launch_c2r3(d, nb, specB, 1, tw3, out, mode, G4, F, mu, gamma4, st, gs);
}

cudaError_t tsvt_core(const Dims &d, int nb, const float *x, const float *y, float ycoef, float t,
                      float *out, int mode, float *G4, const float *F, float mu, int gamma4,
                      const float2 *tw3, float2 *specA, float2 *specB, float2 *V, int *sweeps,
                      cudaStream_t st, Prof *prof = nullptr, GemmSel gs = kSimt,
                      float *ms2 = nullptr, int *sched = nullptr, int pw = 32,
                      int *order = nullptr, int sort = 1) {
  cudaError_t e = tsvt_pre(d, nb, x, y, ycoef, tw3, specA, st, prof, gs);
  if (e != cudaSuccess) return e;
  if ((e = tsvt_jac(d, nb, t, specA, V, sweeps, st, prof, ms2, sched, pw, order, sort)) !=
      cudaSuccess)
    return e;
  return tsvt_post(d, nb, out, mode, G4, F, mu, gamma4, tw3, specA, specB, V, st, prof, gs);
}

}  // namespace

// Standalone t-SVT on caller-provided scratch pieces (no profiling, cold
// Jacobi start): used by the allocation-free entry point.
cudaError_t tsvt_plain(const Dims &d, const float *A, float t, float *out, float2 *tw3,
                       float2 *specA, float2 *specB, float2 *V, int *sweeps, cudaStream_t st) {
  cudaError_t e = launch_tw3(d.n3, tw3, st);
  if (e != cudaSuccess) return e;
  return tsvt_core(d, 1, A, nullptr, 0.0f, t, out, 0, nullptr, nullptr, 0.0f, 0, tw3, specA,
                   specB, V, sweeps, st, nullptr);
}

}  // namespace lrstv

using namespace lrstv;

struct lrstv_plan {
  Dims d;
  lrstv_params prm;
  double mu;
  int iter;
  void *arena;
  size_t arena_bytes;
  int own_arena;  // 0: the plan is one of a batch group's, whose memory the batch owns
  float *Y, *L, *Z, *S, *G1, *G2, *F, *E, *G3, *G4, *T;
  float2 *specA, *specB, *V;
  float2 *Vs;     // V diag g for the reconstruction (warm start keeps V itself)
  float *ms2;     // per gradient tensor: largest mean-square column norm of its slices
  int vwarm;      // V holds the last E-step's right singular vectors
  Tables tb;
  unsigned *res;  // kResRing x 2 residual maxima (float bits)
  int *sweeps;    // 3h
  int *order;     // 3h: the one-CTA-per-slice Jacobi's slice order
  int *gcand, *gconv;  // 3h each: the tensor-core Gram check's candidates and flags
  int *jsched;    // task-graph Jacobi scratch (jacobi_task_ints(3h))
  int *gemm_err;  // tensor-core GEMM wait timeouts
  // graph cache for lrstv_plan_run
  cudaGraphExec_t gexec;
  const void *gY;
  void *gX, *gS;
  int giters;
  cudaStream_t cap_stream;
  // iterate_async runs the next iteration's L/T_z and Z-solve (which do not
  // read E) on `side` while the current E-step runs: Z-solve scratch of its own
  cudaStream_t side;
  cudaEvent_t ev_fs, ev_side;
  float2 *zA, *zB;
  // ... and, with the warm start, the next E-step's Newton-Schulz step on V,
  // as soon as the current E-step has read V (ns_req: schedule it; ns_ready:
  // V has had it, after ev_ns; Vn1, Vn2: its products)
  cudaEvent_t ev_sig, ev_ns;
  float2 *Vn1, *Vn2;
  int ns_req, ns_ready;
  // Tucker (HOOI) L-update of the full TDLRSTV model (lrstv_plan_set_tucker)
  int tucker;
  void *tk_mem;
  TuckerWs tk;
  Prof prof;
};

#define CK(x)                                   \
  do {                                          \
    if ((x) != cudaSuccess) return LRSTV_ERR_CUDA; \
  } while (0)

namespace {

// The task-graph Jacobi's scratch, or null for one CTA per slice.
int *plan_sched(const lrstv_plan *pl) {
  return (pl->prm.flags & LRSTV_FLAG_JACOBI_PER_SLICE) ? nullptr : pl->jsched;
}

// The packed Jacobi's panel width for a plan's flags.
int plan_pw(const lrstv_plan *pl) { return (pl->prm.flags & LRSTV_FLAG_JACOBI_PANEL16) ? 16 : 32; }

// Whether the task-graph Jacobi orders each sweep's columns by norm.
int plan_sort(const lrstv_plan *pl) {
  return (pl->prm.flags & LRSTV_FLAG_JACOBI_FIXED_ORDER) ? 0 : 1;
}

GemmSel plan_gemm(const lrstv_plan *pl) {
  if (pl->prm.flags & LRSTV_FLAG_SIMT_GEMM) return kSimt;
  return GemmSel{true, pl->gemm_err, (pl->prm.flags & LRSTV_FLAG_BF16X3) ? 1 : 0,
                 (pl->prm.flags & LRSTV_FLAG_SIMT_DFT) == 0};
}

// Warm start of a plan's E-step: one Newton-Schulz step on V (the previous
// E-step's right singular vectors): C = V V^H (into Vs), D = C V (into Dscr),
// V := 1.5 V - 0.5 D; then W = A V into Wout (A, Wout, Dscr: the plan's
// specA / specB in either role; Dscr may be Wout).
// One Newton-Schulz step on every slice's V on stream st: C = V V^H (into
// Cscr), D = C V (into Dscr, slice stride dstride), V := 1.5 V - 0.5 D.
cudaError_t ns_basis(lrstv_plan *pl, float2 *Cscr, float2 *Dscr, long long dstride,
                     cudaStream_t st, int nb = 1) {
  const Dims &d = pl->d;
  const int ns = 3 * d.h * nb;
  const GemmSel gs = plan_gemm(pl);
  const long long nc2 = (long long)d.nc * d.nc;
  auto run = [&](const CGemm &g) {
    Span sp(&pl->prof, LRSTV_K_WARM_E, st);
    return gemm(g, gs, st);
  };
  cudaError_t e;
  CGemm g{};
  g.batch = ns;
  g.A = pl->V; g.sA = nc2; g.lda = d.nc;
  g.B = pl->V; g.sB = nc2; g.ldb = d.nc; g.opB = 1;
  g.C = Cscr; g.sC = nc2; g.ldc = d.nc;
  g.M = d.nc; g.N = d.nc; g.K = d.nc;
  if ((e = run(g)) != cudaSuccess) return e;
  g.A = Cscr; g.B = pl->V; g.opB = 0;
  g.C = Dscr; g.sC = dstride; g.ldc = d.nc;
  if ((e = run(g)) != cudaSuccess) return e;
  Span sp(&pl->prof, LRSTV_K_WARM_E, st);
  return launch_ns_update(d.nc, ns, (size_t)dstride, pl->V, Dscr, st);
}

// Warm start of a plan's E-step: the Newton-Schulz step on V (unless it
// already ran, ns_ready), then W = A V into Wout (A, Wout, Dscr: the plan's
// specA / specB in either role; Dscr may be Wout).  nb > 1: the first plan of
// a batch group, for all nb cubes of the group.
cudaError_t warm_basis(lrstv_plan *pl, const float2 *A, float2 *Wout, float2 *Dscr,
                       cudaStream_t st, int nb = 1) {
  const Dims &d = pl->d;
  const int ns = 3 * d.h * nb;
  const long long nc2 = (long long)d.nc * d.nc, P = (long long)d.P;
  cudaError_t e;
  if (pl->ns_ready) {
    if ((e = cudaStreamWaitEvent(st, pl->ev_ns, 0)) != cudaSuccess) return e;
  } else if ((e = ns_basis(pl, pl->Vs, Dscr, P, st, nb)) != cudaSuccess) {
    return e;
  }
  pl->ns_ready = 0;
  CGemm g{};
  g.batch = ns;
  g.A = A; g.sA = P; g.lda = d.nr;
  g.B = pl->V; g.sB = nc2; g.ldb = d.nc; g.opB = 0;
  g.C = Wout; g.sC = P; g.ldc = d.nr;
  g.M = d.nr; g.N = d.nc; g.K = d.nc;
  Span sp(&pl->prof, LRSTV_K_WARM_E, st);
  return gemm(g, plan_gemm(pl), st);
}

// The E-step with a warm-started Jacobi (LRSTV_FLAG_WARM_START).  V keeps the
// previous E-step's right singular vectors of each Fourier slice; one
// Newton-Schulz step V := V (3I - V^H V)/2 (two tensor-core GEMMs) removes the
// rounding drift of its unitarity, W = A V starts the sweeps nearly
// orthogonal, and the rotations accumulate onto V.  The Jacobi runs with a
// negative threshold (V kept unscaled) and k_sigma_scale forms V diag g for
// the reconstruction, exactly as the Jacobi epilogue would.
cudaError_t tsvt_warm(lrstv_plan *pl, float ycoef, float t, float mu, int gamma4, cudaStream_t st) {
  const Dims &d = pl->d;
  const int ns = 3 * d.h;
  const GemmSel gs = plan_gemm(pl);
  const long long nc2 = (long long)d.nc * d.nc, P = (long long)d.P;
  cudaError_t e = tsvt_pre(d, 3, pl->F, pl->G4, ycoef, pl->tb.tw3, pl->specA, st, &pl->prof, gs);
  if (e != cudaSuccess) return e;
  float2 *Wm = pl->specA, *R = pl->specB;
  if (pl->vwarm) {
    if ((e = warm_basis(pl, pl->specA, pl->specB, pl->specB, st)) != cudaSuccess) return e;
    Wm = pl->specB;
    R = pl->specA;
  }
  if ((e = launch_group_ms2(d, ns, Wm, d.h, pl->ms2, st)) != cudaSuccess) return e;
  // slices whose previous run took one sweep: the Gram check on the tensor
  // cores (into the free spectrum buffer R) shows which would rotate nothing
  const bool gram = gs.tc;
  if (gram) {
    Span sp(&pl->prof, LRSTV_K_WARM_E, st);
    if ((e = launch_gram_check(d, ns, Wm, R, pl->sweeps, pl->gcand, pl->gconv, t, pl->ms2, d.h,
                               pl->gemm_err, st)) != cudaSuccess)
      return e;
  }
  {
    JacOpt o;
    o.conv = gram ? pl->gconv : nullptr;
    o.warm = pl->vwarm;
    o.t_svt = t;
    o.ms2 = pl->ms2;
    o.group = d.h;
    o.sched = plan_sched(pl);
    o.spare_sms = kJacobiSpareSMs;
    o.pw = plan_pw(pl);
    o.order = pl->order;
    o.sort = plan_sort(pl);
    Span sp(&pl->prof, LRSTV_K_JACOBI, st);
    e = launch_jacobi(d, ns, Wm, pl->V, -1.0f, kMaxSweeps, pl->sweeps,
                      pl->prof.on ? pl->prof.d_work : nullptr, st, o);
  }
  if (e != cudaSuccess) return e;
  {
    Span sp(&pl->prof, LRSTV_K_WARM_E, st);
    if ((e = launch_sigma_scale(d, ns, Wm, pl->V, t, nullptr, pl->Vs, st)) != cudaSuccess)
      return e;
  }
  if (pl->ns_req) {
    // V is read: the next E-step's Newton-Schulz step runs on the side
    // stream, with scratch of its own, while this E-step finishes
    if ((e = cudaEventRecord(pl->ev_sig, st)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(pl->side, pl->ev_sig, 0)) != cudaSuccess) return e;
    if ((e = ns_basis(pl, pl->Vn1, pl->Vn2, nc2, pl->side)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(pl->ev_ns, pl->side)) != cudaSuccess) return e;
    pl->ns_ready = 1;
  }
  CGemm g{};
  g.A = Wm; g.sA = P; g.lda = d.nr;
  g.B = pl->Vs; g.sB = nc2; g.ldb = d.nc; g.opB = 1;
  g.C = R; g.sC = P; g.ldc = d.nr;
  g.M = d.nr; g.N = d.nc; g.K = d.nc; g.batch = ns;
  {
    Span sp(&pl->prof, LRSTV_K_CGEMM_E, st);
    if ((e = gemm(g, gs, st)) != cudaSuccess) return e;
  }
  pl->vwarm = 1;
  Span sp(&pl->prof, LRSTV_K_C2R_E, st);
  return launch_c2r3(d, 3, R, 1, pl->tb.tw3, pl->E, 1, pl->G4, pl->F, mu, gamma4, st, gs);
}

// Block `field` of m plans: one piece of m * count elements, plan i's part i.
template <class T>
void take_each(Carver &c, lrstv_plan *const *pls, int m, size_t count, T *lrstv_plan::*field) {
  T *p = c.take<T>((size_t)m * count);
  for (int i = 0; i < m; ++i) pls[i]->*field = p ? p + (size_t)i * count : nullptr;
}

// The memory of m plans of one shape (m = 1: a plan on its own) carved out of
// base (null: only the size), block by block: each block holds the m plans'
// parts back to back, so that the m cubes form a packed batch (cube i's state
// cube at i N floats, its Fourier slices at 3 i h P complex, ...) that one
// launch per kernel serves.  The DFT tables are carved once and shared.
size_t group_layout(lrstv_plan *const *pls, int m, void *base) {
  const Dims &d = pls[0]->d;
  const size_t h = (size_t)d.h, nc2 = (size_t)d.nc * d.nc;
  Carver c(base);
  take_each(c, pls, m, d.N, &lrstv_plan::Y);
  take_each(c, pls, m, d.N, &lrstv_plan::L);
  take_each(c, pls, m, d.N, &lrstv_plan::Z);
  take_each(c, pls, m, d.N, &lrstv_plan::S);
  take_each(c, pls, m, d.N, &lrstv_plan::G1);
  take_each(c, pls, m, d.N, &lrstv_plan::G2);
  take_each(c, pls, m, 3 * d.N, &lrstv_plan::F);
  take_each(c, pls, m, 3 * d.N, &lrstv_plan::E);
  take_each(c, pls, m, 3 * d.N, &lrstv_plan::G3);
  take_each(c, pls, m, 3 * d.N, &lrstv_plan::G4);
  take_each(c, pls, m, d.N, &lrstv_plan::T);
  take_each(c, pls, m, 3 * h * d.P, &lrstv_plan::specA);
  take_each(c, pls, m, 3 * h * d.P, &lrstv_plan::specB);
  take_each(c, pls, m, 3 * h * nc2, &lrstv_plan::V);
  take_each(c, pls, m, 3 * h * nc2, &lrstv_plan::Vs);
  take_each(c, pls, m, 3 * h * nc2, &lrstv_plan::Vn1);
  take_each(c, pls, m, 3 * h * nc2, &lrstv_plan::Vn2);
  take_each(c, pls, m, 3, &lrstv_plan::ms2);
  take_each(c, pls, m, h * d.P, &lrstv_plan::zA);
  take_each(c, pls, m, h * d.P, &lrstv_plan::zB);
  Tables tb;
  carve_tables(c, d, tb);
  for (int i = 0; i < m; ++i) pls[i]->tb = tb;
  take_each(c, pls, m, 2 * (size_t)kResRing, &lrstv_plan::res);
  take_each(c, pls, m, 3 * h, &lrstv_plan::sweeps);
  take_each(c, pls, m, 3 * h, &lrstv_plan::order);
  take_each(c, pls, m, 3 * h, &lrstv_plan::gcand);
  take_each(c, pls, m, 3 * h, &lrstv_plan::gconv);
  take_each(c, pls, m, (size_t)jacobi_task_ints(3 * d.h), &lrstv_plan::jsched);
  take_each(c, pls, m, 1, &lrstv_plan::gemm_err);
  unsigned long long *work = c.take<unsigned long long>(2 * (size_t)m);
  for (int i = 0; i < m; ++i) pls[i]->prof.d_work = work ? work + 2 * (size_t)i : nullptr;
  return c.off;
}

float *block_ptr(const lrstv_plan *pl, int block, size_t *count) {
  const size_t N = pl->d.N;
  *count = N;
  switch (block) {
    case LRSTV_Y: return pl->Y;
    case LRSTV_L: return pl->L;
    case LRSTV_Z: return pl->Z;
    case LRSTV_S: return pl->S;
    case LRSTV_GAMMA1: return pl->G1;
    case LRSTV_GAMMA2: return pl->G2;
    case LRSTV_TZ: return pl->T;
    case LRSTV_F: *count = 3 * N; return pl->F;
    case LRSTV_E: *count = 3 * N; return pl->E;
    case LRSTV_GAMMA3: *count = 3 * N; return pl->G3;
    case LRSTV_GAMMA4: *count = 3 * N; return pl->G4;
    default: return nullptr;
  }
}

void drop_graph(lrstv_plan *pl) {
  if (pl->gexec) cudaGraphExecDestroy(pl->gexec);
  pl->gexec = nullptr;
  pl->gY = nullptr;
  pl->gX = pl->gS = nullptr;
  pl->giters = -1;
}

int init_async(lrstv_plan *pl, const float *Y, cudaStream_t st) {
  const size_t bytes = sizeof(float) * pl->d.N;
  if (Y != pl->Y) CK(cudaMemcpyAsync(pl->Y, Y, bytes, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(pl->L, pl->Y, bytes, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(pl->Z, pl->Y, bytes, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemsetAsync(pl->S, 0, bytes, st));
  CK(cudaMemsetAsync(pl->G1, 0, bytes, st));
  CK(cudaMemsetAsync(pl->G2, 0, bytes, st));
  CK(cudaMemsetAsync(pl->F, 0, 3 * bytes, st));
  CK(cudaMemsetAsync(pl->E, 0, 3 * bytes, st));
  CK(cudaMemsetAsync(pl->G3, 0, 3 * bytes, st));
  CK(cudaMemsetAsync(pl->G4, 0, 3 * bytes, st));
  CK(cudaMemsetAsync(pl->res, 0, sizeof(unsigned) * 2 * kResRing, st));
  CK(cudaMemsetAsync(pl->sweeps, 0, sizeof(int) * 3 * pl->d.h, st));
  pl->mu = pl->prm.mu0;
  pl->iter = 0;
  pl->vwarm = 0;
  pl->ns_ready = 0;
  pl->tk.valid = 0;
  pl->tk.vvalid[0] = pl->tk.vvalid[1] = pl->tk.vvalid[2] = 0;
  if (pl->tucker) CK(cudaMemsetAsync(pl->tk.sweeps, 0, sizeof(int) * kTuckerSweepSlots, st));
  return LRSTV_OK;
}

// Steps 1 and 2 with an explicit penalty and Z-solve scratch.
int step_l_tz_mu(lrstv_plan *pl, double mu, cudaStream_t st) {
  {
    Span sp(&pl->prof, LRSTV_K_L_TZ, st);
    CK(launch_l_tz(pl->d, pl->Y, pl->S, pl->Z, pl->G1, pl->G2, pl->F, pl->G3, (float)mu, pl->prm.w,
                   pl->L, pl->T, st));
  }
  if (pl->tucker) {
    // the target just written to L is replaced by its Tucker projection, and
    // T_z is formed again from the projected L
    Span sp(&pl->prof, LRSTV_K_TUCKER, st);
    pl->tk.warm = (pl->prm.flags & LRSTV_FLAG_WARM_START) != 0;
    CK(tucker_project(pl->tk, pl->L, st));
    CK(launch_tz(pl->d, pl->L, pl->G2, pl->F, pl->G3, (float)mu, pl->prm.w, pl->T, st));
  }
  return LRSTV_OK;
}

int step_z_mu(lrstv_plan *pl, double mu, float2 *A, float2 *B, cudaStream_t st) {
  CK(zsolve_core(pl->d, 1, pl->tb, pl->T, (float)mu, pl->Z, A, B, st, &pl->prof, plan_gemm(pl)));
  return LRSTV_OK;
}

// `iters` iterations.  Iteration k+1's L/T_z and Z-solve read S, Z, Gamma1..3
// and F of iteration k (written by its fused F/S/multiplier step) but not E or
// Gamma4, so they run on the plan's low-priority side stream while iteration
// k's E-step runs on `st`; the next F/S step waits for both.  The results are
// those of the steps run one after another, bit for bit.
int iterate_async(lrstv_plan *pl, int iters, cudaStream_t st) {
  int rc;
  for (int it = 0; it < iters; ++it) {
    if (it == 0) {
      if ((rc = step_l_tz_mu(pl, pl->mu, st)) != LRSTV_OK) return rc;
      if ((rc = step_z_mu(pl, pl->mu, pl->zA, pl->zB, st)) != LRSTV_OK) return rc;
    } else {
      CK(cudaStreamWaitEvent(st, pl->ev_side, 0));
    }
    if ((rc = lrstv_step_fs_dual(pl, st)) != LRSTV_OK) return rc;
    if (it + 1 < iters) {
      const double m = (double)pl->prm.rho * pl->mu;
      const double mu_next = m < (double)pl->prm.mu_max ? m : (double)pl->prm.mu_max;
      CK(cudaEventRecord(pl->ev_fs, st));
      CK(cudaStreamWaitEvent(pl->side, pl->ev_fs, 0));
      if ((rc = step_l_tz_mu(pl, mu_next, pl->side)) != LRSTV_OK) return rc;
      if ((rc = step_z_mu(pl, mu_next, pl->zA, pl->zB, pl->side)) != LRSTV_OK) return rc;
      CK(cudaEventRecord(pl->ev_side, pl->side));
    }
    // with another iteration to follow (whose E-step joins the side stream
    // back), the next Newton-Schulz step may start early
    pl->ns_req = it + 1 < iters ? 1 : 0;
    rc = lrstv_step_e(pl, st);
    pl->ns_req = 0;
    if (rc != LRSTV_OK) return rc;
    if ((rc = lrstv_step_mu(pl)) != LRSTV_OK) return rc;
  }
  return LRSTV_OK;
}

void plan_object_free(lrstv_plan *pl);

// A plan object of one shape and parameter set with its streams and events,
// but no device memory (group_layout and arena_start give it that).
int plan_object(int n1, int n2, int n3, const lrstv_params *params, lrstv_plan **plan) {
  int rc = check_shape(n1, n2, n3);
  if (rc) return rc;
  if ((rc = check_params(params))) return rc;
  lrstv_plan *pl = new (std::nothrow) lrstv_plan();
  if (!pl) return LRSTV_ERR_ALLOC;
  pl->d = make_dims(n1, n2, n3);
  pl->prm = *params;
  pl->giters = -1;
  pl->mu = pl->prm.mu0;
  int lo_prio = 0, hi_prio = 0;
  if (cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio) != cudaSuccess ||
      cudaStreamCreateWithPriority(&pl->side, cudaStreamNonBlocking, lo_prio) != cudaSuccess ||
      cudaEventCreateWithFlags(&pl->ev_fs, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&pl->ev_side, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&pl->ev_sig, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&pl->ev_ns, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    plan_object_free(pl);
    return LRSTV_ERR_CUDA;
  }
  *plan = pl;
  return LRSTV_OK;
}

void plan_object_free(lrstv_plan *pl) {
  if (!pl) return;
  if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
  if (pl->side) cudaStreamDestroy(pl->side);
  if (pl->ev_fs) cudaEventDestroy(pl->ev_fs);
  if (pl->ev_side) cudaEventDestroy(pl->ev_side);
  if (pl->ev_sig) cudaEventDestroy(pl->ev_sig);
  if (pl->ev_ns) cudaEventDestroy(pl->ev_ns);
  delete pl;
}

// Zeroes a fresh arena of `bytes` and fills the DFT tables that pl holds
// (shared by every plan carved from the arena); returns when done.
int arena_start(lrstv_plan *pl, void *arena, size_t bytes) {
  if (cudaMemsetAsync(arena, 0, bytes, pl->cap_stream) != cudaSuccess ||
      launch_tables(pl->d, pl->prm.w, pl->tb.tw3, pl->tb.F1, pl->tb.G1, pl->tb.F2, pl->tb.G2,
                    pl->tb.lam1, pl->tb.lam2, pl->tb.lam3, pl->cap_stream) != cudaSuccess ||
      cudaStreamSynchronize(pl->cap_stream) != cudaSuccess) {
    cudaGetLastError();
    return LRSTV_ERR_CUDA;
  }
  return LRSTV_OK;
}

int copy_out(lrstv_plan *pl, float *X, float *S, cudaMemcpyKind kind, cudaStream_t st) {
  const size_t bytes = sizeof(float) * pl->d.N;
  if (X) CK(cudaMemcpyAsync(X, pl->L, bytes, kind, st));
  if (S) CK(cudaMemcpyAsync(S, pl->S, bytes, kind, st));
  return LRSTV_OK;
}

}  // namespace

extern "C" {

const char *lrstv_status_string(int s) {
  switch (s) {
    case LRSTV_OK: return "ok";
    case LRSTV_ERR_ARG: return "invalid argument";
    case LRSTV_ERR_SHAPE: return "unsupported cube shape";
    case LRSTV_ERR_CUDA: return "CUDA runtime error";
    case LRSTV_ERR_ALLOC: return "device allocation failed";
    case LRSTV_ERR_NOT_CONVERGED: return "Jacobi SVD reached its sweep cap";
    case LRSTV_ERR_NONFINITE: return "non-finite residual";
    case LRSTV_ERR_STATE: return "call out of order";
    default: return "unknown status";
  }
}

int lrstv_max_spatial(void) { return kMaxSpatial; }

int lrstv_check_bounded_wait(long long tries, int arrive, int *timed_out, int *lanes_freed) {
  if (!timed_out || !lanes_freed || tries < 1 || tries > cgemm_tc_wait_limit())
    return LRSTV_ERR_ARG;
  int *d = nullptr;
  if (cudaMalloc(&d, 2 * sizeof(int)) != cudaSuccess) return LRSTV_ERR_ALLOC;
  int h[2] = {0, 0};
  cudaError_t e = cudaMemset(d, 0, sizeof h);
  if (e == cudaSuccess) e = launch_wait_probe(tries, arrive ? 1 : 0, d, 0);
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return LRSTV_ERR_CUDA;
  *timed_out = h[0];
  *lanes_freed = h[1];
  return LRSTV_OK;
}

int lrstv_peak_probe(int unit, long long work, double *tflops, double *ms) {
  if (!tflops || !ms || unit < 0 || unit > 3 || work < 1 || work > (1ll << 40))
    return LRSTV_ERR_ARG;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) {
    cudaGetLastError();
    return LRSTV_ERR_CUDA;
  }
  void *d = nullptr;
  if (cudaMalloc(&d, 1024 * sizeof(float)) != cudaSuccess) return LRSTV_ERR_ALLOC;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double flops = 0.0;
  float t = 0.0f;
  int err = 0;
  auto launch = [&](long long w) {
    return unit < 2 ? launch_fma_peak(unit, nsm, w, (float *)d, 0, &flops)
                    : launch_mma_peak(unit - 2, nsm, w, (int *)d, 0, &flops);
  };
  cudaError_t e = cudaMemset(d, 0, 1024 * sizeof(float));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = launch(work / 16 + 1);  // untimed: loads the module, wakes the clocks
  if (e == cudaSuccess) e = cudaEventRecord(e0, 0);
  if (e == cudaSuccess) e = launch(work);
  if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e == cudaSuccess && unit >= 2) e = cudaMemcpy(&err, d, sizeof(int), cudaMemcpyDeviceToHost);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(d);
  if (e != cudaSuccess || err || !(t > 0.0f)) {
    cudaGetLastError();
    return LRSTV_ERR_CUDA;
  }
  *ms = t;
  *tflops = flops / (t * 1e-3) / 1e12;
  return LRSTV_OK;
}

const char *lrstv_kernel_name(int k) {
  static const char *names[LRSTV_NKERNEL] = {"l_tz", "r2c_z", "cgemm_z", "c2r_z", "fs_dual",
                                             "r2c_e", "jacobi", "cgemm_e", "c2r_e", "warm_e",
                                             "tucker"};
  return (k >= 0 && k < LRSTV_NKERNEL) ? names[k] : "unknown";
}

int lrstv_profile_enable(lrstv_plan *pl, int on) {
  if (!pl) return LRSTV_ERR_ARG;
  Prof &p = pl->prof;
  if (on && !p.ev) {
    p.ev = new (std::nothrow) cudaEvent_t[2 * Prof::kCap];
    if (!p.ev) return LRSTV_ERR_ALLOC;
    for (int i = 0; i < 2 * Prof::kCap; ++i) {
      if (cudaEventCreate(&p.ev[i]) != cudaSuccess) {
        for (int j = 0; j < i; ++j) cudaEventDestroy(p.ev[j]);
        delete[] p.ev;
        p.ev = nullptr;
        return LRSTV_ERR_CUDA;
      }
    }
  }
  if (on) {
    CK(cudaDeviceSynchronize());
    CK(cudaMemset(p.d_work, 0, 2 * sizeof(unsigned long long)));
    p.n = 0;
  }
  p.on = on ? 1 : 0;
  return LRSTV_OK;
}

int lrstv_profile_read(lrstv_plan *pl, lrstv_profile *out) {
  if (!pl || !out) return LRSTV_ERR_ARG;
  memset(out, 0, sizeof(*out));
  Prof &p = pl->prof;
  for (int i = 0; i < p.n; ++i) {
    CK(cudaEventSynchronize(p.ev[2 * i + 1]));
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, p.ev[2 * i], p.ev[2 * i + 1]));
    out->launches[p.cls[i]] += 1;
    out->ms[p.cls[i]] += ms;
  }
  unsigned long long w[2];
  CK(cudaMemcpy(w, p.d_work, sizeof(w), cudaMemcpyDeviceToHost));
  out->jacobi_pairs = w[0];
  out->jacobi_rotations = w[1];
  return LRSTV_OK;
}

int lrstv_plan_create(int n1, int n2, int n3, const lrstv_params *params, lrstv_plan **plan) {
  if (!plan) return LRSTV_ERR_ARG;
  *plan = nullptr;
  lrstv_plan *pl = nullptr;
  int rc = plan_object(n1, n2, n3, params, &pl);
  if (rc != LRSTV_OK) return rc;
  const size_t bytes = group_layout(&pl, 1, nullptr);
  void *arena = nullptr;
  if (cudaMalloc(&arena, bytes) != cudaSuccess) {
    cudaGetLastError();
    plan_object_free(pl);
    return LRSTV_ERR_ALLOC;
  }
  group_layout(&pl, 1, arena);
  pl->arena = arena;
  pl->arena_bytes = bytes;
  pl->own_arena = 1;
  if ((rc = arena_start(pl, arena, bytes)) != LRSTV_OK) {
    cudaFree(arena);
    plan_object_free(pl);
    return rc;
  }
  *plan = pl;
  return LRSTV_OK;
}

int lrstv_plan_destroy(lrstv_plan *pl) {
  if (!pl) return LRSTV_ERR_ARG;
  drop_graph(pl);
  int rc = LRSTV_OK;
  if (pl->prof.ev) {
    for (int i = 0; i < 2 * Prof::kCap; ++i) cudaEventDestroy(pl->prof.ev[i]);
    delete[] pl->prof.ev;
  }
  if (cudaStreamDestroy(pl->cap_stream) != cudaSuccess) rc = LRSTV_ERR_CUDA;
  if (cudaStreamDestroy(pl->side) != cudaSuccess) rc = LRSTV_ERR_CUDA;
  if (cudaEventDestroy(pl->ev_fs) != cudaSuccess) rc = LRSTV_ERR_CUDA;
  if (cudaEventDestroy(pl->ev_side) != cudaSuccess) rc = LRSTV_ERR_CUDA;
  if (cudaEventDestroy(pl->ev_sig) != cudaSuccess) rc = LRSTV_ERR_CUDA;
  if (cudaEventDestroy(pl->ev_ns) != cudaSuccess) rc = LRSTV_ERR_CUDA;
  if (pl->own_arena && cudaFree(pl->arena) != cudaSuccess) rc = LRSTV_ERR_CUDA;
  if (pl->tk_mem && cudaFree(pl->tk_mem) != cudaSuccess) rc = LRSTV_ERR_CUDA;
  delete pl;
  return rc;
}

int lrstv_plan_set_tucker(lrstv_plan *pl, const int ranks[3]) {
  if (!pl) return LRSTV_ERR_ARG;
  const bool off = !ranks || (ranks[0] == 0 && ranks[1] == 0 && ranks[2] == 0);
  const int n[3] = {pl->d.n1, pl->d.n2, pl->d.n3};
  if (!off) {
    for (int i = 0; i < 3; ++i)
      if (ranks[i] < 1 || ranks[i] > n[i]) return LRSTV_ERR_ARG;
    if (n[2] > kMaxSpatial) return LRSTV_ERR_SHAPE;  // each mode's Gram goes through the Jacobi
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return LRSTV_ERR_CUDA;
  drop_graph(pl);
  if (pl->tk_mem) cudaFree(pl->tk_mem);
  pl->tk_mem = nullptr;
  pl->tucker = 0;
  if (off) return LRSTV_OK;
  const size_t bytes = tucker_ws_bytes(n[0], n[1], n[2], ranks);
  if (cudaMalloc(&pl->tk_mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    pl->tk_mem = nullptr;
    return LRSTV_ERR_ALLOC;
  }
  tucker_carve(pl->tk, pl->tk_mem, n[0], n[1], n[2], ranks);
  if (cudaMemset(pl->tk.sweeps, 0, sizeof(int) * kTuckerSweepSlots) != cudaSuccess) return LRSTV_ERR_CUDA;
  pl->tucker = 1;
  return LRSTV_OK;
}

int lrstv_plan_tucker_factor(const lrstv_plan *pl, int mode, float *U, void *stream) {
  if (!pl || !U || mode < 0 || mode > 2) return LRSTV_ERR_ARG;
  if (!pl->tucker || !pl->tk.valid) return LRSTV_ERR_STATE;
  const size_t n = (size_t)pl->tk.n[mode] * pl->tk.r[mode];
  CK(cudaMemcpyAsync(U, pl->tk.U[mode], sizeof(float) * n, cudaMemcpyDeviceToDevice,
                     (cudaStream_t)stream));
  return LRSTV_OK;
}

int lrstv_plan_bytes(const lrstv_plan *pl, size_t *bytes) {
  if (!pl || !bytes) return LRSTV_ERR_ARG;
  *bytes = pl->arena_bytes;
  return LRSTV_OK;
}

int lrstv_plan_set_params(lrstv_plan *pl, const lrstv_params *params) {
  if (!pl) return LRSTV_ERR_ARG;
  int rc = check_params(params);
  if (rc) return rc;
  const bool wchg = memcmp(pl->prm.w, params->w, sizeof(params->w)) != 0;
  pl->prm = *params;
  drop_graph(pl);
  if (wchg) {
    const Tables &t = pl->tb;
    if (launch_tables(pl->d, pl->prm.w, t.tw3, t.F1, t.G1, t.F2, t.G2, t.lam1, t.lam2, t.lam3,
                      pl->cap_stream) != cudaSuccess ||
        cudaStreamSynchronize(pl->cap_stream) != cudaSuccess)
      return LRSTV_ERR_CUDA;
  }
  return LRSTV_OK;
}

int lrstv_init(lrstv_plan *pl, const float *Y, void *stream) {
  if (!pl || !Y) return LRSTV_ERR_ARG;
  return init_async(pl, Y, (cudaStream_t)stream);
}

int lrstv_step_l_tz(lrstv_plan *pl, void *stream) {
  if (!pl) return LRSTV_ERR_ARG;
  return step_l_tz_mu(pl, pl->mu, (cudaStream_t)stream);
}

int lrstv_step_z(lrstv_plan *pl, void *stream) {
  if (!pl) return LRSTV_ERR_ARG;
  return step_z_mu(pl, pl->mu, pl->specA, pl->specB, (cudaStream_t)stream);
}

int lrstv_step_fs_dual(lrstv_plan *pl, void *stream) {
  if (!pl) return LRSTV_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const double mu = pl->mu;
  const double thr_f = (pl->prm.flags & LRSTV_FLAG_F_THRESH_EXACT) ? pl->prm.tau / (2.0 * mu)
                                                                     : pl->prm.tau / mu;
  const double thr_s = pl->prm.lambda / mu;
  unsigned *slot = pl->res + 2 * (size_t)(pl->iter % kResRing);
  CK(cudaMemsetAsync(slot, 0, 2 * sizeof(unsigned), st));
  Span sp(&pl->prof, LRSTV_K_FS_DUAL, st);
  CK(launch_fs_dual(pl->d, pl->Y, pl->L, pl->Z, pl->S, pl->G1, pl->G2, pl->F, pl->E, pl->G3,
                    pl->G4, (float)mu, (float)thr_f, (float)thr_s, pl->prm.w, slot, st,
                    (pl->prm.flags & LRSTV_FLAG_ISO_TV) ? 1 : 0));
  return LRSTV_OK;
}

int lrstv_step_e(lrstv_plan *pl, void *stream) {
  if (!pl) return LRSTV_ERR_ARG;
  const double mu = pl->mu;
  const int gamma4 = (pl->prm.flags & LRSTV_FLAG_NO_GAMMA4) ? 0 : 1;
  if (pl->prm.flags & LRSTV_FLAG_WARM_START) {
    CK(tsvt_warm(pl, (float)(1.0 / mu), (float)(pl->prm.alpha / mu), (float)mu, gamma4,
                 (cudaStream_t)stream));
    return LRSTV_OK;
  }
  CK(tsvt_core(pl->d, 3, pl->F, pl->G4, (float)(1.0 / mu), (float)(pl->prm.alpha / mu), pl->E, 1,
               pl->G4, pl->F, (float)mu, gamma4, pl->tb.tw3, pl->specA, pl->specB, pl->V,
               pl->sweeps, (cudaStream_t)stream, &pl->prof, plan_gemm(pl), pl->ms2,
               plan_sched(pl), plan_pw(pl), pl->order, plan_sort(pl)));
  return LRSTV_OK;
}

int lrstv_step_mu(lrstv_plan *pl) {
  if (!pl) return LRSTV_ERR_ARG;
  const double m = (double)pl->prm.rho * pl->mu;
  pl->mu = m < (double)pl->prm.mu_max ? m : (double)pl->prm.mu_max;
  pl->iter += 1;
  return LRSTV_OK;
}

int lrstv_iterate(lrstv_plan *pl, int iters, void *stream) {
  if (!pl || iters < 0) return LRSTV_ERR_ARG;
  return iterate_async(pl, iters, (cudaStream_t)stream);
}

int lrstv_get_slice_sweeps(lrstv_plan *pl, int *sweeps_host, int count, void *stream) {
  if (!pl || !sweeps_host || count != 3 * pl->d.h) return LRSTV_ERR_ARG;
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  CK(cudaMemcpy(sweeps_host, pl->sweeps, sizeof(int) * count, cudaMemcpyDeviceToHost));
  return LRSTV_OK;
}

int lrstv_get_stats(lrstv_plan *pl, lrstv_stats *stats, void *stream) {
  if (!pl || !stats) return LRSTV_ERR_ARG;
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  memset(stats, 0, sizeof(*stats));
  stats->iters = pl->iter;
  stats->mu = (float)pl->mu;
  if (pl->iter > 0) {
    unsigned r[2];
    CK(cudaMemcpy(r, pl->res + 2 * (size_t)((pl->iter - 1) % kResRing), sizeof(r),
                  cudaMemcpyDeviceToHost));
    memcpy(&stats->res_inf[0], &r[0], sizeof(float));
    memcpy(&stats->res_inf[1], &r[1], sizeof(float));
  }
  const int ns = 3 * pl->d.h;
  int *sw = new (std::nothrow) int[ns];
  if (!sw) return LRSTV_ERR_ALLOC;
  if (cudaMemcpy(sw, pl->sweeps, sizeof(int) * ns, cudaMemcpyDeviceToHost) != cudaSuccess) {
    delete[] sw;
    return LRSTV_ERR_CUDA;
  }
  {
    int ge = 0;
    if (cudaMemcpy(&ge, pl->gemm_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
      delete[] sw;
      return LRSTV_ERR_CUDA;
    }
    stats->gemm_errors = ge;
  }
  for (int s = 0; s < ns; ++s) {
    if (sw[s] < 0) stats->jacobi_unconverged += 1;
    const int a = sw[s] < 0 ? -sw[s] : sw[s];
    if (a > stats->jacobi_max_sweeps) stats->jacobi_max_sweeps = a;
  }
  delete[] sw;
  if (pl->tucker) {  // the eigen-solves of the Tucker L-update count alongside
    int tsw[kTuckerSweepSlots];
    CK(cudaMemcpy(tsw, pl->tk.sweeps, sizeof(tsw), cudaMemcpyDeviceToHost));
    for (int s = 0; s < kTuckerSweepSlots; ++s) {
      if (tsw[s] < 0) stats->jacobi_unconverged += 1;
      const int a = tsw[s] < 0 ? -tsw[s] : tsw[s];
      if (a > stats->jacobi_max_sweeps) stats->jacobi_max_sweeps = a;
    }
  }
  if (stats->gemm_errors) return LRSTV_ERR_CUDA;
  if (pl->prm.flags & LRSTV_FLAG_STRICT) {
    if (!isfinite(stats->res_inf[0]) || !isfinite(stats->res_inf[1])) return LRSTV_ERR_NONFINITE;
    if (stats->jacobi_unconverged) return LRSTV_ERR_NOT_CONVERGED;
  }
  return LRSTV_OK;
}

int lrstv_state_get(const lrstv_plan *pl, int block, float *dst, void *stream) {
  if (!pl || !dst) return LRSTV_ERR_ARG;
  size_t n;
  float *src = block_ptr(pl, block, &n);
  if (!src) return LRSTV_ERR_ARG;
  CK(cudaMemcpyAsync(dst, src, sizeof(float) * n, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return LRSTV_OK;
}

int lrstv_state_set(lrstv_plan *pl, int block, const float *src, void *stream) {
  if (!pl || !src) return LRSTV_ERR_ARG;
  size_t n;
  float *dst = block_ptr(pl, block, &n);
  if (!dst) return LRSTV_ERR_ARG;
  CK(cudaMemcpyAsync(dst, src, sizeof(float) * n, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  pl->vwarm = 0;  // the imported state has no Jacobi history
  pl->ns_ready = 0;
  pl->tk.valid = 0;  // nor Tucker factors
  pl->tk.vvalid[0] = pl->tk.vvalid[1] = pl->tk.vvalid[2] = 0;
  return LRSTV_OK;
}

int lrstv_get_mu(const lrstv_plan *pl, double *mu, int *iters) {
  if (!pl) return LRSTV_ERR_ARG;
  if (mu) *mu = pl->mu;
  if (iters) *iters = pl->iter;
  return LRSTV_OK;
}

int lrstv_set_mu(lrstv_plan *pl, double mu, int iters) {
  if (!pl || !(mu > 0.0) || !isfinite(mu) || iters < 0) return LRSTV_ERR_ARG;
  pl->mu = mu;
  pl->iter = iters;
  return LRSTV_OK;
}

int lrstv_plan_run(lrstv_plan *pl, const float *Y, float *X, float *S, lrstv_stats *stats,
                   void *stream) {
  if (!pl || !Y) return LRSTV_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int iters = pl->prm.max_iter;
  int rc;
  if (pl->prm.flags & LRSTV_FLAG_GRAPH) {
    if (!pl->gexec || pl->gY != Y || pl->gX != X || pl->gS != S || pl->giters != iters) {
      drop_graph(pl);
      cudaGraph_t graph = nullptr;
      CK(cudaStreamBeginCapture(pl->cap_stream, cudaStreamCaptureModeThreadLocal));
      rc = init_async(pl, Y, pl->cap_stream);
      if (rc == LRSTV_OK) rc = iterate_async(pl, iters, pl->cap_stream);
      if (rc == LRSTV_OK) rc = copy_out(pl, X, S, cudaMemcpyDeviceToDevice, pl->cap_stream);
      cudaError_t ce = cudaStreamEndCapture(pl->cap_stream, &graph);
      if (rc != LRSTV_OK || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return rc != LRSTV_OK ? rc : LRSTV_ERR_CUDA;
      }
      ce = cudaGraphInstantiate(&pl->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (ce != cudaSuccess) {
        pl->gexec = nullptr;
        return LRSTV_ERR_CUDA;
      }
      pl->gY = Y;
      pl->gX = X;
      pl->gS = S;
      pl->giters = iters;
    }
    CK(cudaGraphLaunch(pl->gexec, st));
    // host-side scalars as after an eager run
    pl->mu = pl->prm.mu0;
    pl->iter = 0;
    for (int it = 0; it < iters; ++it) lrstv_step_mu(pl);
    pl->vwarm = (iters > 0 && (pl->prm.flags & LRSTV_FLAG_WARM_START)) ? 1 : 0;
  } else {
    if ((rc = init_async(pl, Y, st)) != LRSTV_OK) return rc;
    if ((rc = iterate_async(pl, iters, st)) != LRSTV_OK) return rc;
    if ((rc = copy_out(pl, X, S, cudaMemcpyDeviceToDevice, st)) != LRSTV_OK) return rc;
  }
  if (stats) return lrstv_get_stats(pl, stats, stream);
  return LRSTV_OK;
}

int lrstv_plan_autotune(lrstv_plan *pl, const float *Y, int iters, unsigned allowed,
                        unsigned *chosen, float *ms_out, void *stream) {
  if (!pl || !Y || iters < 0) return LRSTV_ERR_ARG;
  if (allowed & ~(unsigned)(LRSTV_FLAG_SIMT_GEMM | LRSTV_FLAG_WARM_START | LRSTV_FLAG_SIMT_DFT |
                            LRSTV_FLAG_JACOBI_PER_SLICE | LRSTV_FLAG_JACOBI_PANEL16 |
                            LRSTV_FLAG_JACOBI_FIXED_ORDER | LRSTV_FLAG_BF16X3))
    return LRSTV_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int n = iters > 0 ? iters : pl->prm.max_iter;
  const unsigned base = pl->prm.flags & ~allowed;
  // candidates: every subset of `allowed` that check_params accepts
  unsigned cands[64];
  int nc = 0;
  for (unsigned sub = 0; sub <= allowed; ++sub) {
    if ((sub & ~allowed) != 0) continue;
    // SIMT_GEMM already puts the DFTs on the SIMT kernels
    if ((sub & LRSTV_FLAG_SIMT_GEMM) && (sub & LRSTV_FLAG_SIMT_DFT)) continue;
    lrstv_params trial = pl->prm;
    trial.flags = base | sub;
    if (check_params(&trial) == LRSTV_OK && nc < 64) cands[nc++] = base | sub;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return LRSTV_ERR_CUDA;
  }
  const unsigned keep = pl->prm.flags;
  unsigned best = keep;
  float best_ms = -1.0f;
  int rc = LRSTV_OK;
  for (int c = 0; c < nc && rc == LRSTV_OK; ++c) {
    pl->prm.flags = cands[c];
    drop_graph(pl);
    // one untimed pass (first-launch costs), then the timed one
    for (int pass = 0; pass < 2 && rc == LRSTV_OK; ++pass) {
      if (pass == 1 && cudaEventRecord(e0, st) != cudaSuccess) rc = LRSTV_ERR_CUDA;
      if (rc == LRSTV_OK) rc = init_async(pl, Y, st);
      if (rc == LRSTV_OK) rc = iterate_async(pl, n, st);
      if (rc == LRSTV_OK && pass == 1 && cudaEventRecord(e1, st) != cudaSuccess) rc = LRSTV_ERR_CUDA;
    }
    float ms = 0.0f;
    if (rc == LRSTV_OK && (cudaEventSynchronize(e1) != cudaSuccess ||
                           cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      rc = LRSTV_ERR_CUDA;
    if (rc == LRSTV_OK && (best_ms < 0.0f || ms < best_ms)) {
      best_ms = ms;
      best = cands[c];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  pl->prm.flags = rc == LRSTV_OK ? best : keep;
  drop_graph(pl);
  if (rc != LRSTV_OK) return rc;
  if (chosen) *chosen = best;
  if (ms_out) *ms_out = best_ms;
  // leave the plan initialised from Y with the chosen flags
  return init_async(pl, Y, st);
}

int lrstv_plan_run_host(lrstv_plan *pl, const float *Y_host, float *X_host, float *S_host,
                        lrstv_stats *stats, void *stream) {
  if (!pl || !Y_host) return LRSTV_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(pl->Y, Y_host, sizeof(float) * pl->d.N, cudaMemcpyHostToDevice, st));
  int rc = lrstv_plan_run(pl, pl->Y, nullptr, nullptr, nullptr, stream);
  if (rc != LRSTV_OK) return rc;
  if ((rc = copy_out(pl, X_host, S_host, cudaMemcpyDeviceToHost, st)) != LRSTV_OK) return rc;
  if (stats) return lrstv_get_stats(pl, stats, stream);
  CK(cudaStreamSynchronize(st));
  return LRSTV_OK;
}

int lrstv_denoise(const float *Y, int n1, int n2, int n3, const lrstv_params *params, float *X,
                  float *S, lrstv_stats *stats, void *stream) {
  if (!Y) return LRSTV_ERR_ARG;
  lrstv_plan *pl = nullptr;
  int rc = lrstv_plan_create(n1, n2, n3, params, &pl);
  if (rc != LRSTV_OK) return rc;
  lrstv_stats local;
  rc = lrstv_plan_run(pl, Y, X, S, stats ? stats : &local, stream);
  int rc2 = lrstv_plan_destroy(pl);
  return rc != LRSTV_OK ? rc : rc2;
}

}  // extern "C"

// ------------------------------------------------------------------ batches
// A batch keeps its cubes in groups of one shape and one parameter set.  A
// group's plans are carved from one arena by group_layout, so that its cubes
// form a packed batch: each step of an iteration is one launch per kernel for
// the whole group (the stencils, the mode-3 and spatial DFTs, the GEMMs and
// the small per-slice kernels), and the Jacobi is one persistent launch over
// the slices of every group.  A batched step's launches thus grow with the
// number of distinct shapes, not with the number of cubes.  The arithmetic
// of every cube is that of a plan of its own, so the results are the same
// bit for bit.
struct BatchGroup {
  int m;              // cubes
  lrstv_plan **pls;   // their plans, in batch order; pls[0] holds the group's block bases
  void *arena;
  int big;            // slices taller than the persistent kernel takes: one launch
};

struct lrstv_batch {
  int n;
  lrstv_plan **plans;
  int ngroups;
  BatchGroup *groups;
  void *arena;           // the slice work list and its counter
  SliceTask *d_tasks;
  int ntasks;
  int *d_counter;
  int grid;
  size_t smem;
  int max_nr;  // the tallest slice in the persistent work list
  cudaStream_t cap_stream;
  cudaGraphExec_t gexec;
  const float **gY;
  float **gX, **gS;
  int giters;
};

namespace {

void batch_drop_graph(lrstv_batch *b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = nullptr;
  b->giters = -1;
}

void batch_free(lrstv_batch *b) {
  if (!b) return;
  batch_drop_graph(b);
  if (b->plans)
    for (int i = 0; i < b->n; ++i)
      if (b->plans[i]) lrstv_plan_destroy(b->plans[i]);
  if (b->groups)
    for (int k = 0; k < b->ngroups; ++k) {
      if (b->groups[k].arena) cudaFree(b->groups[k].arena);
      delete[] b->groups[k].pls;
    }
  delete[] b->groups;
  delete[] b->plans;
  delete[] b->gY;
  delete[] b->gX;
  delete[] b->gS;
  if (b->arena) cudaFree(b->arena);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  delete b;
}

int task_cmp(const void *x, const void *y) {
  const SliceTask *a = (const SliceTask *)x, *b = (const SliceTask *)y;
  const double ca = (double)a->nr * a->nc * a->nc, cb = (double)b->nr * b->nc * b->nc;
  if (ca != cb) return ca > cb ? -1 : 1;
  return a->W < b->W ? -1 : (a->W > b->W ? 1 : 0);  // a fixed order among equals
}

bool group_tucker(const BatchGroup &g) {
  for (int i = 0; i < g.m; ++i)
    if (g.pls[i]->tucker) return true;
  return false;
}

// Steps 1 and 2 (L, T_z, Z-solve) of every cube of a group.  Cubes with the
// Tucker L-update take their own launches.
int group_l_tz_z(const BatchGroup &g, cudaStream_t st) {
  int rc;
  if (group_tucker(g)) {
    for (int i = 0; i < g.m; ++i) {
      if ((rc = lrstv_step_l_tz(g.pls[i], st)) != LRSTV_OK) return rc;
      if ((rc = lrstv_step_z(g.pls[i], st)) != LRSTV_OK) return rc;
    }
    return LRSTV_OK;
  }
  lrstv_plan *p = g.pls[0];
  const float mu = (float)p->mu;
  {
    Span sp(&p->prof, LRSTV_K_L_TZ, st);
    CK(launch_l_tz(p->d, p->Y, p->S, p->Z, p->G1, p->G2, p->F, p->G3, mu, p->prm.w, p->L, p->T,
                   st, g.m));
  }
  CK(zsolve_core(p->d, g.m, p->tb, p->T, mu, p->Z, p->specA, p->specB, st, &p->prof,
                 plan_gemm(p)));
  return LRSTV_OK;
}

// Steps 3, 5, 6 (F, S, Gamma1..3) of every cube of a group; each cube's
// residual maxima go to its own ring slot.
int group_fs_dual(const BatchGroup &g, cudaStream_t st) {
  lrstv_plan *p = g.pls[0];
  const double mu = p->mu;
  const double thr_f = (p->prm.flags & LRSTV_FLAG_F_THRESH_EXACT) ? p->prm.tau / (2.0 * mu)
                                                                   : p->prm.tau / mu;
  const double thr_s = p->prm.lambda / mu;
  const size_t rs = 2 * (size_t)kResRing;  // words between consecutive cubes' rings
  unsigned *slot = p->res + 2 * (size_t)(p->iter % kResRing);
  CK(cudaMemset2DAsync(slot, rs * sizeof(unsigned), 0, 2 * sizeof(unsigned), (size_t)g.m, st));
  Span sp(&p->prof, LRSTV_K_FS_DUAL, st);
  CK(launch_fs_dual(p->d, p->Y, p->L, p->Z, p->S, p->G1, p->G2, p->F, p->E, p->G3, p->G4,
                    (float)mu, (float)thr_f, (float)thr_s, p->prm.w, slot, st,
                    (p->prm.flags & LRSTV_FLAG_ISO_TV) ? 1 : 0, g.m, rs));
  return LRSTV_OK;
}

// Step 4 (E) of every cube: per group the mode-3 DFT, the warm start's
// products and the RMS norms; one persistent Jacobi launch over the slices of
// all groups (taller slices: one launch per group); per group sigma and
// V diag g, the reconstruction and the inverse DFT with Gamma4.
int batch_e_step(lrstv_batch *b, cudaStream_t st) {
  const double mu = b->plans[0]->mu;
  const bool wflag = (b->plans[0]->prm.flags & LRSTV_FLAG_WARM_START) != 0;
  const int warm = wflag && b->plans[0]->vwarm;
  // the Jacobi always works on specA: a warm start transforms into it from specB
  for (int k = 0; k < b->ngroups; ++k) {
    const BatchGroup &g = b->groups[k];
    lrstv_plan *p = g.pls[0];
    const Dims &d = p->d;
    CK(tsvt_pre(d, 3 * g.m, p->F, p->G4, (float)(1.0 / mu), p->tb.tw3,
                warm ? p->specB : p->specA, st, &p->prof, plan_gemm(p)));
    if (warm) CK(warm_basis(p, p->specB, p->specA, p->specA, st, g.m));
    CK(launch_group_ms2(d, 3 * d.h * g.m, p->specA, d.h, p->ms2, st));
    if (wflag && plan_gemm(p).tc) {
      Span sp(&p->prof, LRSTV_K_WARM_E, st);
      CK(launch_gram_check(d, 3 * d.h * g.m, p->specA, p->specB, p->sweeps, p->gcand, p->gconv,
                           (float)(p->prm.alpha / mu), p->ms2, d.h, p->gemm_err, st));
    }
  }
  if (b->ntasks > 0) {
    CK(cudaMemsetAsync(b->d_counter, 0, sizeof(int), st));
    Prof *prof = &b->plans[0]->prof;
    Span sp(prof, LRSTV_K_JACOBI, st);
    CK(launch_jacobi_batch(b->d_tasks, b->ntasks, b->d_counter, mu, kMaxSweeps,
                           prof->on ? prof->d_work : nullptr, b->grid, b->smem, st, warm,
                           wflag ? 1 : 0, b->max_nr, plan_sort(b->plans[0])));
  }
  for (int k = 0; k < b->ngroups; ++k) {
    const BatchGroup &g = b->groups[k];
    if (!g.big) continue;
    lrstv_plan *p = g.pls[0];
    Span sp(&p->prof, LRSTV_K_JACOBI, st);
    JacOpt o;
    o.warm = warm;
    o.t_svt = (float)(p->prm.alpha / mu);
    o.ms2 = p->ms2;
    o.group = p->d.h;
    o.order = p->order;
    o.sort = plan_sort(p);
    CK(launch_jacobi(p->d, 3 * p->d.h * g.m, p->specA, p->V, wflag ? -1.0f : o.t_svt,
                     kMaxSweeps, p->sweeps, p->prof.on ? p->prof.d_work : nullptr, st, o));
  }
  for (int k = 0; k < b->ngroups; ++k) {
    const BatchGroup &g = b->groups[k];
    lrstv_plan *p = g.pls[0];
    const Dims &d = p->d;
    const int gamma4 = (p->prm.flags & LRSTV_FLAG_NO_GAMMA4) ? 0 : 1;
    if (wflag)
      CK(launch_sigma_scale(d, 3 * d.h * g.m, p->specA, p->V, (float)(p->prm.alpha / mu),
                            nullptr, p->Vs, st));
    CK(tsvt_post(d, 3 * g.m, p->E, 1, p->G4, p->F, (float)mu, gamma4, p->tb.tw3, p->specA,
                 p->specB, wflag ? p->Vs : p->V, st, &p->prof, plan_gemm(p)));
    if (wflag)
      for (int i = 0; i < g.m; ++i) g.pls[i]->vwarm = 1;
  }
  return LRSTV_OK;
}

int batch_iterate_async(lrstv_batch *b, int iters, cudaStream_t st) {
  for (int it = 0; it < iters; ++it) {
    int rc;
    for (int k = 0; k < b->ngroups; ++k)
      if ((rc = group_l_tz_z(b->groups[k], st)) != LRSTV_OK) return rc;
    for (int k = 0; k < b->ngroups; ++k)
      if ((rc = group_fs_dual(b->groups[k], st)) != LRSTV_OK) return rc;
    if ((rc = batch_e_step(b, st)) != LRSTV_OK) return rc;
    for (int i = 0; i < b->n; ++i)
      if ((rc = lrstv_step_mu(b->plans[i])) != LRSTV_OK) return rc;
  }
  return LRSTV_OK;
}

int batch_init_async(lrstv_batch *b, const float *const *Y, cudaStream_t st) {
  for (int i = 0; i < b->n; ++i) {
    if (!Y[i]) return LRSTV_ERR_ARG;
    int rc = init_async(b->plans[i], Y[i], st);
    if (rc != LRSTV_OK) return rc;
  }
  return LRSTV_OK;
}

int batch_copy_out(lrstv_batch *b, float *const *X, float *const *S, cudaStream_t st) {
  for (int i = 0; i < b->n; ++i) {
    int rc = copy_out(b->plans[i], X ? X[i] : nullptr, S ? S[i] : nullptr,
                      cudaMemcpyDeviceToDevice, st);
    if (rc != LRSTV_OK) return rc;
  }
  return LRSTV_OK;
}

bool same_group(const lrstv_plan *p, const int *dims, const lrstv_params *prm) {
  return p->d.n1 == dims[0] && p->d.n2 == dims[1] && p->d.n3 == dims[2] &&
         memcmp(&p->prm, prm, sizeof(lrstv_params)) == 0;
}

// The groups' plans and memory (see BatchGroup); b->plans[i] is cube i's plan.
int batch_groups(lrstv_batch *b, const int *dims, const lrstv_params *params) {
  int *gid = new (std::nothrow) int[b->n];
  int *cnt = new (std::nothrow) int[b->n]();
  if (!gid || !cnt) {
    delete[] gid;
    delete[] cnt;
    return LRSTV_ERR_ALLOC;
  }
  int rc = LRSTV_OK;
  // plan objects, and each cube's group (the first cube of each group leads it)
  int *lead = new (std::nothrow) int[b->n];
  if (!lead) rc = LRSTV_ERR_ALLOC;
  for (int i = 0; rc == LRSTV_OK && i < b->n; ++i) {
    rc = plan_object(dims[3 * i], dims[3 * i + 1], dims[3 * i + 2], &params[i], &b->plans[i]);
    if (rc != LRSTV_OK) break;
    gid[i] = -1;
    for (int k = 0; k < b->ngroups; ++k)
      if (same_group(b->plans[lead[k]], dims + 3 * i, &params[i])) {
        gid[i] = k;
        break;
      }
    if (gid[i] < 0) {
      gid[i] = b->ngroups;
      lead[b->ngroups++] = i;
    }
    cnt[gid[i]] += 1;
  }
  if (rc == LRSTV_OK) {
    b->groups = new (std::nothrow) BatchGroup[b->ngroups]();
    if (!b->groups) rc = LRSTV_ERR_ALLOC;
  }
  for (int k = 0; rc == LRSTV_OK && k < b->ngroups; ++k) {
    BatchGroup &g = b->groups[k];
    g.pls = new (std::nothrow) lrstv_plan *[cnt[k]];
    if (!g.pls) rc = LRSTV_ERR_ALLOC;
  }
  for (int i = 0; rc == LRSTV_OK && i < b->n; ++i) {
    BatchGroup &g = b->groups[gid[i]];
    g.pls[g.m++] = b->plans[i];
  }
  for (int k = 0; rc == LRSTV_OK && k < b->ngroups; ++k) {
    BatchGroup &g = b->groups[k];
    const size_t bytes = group_layout(g.pls, g.m, nullptr);
    if (cudaMalloc(&g.arena, bytes) != cudaSuccess) {
      cudaGetLastError();
      g.arena = nullptr;
      rc = LRSTV_ERR_ALLOC;
      break;
    }
    group_layout(g.pls, g.m, g.arena);
    for (int i = 0; i < g.m; ++i) {
      g.pls[i]->arena = g.arena;
      g.pls[i]->arena_bytes = bytes / (size_t)g.m;
      g.pls[i]->own_arena = 0;
    }
    rc = arena_start(g.pls[0], g.arena, bytes);
    g.big = g.pls[0]->d.nr > kBatchMaxNr;
  }
  delete[] gid;
  delete[] cnt;
  delete[] lead;
  return rc;
}

}  // namespace

extern "C" {

int lrstv_batch_create(int ncubes, const int *dims, const lrstv_params *params,
                       lrstv_batch **batch) {
  if (!batch || !dims || !params || ncubes < 1) return LRSTV_ERR_ARG;
  *batch = nullptr;
  for (int i = 0; i < ncubes; ++i) {
    int rc = check_shape(dims[3 * i], dims[3 * i + 1], dims[3 * i + 2]);
    if (rc) return rc;
    if ((rc = check_params(&params[i]))) return rc;
    if (params[i].mu0 != params[0].mu0 || params[i].rho != params[0].rho ||
        params[i].mu_max != params[0].mu_max || params[i].max_iter != params[0].max_iter ||
        params[i].flags != params[0].flags)
      return LRSTV_ERR_ARG;
  }
  lrstv_batch *b = new (std::nothrow) lrstv_batch();
  if (!b) return LRSTV_ERR_ALLOC;
  b->giters = -1;
  b->n = ncubes;
  b->plans = new (std::nothrow) lrstv_plan *[ncubes]();
  b->gY = new (std::nothrow) const float *[ncubes]();
  b->gX = new (std::nothrow) float *[ncubes]();
  b->gS = new (std::nothrow) float *[ncubes]();
  if (!b->plans || !b->gY || !b->gX || !b->gS) {
    batch_free(b);
    return LRSTV_ERR_ALLOC;
  }
  int rc = batch_groups(b, dims, params);
  if (rc != LRSTV_OK) {
    batch_free(b);
    return rc;
  }
  int ntasks = 0, maxnr = 1;
  for (int i = 0; i < ncubes; ++i) {
    const Dims &d = b->plans[i]->d;
    if (d.nr <= kBatchMaxNr) {
      ntasks += 3 * d.h;
      if (d.nr > maxnr) maxnr = d.nr;
    }
  }
  b->ntasks = ntasks;
  if (ntasks > 0) {
    SliceTask *h = new (std::nothrow) SliceTask[ntasks];
    if (!h) {
      batch_free(b);
      return LRSTV_ERR_ALLOC;
    }
    int k = 0;
    for (int i = 0; i < ncubes; ++i) {
      lrstv_plan *pl = b->plans[i];
      const Dims &d = pl->d;
      if (d.nr > kBatchMaxNr) continue;
      for (int s = 0; s < 3 * d.h; ++s) {
        h[k].W = pl->specA + (size_t)s * d.P;
        h[k].V = pl->V + (size_t)s * d.nc * d.nc;
        h[k].sweeps = pl->sweeps + s;
        h[k].alpha = pl->prm.alpha;
        h[k].nr = d.nr;
        h[k].nc = d.nc;
        h[k].ms2 = pl->ms2 + s / d.h;
        // the Gram check runs with the warm start on the tensor-core engine
        h[k].conv = ((pl->prm.flags & LRSTV_FLAG_WARM_START) && plan_gemm(pl).tc)
                        ? pl->gconv + s : nullptr;
        ++k;
      }
    }
    qsort(h, (size_t)ntasks, sizeof(SliceTask), task_cmp);
    const size_t tbytes = align_up(sizeof(SliceTask) * (size_t)ntasks);
    int dev = 0, sms = 1;
    if (cudaMalloc(&b->arena, tbytes + kAlign) != cudaSuccess) {
      cudaGetLastError();
      delete[] h;
      batch_free(b);
      return LRSTV_ERR_ALLOC;
    }
    b->d_tasks = (SliceTask *)b->arena;
    b->d_counter = (int *)((char *)b->arena + tbytes);
    const bool ok = cudaMemcpy(b->d_tasks, h, sizeof(SliceTask) * (size_t)ntasks,
                               cudaMemcpyHostToDevice) == cudaSuccess &&
                    cudaGetDevice(&dev) == cudaSuccess &&
                    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess;
    delete[] h;
    if (!ok) {
      cudaGetLastError();
      batch_free(b);
      return LRSTV_ERR_CUDA;
    }
    b->grid = ntasks < sms ? ntasks : sms;  // one 512-thread CTA fills an SM's registers
    b->smem = jacobi_batch_smem(maxnr);
    b->max_nr = maxnr;
  }
  if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    batch_free(b);
    return LRSTV_ERR_CUDA;
  }
  *batch = b;
  return LRSTV_OK;
}

int lrstv_batch_destroy(lrstv_batch *b) {
  if (!b) return LRSTV_ERR_ARG;
  batch_free(b);
  return LRSTV_OK;
}

int lrstv_batch_size(const lrstv_batch *b, int *ncubes) {
  if (!b || !ncubes) return LRSTV_ERR_ARG;
  *ncubes = b->n;
  return LRSTV_OK;
}

int lrstv_batch_groups(const lrstv_batch *b, int *ngroups, int *group_of) {
  if (!b || !ngroups) return LRSTV_ERR_ARG;
  *ngroups = b->ngroups;
  if (group_of)
    for (int i = 0; i < b->n; ++i)
      for (int k = 0; k < b->ngroups; ++k)
        for (int j = 0; j < b->groups[k].m; ++j)
          if (b->groups[k].pls[j] == b->plans[i]) group_of[i] = k;
  return LRSTV_OK;
}

int lrstv_batch_plan(const lrstv_batch *b, int i, lrstv_plan **plan) {
  if (!b || !plan || i < 0 || i >= b->n) return LRSTV_ERR_ARG;
  *plan = b->plans[i];
  return LRSTV_OK;
}

int lrstv_batch_init(lrstv_batch *b, const float *const *Y, void *stream) {
  if (!b || !Y) return LRSTV_ERR_ARG;
  return batch_init_async(b, Y, (cudaStream_t)stream);
}

int lrstv_batch_iterate(lrstv_batch *b, int iters, void *stream) {
  if (!b || iters < 0) return LRSTV_ERR_ARG;
  return batch_iterate_async(b, iters, (cudaStream_t)stream);
}

int lrstv_batch_run(lrstv_batch *b, const float *const *Y, float *const *X, float *const *S,
                    void *stream) {
  if (!b || !Y) return LRSTV_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int iters = b->plans[0]->prm.max_iter;
  int rc;
  if (b->plans[0]->prm.flags & LRSTV_FLAG_GRAPH) {
    bool same = b->gexec && b->giters == iters;
    for (int i = 0; same && i < b->n; ++i)
      same = b->gY[i] == Y[i] && b->gX[i] == (X ? X[i] : nullptr) &&
             b->gS[i] == (S ? S[i] : nullptr);
    if (!same) {
      batch_drop_graph(b);
      cudaGraph_t graph = nullptr;
      CK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
      rc = batch_init_async(b, Y, b->cap_stream);
      if (rc == LRSTV_OK) rc = batch_iterate_async(b, iters, b->cap_stream);
      if (rc == LRSTV_OK) rc = batch_copy_out(b, X, S, b->cap_stream);
      cudaError_t ce = cudaStreamEndCapture(b->cap_stream, &graph);
      if (rc != LRSTV_OK || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return rc != LRSTV_OK ? rc : LRSTV_ERR_CUDA;
      }
      ce = cudaGraphInstantiate(&b->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (ce != cudaSuccess) {
        b->gexec = nullptr;
        return LRSTV_ERR_CUDA;
      }
      for (int i = 0; i < b->n; ++i) {
        b->gY[i] = Y[i];
        b->gX[i] = X ? X[i] : nullptr;
        b->gS[i] = S ? S[i] : nullptr;
      }
      b->giters = iters;
    }
    CK(cudaGraphLaunch(b->gexec, st));
    for (int i = 0; i < b->n; ++i) {
      lrstv_plan *pl = b->plans[i];
      pl->mu = pl->prm.mu0;
      pl->iter = 0;
      for (int it = 0; it < iters; ++it) lrstv_step_mu(pl);
    }
    return LRSTV_OK;
  }
  if ((rc = batch_init_async(b, Y, st)) != LRSTV_OK) return rc;
  if ((rc = batch_iterate_async(b, iters, st)) != LRSTV_OK) return rc;
  return batch_copy_out(b, X, S, st);
}

int lrstv_diff(const float *x, int n1, int n2, int n3, const float w[3], float *g, void *stream) {
  if (!x || !w || !g) return LRSTV_ERR_ARG;
  int rc = check_shape(n1, n2, n3);
  if (rc) return rc;
  CK(launch_diff(make_dims(n1, n2, n3), x, w, g, (cudaStream_t)stream));
  return LRSTV_OK;
}

int lrstv_diff_adjoint(const float *g, int n1, int n2, int n3, const float w[3], float *x,
                       void *stream) {
  if (!x || !w || !g) return LRSTV_ERR_ARG;
  int rc = check_shape(n1, n2, n3);
  if (rc) return rc;
  CK(launch_diff_adjoint(make_dims(n1, n2, n3), g, w, x, (cudaStream_t)stream));
  return LRSTV_OK;
}

int lrstv_soft_threshold(const float *x, size_t n, float d, float *y, void *stream) {
  if ((!x || !y) && n) return LRSTV_ERR_ARG;
  if (!isfinite(d) || d < 0.0f) return LRSTV_ERR_ARG;
  CK(launch_soft(x, n, d, y, (cudaStream_t)stream));
  return LRSTV_OK;
}

static size_t zsolve_ws(const Dims &d, Tables *tb, float2 **A, float2 **B, void *base) {
  Carver c(base);
  *A = c.take<float2>((size_t)d.h * d.P);
  *B = c.take<float2>((size_t)d.h * d.P);
  carve_tables(c, d, *tb);
  return c.off;
}

static size_t tsvt_ws(const Dims &d, float2 **tw, float2 **A, float2 **B, float2 **V, int **sw,
                      void *base) {
  Carver c(base);
  *A = c.take<float2>((size_t)d.h * d.P);
  *B = c.take<float2>((size_t)d.h * d.P);
  *V = c.take<float2>((size_t)d.h * d.nc * d.nc);
  *tw = c.take<float2>(d.n3);
  *sw = c.take<int>(d.h);
  return c.off;
}

int lrstv_zsolve_workspace_size(int n1, int n2, int n3, size_t *bytes) {
  if (!bytes) return LRSTV_ERR_ARG;
  int rc = check_shape(n1, n2, n3);
  if (rc) return rc;
  Tables tb;
  float2 *a, *b;
  *bytes = zsolve_ws(make_dims(n1, n2, n3), &tb, &a, &b, nullptr);
  return LRSTV_OK;
}

int lrstv_tsvt_workspace_size(int n1, int n2, int n3, size_t *bytes) {
  if (!bytes) return LRSTV_ERR_ARG;
  int rc = check_shape(n1, n2, n3);
  if (rc) return rc;
  float2 *tw, *a, *b, *v;
  int *sw;
  *bytes = tsvt_ws(make_dims(n1, n2, n3), &tw, &a, &b, &v, &sw, nullptr);
  return LRSTV_OK;
}

int lrstv_zsolve(const float *T, int n1, int n2, int n3, const float w[3], float mu, float *Z,
                 void *workspace, size_t workspace_bytes, void *stream) {
  if (!T || !w || !Z || !workspace) return LRSTV_ERR_ARG;
  int rc = check_shape(n1, n2, n3);
  if (rc) return rc;
  if (!(mu > 0.0f) || !isfinite(mu) || ((size_t)workspace % kAlign)) return LRSTV_ERR_ARG;
  const Dims d = make_dims(n1, n2, n3);
  Tables tb;
  float2 *A, *B;
  if (zsolve_ws(d, &tb, &A, &B, nullptr) > workspace_bytes) return LRSTV_ERR_ARG;
  zsolve_ws(d, &tb, &A, &B, workspace);
  cudaStream_t st = (cudaStream_t)stream;
  CK(launch_tables(d, w, tb.tw3, tb.F1, tb.G1, tb.F2, tb.G2, tb.lam1, tb.lam2, tb.lam3, st));
  CK(zsolve_core(d, 1, tb, T, mu, Z, A, B, st, nullptr, kSimt));
  return LRSTV_OK;
}

int lrstv_tsvt(const float *Ain, int n1, int n2, int n3, float t, float *out, void *workspace,
               size_t workspace_bytes, int *sweeps_host, void *stream) {
  if (!Ain || !out || !workspace) return LRSTV_ERR_ARG;
  int rc = check_shape(n1, n2, n3);
  if (rc) return rc;
  if (!isfinite(t) || t < 0.0f || ((size_t)workspace % kAlign)) return LRSTV_ERR_ARG;
  const Dims d = make_dims(n1, n2, n3);
  float2 *tw, *A, *B, *V;
  int *sw;
  if (tsvt_ws(d, &tw, &A, &B, &V, &sw, nullptr) > workspace_bytes) return LRSTV_ERR_ARG;
  tsvt_ws(d, &tw, &A, &B, &V, &sw, workspace);
  cudaStream_t st = (cudaStream_t)stream;
  CK(launch_tw3(d.n3, tw, st));
  CK(tsvt_core(d, 1, Ain, nullptr, 0.0f, t, out, 0, nullptr, nullptr, 0.0f, 0, tw, A, B, V, sw,
               st));
  if (sweeps_host) {
    int *h = new (std::nothrow) int[d.h];
    if (!h) return LRSTV_ERR_ALLOC;
    if (cudaMemcpyAsync(h, sw, sizeof(int) * d.h, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      delete[] h;
      return LRSTV_ERR_CUDA;
    }
    // the largest count, or the cap (negative) if any slice hit it
    int worst = 0, capped = 0;
    for (int k = 0; k < d.h; ++k) {
      if (h[k] < 0) capped = h[k];
      else if (h[k] > worst) worst = h[k];
    }
    *sweeps_host = capped ? capped : worst;
    delete[] h;
  }
  return LRSTV_OK;
}

}  // extern "C"
