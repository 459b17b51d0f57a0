// lrstv_internal.cuh -- launchers shared between the translation units of
// liblrstv.so.  Every launcher enqueues on `st` and returns the launch's
// cudaError_t (cudaGetLastError right after the launch).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace lrstv {

struct Dims {
  int n1, n2, n3;
  size_t N;   // n1 n2 n3
  size_t P;   // n1 n2 (pixels of one frontal slice)
  int h;      // n3/2 + 1 non-redundant Fourier frontal slices
  int nr, nc; // Jacobi working matrix: nr = max(n1, n2) rows, nc = min(n1, n2) columns
  int trans;  // 1 when n1 < n2: the working matrix of a slice A is A^H
};

Dims make_dims(int n1, int n2, int n3);

// Largest n1, n2 the Jacobi kernel handles (rows of the working matrix per lane x 32).
constexpr int kMaxSpatial = 512;
// Largest n3: the mode-3 DFT kernels stage n3 twiddles in shared memory.
constexpr int kMaxBands = 4096;

// ---------------------------------------------------------------- stencil.cu
// Step 1 + T_z: L = (Y - S + Z + (G1 - G2)/mu)/2, T = mu L + G2 + D_w^*(mu F - G3).
// nb cubes packed back to back (cube b's single blocks at b N floats, its
// three-component blocks F, G3 at 3 b N), one launch.
cudaError_t launch_l_tz(const Dims &d, const float *Y, const float *S, const float *Z,
                        const float *G1, const float *G2, const float *F, const float *G3,
                        float mu, const float w[3], float *L, float *T, cudaStream_t st,
                        int nb = 1);
// Steps 3, 5, 6: F, S, Gamma1..3; res2 receives atomic maxima of |Y-L-S|, |L-Z|
// as float bits (may be null).  iso: the F threshold acts on each voxel's
// 3-vector (F_1, F_2, F_3) by its 2-norm (isotropic LRSTV, eq. CRSSTV_iso).
// nb cubes packed as for launch_l_tz; cube b's maxima at res2 + b rs.
cudaError_t launch_fs_dual(const Dims &d, const float *Y, const float *L, const float *Z,
                           float *S, float *G1, float *G2, float *F, const float *E, float *G3,
                           const float *G4, float mu, float thr_f, float thr_s, const float w[3],
                           unsigned *res2, cudaStream_t st, int iso = 0, int nb = 1,
                           size_t rs = 0);
cudaError_t launch_diff(const Dims &d, const float *x, const float w[3], float *g, cudaStream_t st);
cudaError_t launch_diff_adjoint(const Dims &d, const float *g, const float w[3], float *x,
                                cudaStream_t st);
cudaError_t launch_soft(const float *x, size_t n, float thr, float *y, cudaStream_t st);

// -------------------------------------------------------------------- dft.cu
// Tables: tw3[m] = exp(-2 pi i m / n3); Fn = exp(-2 pi i a t / n) (n x n,
// column-major), Gn its conjugate; lam_n[a] = w_n^2 4 sin^2(pi a / n).
cudaError_t launch_tables(const Dims &d, const float w[3], float2 *tw3, float2 *F1, float2 *G1,
                          float2 *F2, float2 *G2, float *lam1, float *lam2, float *lam3,
                          cudaStream_t st);
cudaError_t launch_tw3(int n3, float2 *tw3, cudaStream_t st);
// Which engine runs the GEMM-shaped work (the spatial and spectral DFTs, the
// SVT reconstruction): the tensor cores (tcgen05; err receives bounded-wait
// timeouts, prec the split: 0 = 3xTF32, 1 = 3xBF16) or the FP32 SIMT kernels.
struct GemmSel {
  bool tc;
  int *err;
  int prec;  // tensor-core split precision (launch_cgemm_tc)
  bool dft;  // with tc: the mode-3 DFTs on the tensor cores too (else the SIMT kernels)
};
// Mode-3 real-to-half-complex DFT of `nb` cubes x_b - ycoef * y_b (y may be
// null), written as slices b*h + k of `out` (P complex each), in the working
// orientation (A^H when d.trans and `work_orient`).
cudaError_t launch_r2c3(const Dims &d, int nb, const float *x, const float *y, float ycoef,
                        float2 *out, int work_orient, const float2 *tw3, cudaStream_t st,
                        GemmSel gs = {false, nullptr, 0, false});
// Inverse mode-3 DFT (half-complex to real, 1/n3 included) of `nb` spectra.
// mode 0: out_b = result.  mode 1 (E-step epilogue): E_b = result and
// G4_b += mu (E_b - F_b) when `gamma4` (F, G4 given).
cudaError_t launch_c2r3(const Dims &d, int nb, const float2 *spec, int work_orient,
                        const float2 *tw3, float *out, int mode, float *G4, const float *F,
                        float mu, int gamma4, cudaStream_t st,
                        GemmSel gs = {false, nullptr, 0, false});
// Batched complex GEMM, column-major: C_b = A_b * op(B_b), op(B) = B or B^H.
// epi 1: C(a, b) *= scale / (mu (1 + lam1[a] + lam2[b] + lam3[batch])).
// opA 1 (SIMT kernel only): op(A) = A^H, A stored K x M.  epi 2 (SIMT kernel
// only): C_b += A_b op(B_b).  lam3_period > 0: the epi-1 mode-3 eigenvalue of
// batch entry b is lam3[b % lam3_period] (several cubes' spectra in one batch).
struct CGemm {
  const float2 *A; long long sA; int lda; int opA;  // 0: N, 1: conjugate transpose
  const float2 *B; long long sB; int ldb; int opB;  // 0: N, 1: conjugate transpose
  float2 *C; long long sC; int ldc;
  int M, N, K, batch;
  int epi; const float *lam1, *lam2, *lam3; float mu, scale;
  int lam3_period;
  // tensor-core kernel only (may be null): batch entry b is computed only
  // where gate[b] != 0 (the other entries' C is left as it is)
  const int *gate;
};
cudaError_t launch_cgemm(const CGemm &g, cudaStream_t st);

// ---------------------------------------------------------------- tcgemm.cu
// The same GEMM on the tensor cores (tcgen05): prec 0 splits FP32 operands
// into two TF32 halves (3xTF32, FP32-accurate), prec 1 into two BF16 halves
// (3xBF16, about 2^-17 relative error per term, the mixed-precision mode).
// *err (may be null) is set to 1 if a CTA's wait for its MMAs runs out.
cudaError_t launch_cgemm_tc(const CGemm &g, int *err, cudaStream_t st, int prec = 0);
// The mode-3 DFTs of nb cubes on the same tensor-core pipeline (kind 1: real
// cube x - ycoef y -> half spectrum at the working orientation, as
// launch_r2c3; kind 2: half spectrum -> real cube, with the Gamma4 epilogue
// of mode 1, as launch_c2r3).
struct Dft3 {
  const float *x, *y;  // kind 1: cubes (nb N floats each), y may be null
  float ycoef;
  float2 *spec_out;    // kind 1: nb h P complex
  const float2 *spec;  // kind 2: nb h P complex
  float *out;          // kind 2: nb N floats
  float *G4;           // kind 2, mode 1: Gamma4 += mu (out - F)
  const float *F;
  float mu;
  int mode, gamma4;
  const float2 *tw3;   // exp(-2 pi i m / n3), m < n3
  int n1, n2, n3, h, trans;
  size_t P, N;
};
cudaError_t launch_dft3_tc(int kind, const Dft3 &f, int nb, int *err, cudaStream_t st,
                           int prec = 0);
size_t cgemm_tc_smem();
// the tries of the GEMM's bounded barrier wait, and a one-warp check of that
// wait and its timeout path (out: two device ints, zeroed by the caller)
long long cgemm_tc_wait_limit();
cudaError_t launch_wait_probe(long long tries, int arrive, int *out, cudaStream_t st);
// throughput probes (peaks.cu, tcgemm.cu): *flops receives the launch's
// floating-point operations; one launch covers nsm SMs
cudaError_t launch_fma_peak(int paired, int nsm, long long iters, float *sink, cudaStream_t st,
                            double *flops);
cudaError_t launch_mma_peak(int prec, int nsm, long long n_mma, int *err, cudaStream_t st,
                            double *flops);

// -------------------------------------------------------------------- svt.cu
// One-sided Jacobi on `nslices` working matrices W_s (nr x nc, column-major,
// slice stride P), accumulating V_s (nc x nc).  On exit W_s = A_s V_s and the
// columns of V_s are scaled by g_i = max(1 - t / sigma_i, 0), sigma_i = |w_i|,
// so that SVT_t(A_s) = W_s V_s^H; with t < 0 V_s is left unscaled (W_s, V_s are
// then the factors of the SVD A_s = (W_s diag(1/sigma)) diag(sigma) V_s^H).
// sweeps[s] = sweeps used, -cap if the cap hit.
// work (may be null) accumulates [pairs examined, pairs rotated].
// Options of a Jacobi launch.
//  warm: V on entry is the unitary basis W was already multiplied by (the
//    rotations accumulate onto it) instead of the identity.
//  t_svt >= 0: the SVT threshold the factors serve.  A slice with
//    ||W||_F <= t_svt (every singular value at most t_svt) runs no sweep, its
//    SVT being zero (V stays as it came); and the relative tolerance grows to
//    tol max(1, rms / t_svt), rms the columns' RMS norm.
//  ms2 (may be null): per group of `group` consecutive slices (the Fourier
//    slices of one tensor), the largest mean-square column norm, used as
//    rms^2 instead of the slice's own (launch_group_ms2).
//  negl_rel >= 0: columns whose squared norm is at or below negl_rel ||W||_F^2
//    take part in no rotation (default, when negative: (nr eps)^2, the level
//    of rounding residue).  0 rotates every nonzero column: an exactly
//    rank-deficient matrix then still has its leading right singular vectors
//    cleared of null-space components, which rotations against the skipped
//    residue columns would otherwise never remove.
struct JacOpt {
  int warm = 0;
  float t_svt = -1.0f;
  const float *ms2 = nullptr;
  int group = 1;
  float negl_rel = -1.0f;
  // scratch of jacobi_task_ints(nslices) ints: with it, slices of up to 256
  // rows run on the task-graph schedule (all SMs share every slice's panel
  // pairs); without it, one CTA per slice
  int *sched = nullptr;
  // SMs the task-graph grid leaves free for concurrent work (another stream's
  // kernels cannot share an SM with a worker CTA, which takes its shared memory)
  int spare_sms = 0;
  // panel width of the packed kernels (slices of up to 256 rows): 32 columns
  // with 16-warp CTAs, or 16 with 8-warp CTAs, two to an SM
  int pw = 32;
  // scratch of nslices ints: with it, the one-CTA-per-slice kernel starts the
  // slices in the order of their sweeps in the previous run (the sweeps array
  // as passed in), most first, so that long slices do not end a wave alone
  int *order = nullptr;
  // nslices flags of launch_gram_check (may be null): a slice whose flag is
  // set ends after one sweep without running it (that sweep would rotate
  // no pair)
  const int *conv = nullptr;
  // packed kernels (slices of up to 256 rows, either schedule): each sweep
  // pairs the slice's columns in the order of their squared norms, largest
  // first (0: in the stored order)
  int sort = 1;
};
// The Jacobi's base tolerance for slices of nr rows: a pair is rotated when
// |w_p^H w_q| > tol ||w_p|| ||w_q|| (FP32 inner products of nr terms carry
// about sqrt(nr) eps of relative rounding; the tolerance is a few times that).
float jacobi_tol0(int nr);
// Tensor-core pre-check of a warm-started Jacobi run (no counterpart in the
// paper): for every slice s whose previous run took one sweep
// (sweeps[s] == 1; those flags go to cand), G_s = W_s^H W_s on the tensor
// cores (3xTF32, into G: nslices nc x nc complex), then conv[s] = 1 when every
// column pair passes the sweep's rotation test with a margin that covers the
// rounding of G and of the sweep's own FP32 inner products, so that the
// sweep would rotate no pair; conv[s] = 0 otherwise.  t_svt, ms2 and group
// as JacOpt (the threshold-aware tolerance); gemm_err as GemmSel.
cudaError_t launch_gram_check(const Dims &d, int nslices, const float2 *W, float2 *G,
                              const int *sweeps, int *cand, int *conv, float t_svt,
                              const float *ms2, int group, int *gemm_err, cudaStream_t st);
// ints of task-graph scratch for nslices working matrices
size_t jacobi_task_ints(int nslices);
cudaError_t launch_jacobi(const Dims &d, int nslices, float2 *W, float2 *V, float t,
                          int max_sweeps, int *sweeps, unsigned long long *work,
                          cudaStream_t st, const JacOpt &opt = JacOpt());
// ms2[g] = max over slices s of group g (s / group == g) of ||W_s||_F^2 / nc.
cudaError_t launch_group_ms2(const Dims &d, int nslices, const float2 *W, int group, float *ms2,
                             cudaStream_t st);

// sigma_i = |w_i| of every working matrix (into sig, nc doubles a slice, may be
// null) and Vs = V diag(g), g = max(1 - t / sigma, 0): the Jacobi epilogue's
// arithmetic, for a Jacobi run with t < 0 (V kept unscaled).
cudaError_t launch_sigma_scale(const Dims &d, int nslices, const float2 *W, const float2 *V,
                               float t, double *sig, float2 *Vs, cudaStream_t st);
// V := 1.5 V - 0.5 D for nslices nc x nc matrices (V contiguous, D at slice
// stride dstride): with D = V V^H V, one Newton-Schulz step towards the nearest
// unitary matrix.
cudaError_t launch_ns_update(int nc, int nslices, size_t dstride, float2 *V, const float2 *D,
                             cudaStream_t st);

// One slice of a batched Jacobi launch (working matrix W, V, sweep slot, the
// cube's alpha; threshold alpha / mu formed on the device).
struct SliceTask {
  float2 *W, *V;
  int *sweeps;
  float alpha;
  int nr, nc;
  const float *ms2;  // the slice's group value of launch_group_ms2 (may be null)
  const int *conv;   // the slice's launch_gram_check flag (may be null)
};
// Largest slice height the persistent batch kernel takes.
constexpr int kBatchMaxNr = 256;  // the packed kernel's tallest slice
size_t jacobi_batch_smem(int max_nr);
// Persistent work-list Jacobi over `ntasks` slices; *counter must be 0.  warm:
// as launch_jacobi; keep: V left unscaled (threshold taken as negative).
// max_nr: the tallest slice (up to 256 rows).  sort: as JacOpt::sort.
cudaError_t launch_jacobi_batch(const SliceTask *tasks, int ntasks, int *counter, double mu,
                                int max_sweeps, unsigned long long *work, int grid, size_t smem,
                                cudaStream_t st, int warm, int keep, int max_nr, int sort);

// ------------------------------------------------------------------- api.cu
constexpr size_t kAlign = 256;
// Jacobi sweep cap per slice and E-step.  Warm-started E-steps need one or
// two sweeps late in a run and about ten early; a cold start late in a run
// (the first E-step after lrstv_state_set) needs 14-30 sweeps on most slices
// of a 200 x 200 x 80 cube at iteration 30, so the cap sits well above that.
constexpr int kMaxSweeps = 60;

inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Hands out 256-byte-aligned pieces of one allocation (or counts the bytes
// when base is null).
struct Carver {
  char *base;
  size_t off = 0;
  explicit Carver(void *b) : base((char *)b) {}
  template <class T>
  T *take(size_t count) {
    T *p = base ? (T *)(base + off) : nullptr;
    off = align_up(off + sizeof(T) * count);
    return p;
  }
};

// DFT tables of one cube shape (launch_tables fills them).
struct Tables {
  float2 *tw3, *F1, *G1, *F2, *G2;
  float *lam1, *lam2, *lam3;
};
void carve_tables(Carver &c, const Dims &d, Tables &t);
// LRSTV_OK or the status a shape outside the kernels' limits gets.
int check_shape(int n1, int n2, int n3);

struct Prof;  // per-kernel event profiler of a plan; null: not profiled

// Which GEMM implementation a call uses: the tensor cores (with an error
// slot for bounded-wait timeouts) or the FP32 SIMT kernel.
constexpr GemmSel kSimt = {false, nullptr, 0, false};
cudaError_t gemm(const CGemm &g, GemmSel gs, cudaStream_t st);

// Z-solve (eq. Z_solution) of nb cubes of shape d stored back to back:
// Z_b = (mu (I + D_w^* D_w))^{-1} T_b through the 3-D DFT.  specA, specB:
// nb h P complex scratch each.
cudaError_t zsolve_core(const Dims &d, int nb, const Tables &tb, const float *T, float mu,
                        float *Z, float2 *specA, float2 *specB, cudaStream_t st, Prof *prof,
                        GemmSel gs);

// --------------------------------------------------------------- tucker.cu
// Workspace and state of the Tucker (HOOI) L-update of one cube: factors U_n
// (n_n x r_n, column-major), two scratch cubes, the Gram matrix and the
// Jacobi buffers of its eigen-solve.  valid = 0: the next projection starts
// from the truncated HOSVD.
struct TuckerWs {
  int n[3], r[3];
  float *U[3];
  float *s0, *s1, *G;
  float2 *W, *D;       // the Jacobi's W, a GEMM scratch
  float *Vr, *Wr;      // real parts of a warm start's basis and of G times it
  float2 *Vm[3];       // per mode: eigenvectors of the last solve (warm start)
  int *sweeps;          // Jacobi sweeps (-cap if capped): modes' HOOI solves, then HOSVD's
  int valid;           // U holds factors (else the next projection starts from the HOSVD)
  int vvalid[3];       // Vm[n] holds eigenvectors
  int warm;            // eigen-solves start from Vm[n] when it holds eigenvectors
};
constexpr int kTuckerSweepSlots = 6;
size_t tucker_ws_bytes(int n1, int n2, int n3, const int r[3]);
void tucker_carve(TuckerWs &t, void *ws, int n1, int n2, int n3, const int r[3]);
// X (in place) := X x1 U1 U1^T x2 U2 U2^T x3 U3 U3^T after one HOOI sweep.
cudaError_t tucker_project(TuckerWs &t, float *X, cudaStream_t st);
// T = mu L + Gamma2 + D_w^*(mu F - Gamma3) for a given L.
cudaError_t launch_tz(const Dims &d, const float *L, const float *G2, const float *F,
                      const float *G3, float mu, const float w[3], float *T, cudaStream_t st);

// t-SVT of one cube with threshold t on caller-provided scratch: tw3 (n3),
// specA and specB (h P each), V (h nc^2), sweeps (h); every piece is written
// before it is read.
cudaError_t tsvt_plain(const Dims &d, const float *A, float t, float *out, float2 *tw3,
                       float2 *specA, float2 *specB, float2 *V, int *sweeps, cudaStream_t st);

}  // namespace lrstv
