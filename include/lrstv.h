/*
 * lrstv.h -- C ABI of the GB300 (sm_103a) plain-LRSTV hyperspectral denoiser.
 *
 * Method: arXiv 2204.12879, "Low-rank Meets Sparseness: An Integrated
 * Spatial-Spectral Total Variation Approach to Hyperspectral Denoising".
 * The library runs the ADMM iteration of Section III-C (Algorithm 1) for the
 * model min ||L||_LRSTV + lambda ||S||_1 s.t. Y = L + S (eq. TDLRSTV without
 * the Tucker constraint, i.e. full Tucker ranks, so the HOOI step of the
 * L-update is the identity).
 *
 * Conventions (every entry point):
 *  - Cubes are FP32, n1 x n2 x n3, element (i, j, k) at i + n1*(j + n2*k)
 *    (mode 1 fastest, frontal slices contiguous).  N = n1*n2*n3.
 *  - Unless a name ends in _host, array arguments are DEVICE pointers owned
 *    by the caller; the library never frees them.  Gradient-shaped arrays
 *    (g, F, E, Gamma3, Gamma4) hold the three modes back to back: 3N floats.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is stream-ordered and asynchronous unless stated.
 *  - Every call returns an lrstv_status.  No call aborts, traps or prints.
 *  - A plan owns all of its device memory (one allocation made by
 *    lrstv_plan_create); no other call of a plan allocates.
 */
#ifndef LRSTV_H
#define LRSTV_H
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lrstv_status {
  LRSTV_OK = 0,
  LRSTV_ERR_ARG = 1,            /* null pointer, bad flag, bad scalar          */
  LRSTV_ERR_SHAPE = 2,          /* size outside what the kernels support       */
  LRSTV_ERR_CUDA = 3,           /* a CUDA runtime call or launch failed        */
  LRSTV_ERR_ALLOC = 4,          /* device memory could not be allocated        */
  LRSTV_ERR_NOT_CONVERGED = 5,  /* a Jacobi SVD hit its sweep cap              */
  LRSTV_ERR_NONFINITE = 6,      /* a residual is NaN or Inf                    */
  LRSTV_ERR_STATE = 7           /* call out of order (a backward pass with no
                                   forward pass before it)                     */
} lrstv_status;

/* Flags (lrstv_params.flags). */
#define LRSTV_FLAG_F_THRESH_EXACT 1u /* F threshold tau/(2 mu), the exact minimiser of the
                                        F-subproblem, instead of the printed tau/mu (eq. F_solution) */
#define LRSTV_FLAG_NO_GAMMA4 2u      /* keep Gamma4 = 0 (the paper lists only Gamma1..3 updates) */
#define LRSTV_FLAG_GRAPH 4u          /* lrstv_plan_run replays its iterations as one CUDA graph */
#define LRSTV_FLAG_STRICT 8u         /* stats report NOT_CONVERGED / NONFINITE as the return status */
#define LRSTV_FLAG_SIMT_GEMM 16u     /* spatial DFT and SVT-reconstruction GEMMs on the FP32 SIMT
                                        path instead of the tensor cores (tcgen05, 3xTF32) */
#define LRSTV_FLAG_WARM_START 32u    /* each E-step's Jacobi SVDs start from the previous E-step's
                                        right singular vectors (made unitary again by one
                                        Newton-Schulz step) instead of the identity: the same
                                        t-SVT to rounding, in fewer sweeps.  The first E-step after
                                        lrstv_init or lrstv_state_set starts cold. */
#define LRSTV_FLAG_ISO_TV 64u        /* isotropic LRSTV (eq. CRSSTV_iso, read with the per-pixel
                                        2-norm of the isotropic TV of Section II-B and
                                        tau_n = (tau w_n)^2): the F-update thresholds each voxel's
                                        3-vector (F_1, F_2, F_3) by its 2-norm,
                                        F_v = x_v max(1 - thr / |x_v|_2, 0), thr as for the
                                        anisotropic threshold (tau/mu, or tau/(2 mu) with
                                        LRSTV_FLAG_F_THRESH_EXACT).  Plans and batches only. */
#define LRSTV_FLAG_BF16X3 128u       /* mixed precision: the tensor-core GEMMs (spatial DFTs of
                                        the Z-solve, SVT reconstruction, warm-start products)
                                        split each FP32 operand into two BF16 halves and form
                                        hi*hi + hi*lo + lo*hi with FP32 accumulation (about
                                        2^-17 relative error per term instead of 3xTF32's
                                        2^-21); storage, the Jacobi and the thresholds stay
                                        FP32, the sigma-vs-threshold decisions FP64.  Not with
                                        LRSTV_FLAG_SIMT_GEMM (ERR_ARG). */
#define LRSTV_FLAG_JACOBI_PER_SLICE 512u /* run each Fourier slice's Jacobi sweeps in one CTA
                                        (its column panels in sequence) instead of the
                                        task-graph schedule, in which every SM takes panel-pair
                                        tasks of any slice (slices up to 256 rows; the same
                                        t-SVT to rounding, the pairs visited in another
                                        order).  Batches always run their slices this way, so
                                        a batch's cube equals a plan made with this flag. */
#define LRSTV_FLAG_SIMT_DFT 256u     /* the mode-3 (spectral) DFTs on the FP32 SIMT kernels (direct
                                        sums with twiddle tables) instead of the tensor-core
                                        pipeline (3xTF32, or 3xBF16 with LRSTV_FLAG_BF16X3);
                                        LRSTV_FLAG_SIMT_GEMM puts them there too */
#define LRSTV_FLAG_JACOBI_PANEL16 1024u /* the Jacobi's column panels 16 wide, each CTA 8 warps
                                        and two CTAs to an SM, instead of 32 wide with 16-warp
                                        CTAs (slices up to 256 rows; the same t-SVT to
                                        rounding, the pairs visited in another order).
                                        Batches run 32-column panels whatever the flag. */
#define LRSTV_FLAG_JACOBI_FIXED_ORDER 4096u /* the Jacobi pairs a slice's columns in their
                                        stored order in every sweep, instead of ordering them
                                        by squared norm, largest first, at the start of each
                                        sweep (de Rijk's ordering: fewer sweeps; the same t-SVT
                                        to rounding).  Slices of up to 256 rows, either
                                        schedule; a batch follows its first cube's flag. */
#define LRSTV_FLAG_UNROLL_RECOMPUTE 2048u /* unrolled iteration only: the forward pass keeps one
                                        slot of SVD factors instead of one per iteration, and
                                        the backward pass recomputes iteration k's factors
                                        from its checkpointed states (the same kernels on the
                                        same inputs: bit-identical gradients) before its t-SVT
                                        adjoint; a warm start still keeps every iteration's V,
                                        the next iteration's starting point */

/* Scalars of Algorithm 1 (Section III-C; parameter roles in Section IV-D).
 *  tau     weight of ||D_w L||_1 (gradient sparsity)
 *  alpha   weight of the tensor nuclear norm of the gradient maps
 *  lambda  weight of ||S||_1 (the paper suggests C / sqrt(n1 n2))
 *  w[3]    weights of D_w = [w1 D1; w2 D2; w3 D3]
 *  mu0, rho, mu_max   penalty schedule mu := min(rho mu, mu_max) (step 7)
 *  eps     stopping tolerance of the convergence check (reported only; the
 *          iteration count is max_iter)
 *  max_iter iterations run by lrstv_plan_run / lrstv_denoise (>= 0) */
typedef struct lrstv_params {
  float tau, alpha, lambda;
  float w[3];
  float mu0, rho, mu_max, eps;
  int max_iter;
  unsigned flags;
} lrstv_params;

/* Filled after a synchronising call (lrstv_get_stats, lrstv_plan_run*). */
typedef struct lrstv_stats {
  int iters;                 /* iterations run since lrstv_init                  */
  float res_inf[2];          /* ||Y-L-S||_inf and ||L-Z||_inf after the last one */
  float mu;                  /* penalty for the next iteration                   */
  int jacobi_unconverged;    /* Fourier slices whose SVD hit the sweep cap (last E-step) */
  int jacobi_max_sweeps;     /* largest sweep count of the last E-step           */
  int gemm_errors;           /* tensor-core GEMM tiles whose bounded wait ran out (0) */
} lrstv_stats;

/* State blocks for lrstv_state_get / lrstv_state_set.  Blocks of 3N floats
 * are marked [3]. */
typedef enum lrstv_block {
  LRSTV_Y = 0, LRSTV_L = 1, LRSTV_Z = 2, LRSTV_S = 3, LRSTV_GAMMA1 = 4, LRSTV_GAMMA2 = 5,
  LRSTV_F = 6 /*[3]*/, LRSTV_E = 7 /*[3]*/, LRSTV_GAMMA3 = 8 /*[3]*/, LRSTV_GAMMA4 = 9 /*[3]*/,
  LRSTV_TZ = 10 /* right-hand side T_z of the last Z-step */
} lrstv_block;

typedef struct lrstv_plan lrstv_plan;

/* ---------------------------------------------------------------- status */
const char *lrstv_status_string(int status);
/* Largest n1, n2 supported by the SVT kernels (min(n1, n2) and max(n1, n2)
 * bound the Jacobi working matrix). */
int lrstv_max_spatial(void);
/* Checks the bounded wait that the tensor-core GEMM puts on its MMA
 * barriers, and its timeout path, without a fault: one warp allocates tensor
 * memory as the GEMM does and waits on an mbarrier with the wait cut to
 * `tries` tries (1 .. the GEMM's own limit, 250000 tries, about a second:
 * one try that finds the phase incomplete suspends for a few microseconds).
 * With arrive != 0 the
 * barrier's phase is completed first and the wait ends; with arrive == 0
 * nothing arrives and the wait runs out.  *timed_out = 1 when it ran out,
 * else 0; *lanes_freed = the lanes that freed the tensor memory and
 * returned (32).  Synchronous on the legacy default stream; makes and frees
 * one 8-byte device allocation.  ERR_ARG (null output, tries out of range),
 * ERR_ALLOC, ERR_CUDA. */
int lrstv_check_bounded_wait(long long tries, int arrive, int *timed_out, int *lanes_freed);

/* Throughput probe (no counterpart in the paper; it gives the benchmark
 * measured peaks for its roofline fractions): runs one kernel of this library
 * over every SM of the current device and reports its rate.
 *  unit 0: FP32 FMA, scalar fmaf (8 independent chains a thread, 32 warps per SM);
 *  unit 1: FP32 FMA, the paired instruction __ffma2_rn (16 chains);
 *  unit 2: tensor pipe, tcgen05.mma kind::tf32, M = 128, N = 256, K = 8 per
 *          instruction, operands in shared memory, one CTA and one issuing
 *          thread per SM, two alternating TMEM accumulators;
 *  unit 3: the same with kind::f16 on BF16 operands (K = 16 per instruction).
 * work: loop trips per thread (units 0, 1) or MMAs per SM (units 2, 3), in
 * 1 .. 2^40; about 2e7 FMA trips or 4e6 MMAs take a few hundred ms.  One
 * untimed launch of work/16 + 1 comes first.  *tflops = floating-point
 * operations (2 per FMA, 2 M N K per MMA) / the timed launch's CUDA-event
 * time, *ms that time.  Synchronous on the legacy default stream; makes and
 * frees one 4 KB device allocation.  ERR_ARG, ERR_ALLOC, ERR_CUDA (also when
 * an MMA probe's bounded wait ran out). */
int lrstv_peak_probe(int unit, long long work, double *tflops, double *ms);

/* ------------------------------------------------- full TDLRSTV (Tucker) */
/* Turns the L-update of a plan into the Tucker projection of the full TDLRSTV
 * model (eq. TDLRSTV, Section III-C step 1, eq. X_solution with the Tucker-3
 * model of eq. LRTAmodel): L = X x1 U1 U1^T x2 U2 U2^T x3 U3 U3^T with X =
 * 1/2 (Y - S + Z + (Gamma1 - Gamma2)/mu) and multilinear ranks
 * ranks = {r1, r2, r3} (1 <= r_n <= n_n; the paper sets r1 = 0.8 n1,
 * r2 = 0.8 n2 and tunes r3).  The factors come from one HOOI sweep per ADMM
 * iteration (U1, U2, U3 in turn), started from the previous iteration's
 * factors, or from the truncated HOSVD of X in the first iteration after
 * lrstv_init or lrstv_state_set; with LRSTV_FLAG_WARM_START each mode's
 * eigen-solve also starts from that mode's previous eigenvectors.  The six
 * eigen-solves' sweep counts join lrstv_stats (a capped one counts as
 * unconverged).  ranks NULL or {0, 0, 0}: back to the plain
 * L-update.  Makes a second device allocation owned by the plan (freed by
 * lrstv_plan_destroy or by turning the mode off); synchronises the device.
 * ERR_ARG for ranks out of range, ERR_SHAPE for n3 > lrstv_max_spatial() (each
 * mode's Gram matrix is diagonalised by the Jacobi kernel), ERR_ALLOC if the
 * allocation fails. */
int lrstv_plan_set_tucker(lrstv_plan *plan, const int ranks[3]);

/* The Tucker factor U_n of the last L-update (mode = n - 1 in 0..2): the
 * n_n x r_n matrix (column-major FP32) whose orthonormal columns are the r_n
 * leading eigenvectors of the mode-n Gram matrix of that iteration's HOOI
 * sweep (eq. LRTAmodel's factor matrices), copied to caller device memory U
 * (n_n r_n floats), stream-ordered.  ERR_ARG (null, mode out of range),
 * ERR_STATE (the Tucker L-update is off, or no L-update has run since
 * lrstv_init, lrstv_state_set or lrstv_plan_set_tucker). */
int lrstv_plan_tucker_factor(const lrstv_plan *plan, int mode, float *U, void *stream);

/* ------------------------------------------------------------- profiling */
/* Kernels a plan launches (lrstv_profile indices). */
typedef enum lrstv_kernel {
  LRSTV_K_L_TZ = 0,     /* step 1 + T_z                                   */
  LRSTV_K_R2C_Z = 1,    /* mode-3 DFT of T_z                              */
  LRSTV_K_CGEMM_Z = 2,  /* spatial DFTs + spectral division (4 per Z-step) */
  LRSTV_K_C2R_Z = 3,    /* inverse mode-3 DFT -> Z                        */
  LRSTV_K_FS_DUAL = 4,  /* steps 3, 5, 6                                  */
  LRSTV_K_R2C_E = 5,    /* mode-3 DFT of F - Gamma4/mu                    */
  LRSTV_K_JACOBI = 6,   /* one-sided Jacobi + singular-value threshold    */
  LRSTV_K_CGEMM_E = 7,  /* SVT reconstruction W (V diag g)^H              */
  LRSTV_K_C2R_E = 8,    /* inverse mode-3 DFT -> E, Gamma4 update         */
  LRSTV_K_WARM_E = 9,   /* warm start: Newton-Schulz step on V, W = A V,
                           sigma and V diag g (LRSTV_FLAG_WARM_START)     */
  LRSTV_K_TUCKER = 10,  /* Tucker (HOOI) L-update and T_z from the projected L,
                           one entry per L-update (lrstv_plan_set_tucker) */
  LRSTV_NKERNEL = 11
} lrstv_kernel;

typedef struct lrstv_profile {
  int launches[16];                     /* per lrstv_kernel                        */
  double ms[16];                        /* summed device time (CUDA events)       */
  unsigned long long jacobi_pairs;      /* column pairs examined by Jacobi sweeps  */
  unsigned long long jacobi_rotations;  /* pairs that were rotated                 */
} lrstv_profile;

/* Short name of a lrstv_kernel index ("l_tz", "jacobi", ...; the keys of the
 * benchmark's per-kernel table); "unknown" out of range.  Static storage. */
const char *lrstv_kernel_name(int kernel);
/* on != 0: clears the counters and brackets every later kernel launch of the
 * plan with CUDA events (none while a stream is being captured; at most 4096
 * launches are recorded).  on == 0: stops recording. */
int lrstv_profile_enable(lrstv_plan *plan, int on);
/* Synchronises the recorded launches and sums their times and the Jacobi
 * work counters since the last enable. */
int lrstv_profile_read(lrstv_plan *plan, lrstv_profile *out);

/* ------------------------------------------------------------------ plan */
/* Allocates and initialises every device buffer for an n1 x n2 x n3 cube:
 * the 18 state cubes of Algorithm 1, the half spectrum (n3/2 + 1 complex
 * frontal slices) for the Z-solve and the t-SVT, the per-slice Jacobi
 * matrices, and DFT tables.  Errors: ERR_ARG (null, n < 1), ERR_SHAPE (n1 or
 * n2 above lrstv_max_spatial(), n3 above 4096, or 3 n1 n2 n3 above 2e9),
 * ERR_ALLOC, ERR_CUDA.  Uses the current
 * device; the plan must be used with that device current. */
int lrstv_plan_create(int n1, int n2, int n3, const lrstv_params *params, lrstv_plan **plan);
int lrstv_plan_destroy(lrstv_plan *plan);
/* Bytes of device memory the plan holds. */
int lrstv_plan_bytes(const lrstv_plan *plan, size_t *bytes);
/* Replaces the scalars (tau, alpha, lambda, w, mu0, rho, mu_max, eps,
 * max_iter, flags); takes effect at the next step. */
int lrstv_plan_set_params(lrstv_plan *plan, const lrstv_params *params);

/* Initialisation of Algorithm 1 (left empty by the paper; this library's
 * reading): L = Z = Y, S = F = E = 0, all multipliers 0, mu = mu0, iteration
 * counter 0.  Y: device, N floats. */
int lrstv_init(lrstv_plan *plan, const float *Y, void *stream);

/* ------------------------------------------------------- per-step calls */
/* Step 1 (eq. X_solution, full ranks): L = (Y - S + Z + (Gamma1 - Gamma2)/mu)/2,
 * fused with the right-hand side of the Z-system (eq. Z_solution):
 * T_z = mu L + Gamma2 + D_w^*(mu F - Gamma3). */
int lrstv_step_l_tz(lrstv_plan *plan, void *stream);
/* Step 2 (eq. Z_solution): Z = ifftn(fftn(T_z) / (mu (1 + P_z))). */
int lrstv_step_z(lrstv_plan *plan, void *stream);
/* Steps 3, 5 and 6 fused (eq. F_solution, S_solution, Multipliers):
 * F_n = R_{tau/mu}((w_n D_n Z + Gamma3_n/mu + E_n + Gamma4_n/mu)/2),
 * S = R_{lambda/mu}(Y - L + Gamma1/mu), Gamma1 += mu (Y - L - S),
 * Gamma2 += mu (L - Z), Gamma3_n += mu (w_n D_n Z - F_n).  F reads the E of
 * the previous iteration (Algorithm 1's order); S and Gamma1..3 do not read E,
 * so fusing them before step 4 keeps the order's results. */
int lrstv_step_fs_dual(lrstv_plan *plan, void *stream);
/* Step 4 (eq. E_solution): E_n = t-SVT(F_n - Gamma4_n/mu, alpha/mu) for the
 * three gradient tensors, then Gamma4_n += mu (E_n - F_n) (unless
 * LRSTV_FLAG_NO_GAMMA4). */
int lrstv_step_e(lrstv_plan *plan, void *stream);
/* Step 7: mu := min(rho mu, mu_max), and the iteration counter advances. */
int lrstv_step_mu(lrstv_plan *plan);
/* `iters` full iterations (steps 1-7), stream-ordered, no host sync. */
int lrstv_iterate(lrstv_plan *plan, int iters, void *stream);

/* Synchronises `stream` and reports residuals, mu and Jacobi status. */
int lrstv_get_stats(lrstv_plan *plan, lrstv_stats *stats, void *stream);
/* Per-slice Jacobi sweep counts of the last E-step (synchronises `stream`):
 * count must be 3 (n3/2 + 1); entry n (n3/2 + 1) + k is Fourier slice k of
 * gradient tensor n, negative if it hit the sweep cap, 0 if it needed none. */
int lrstv_get_slice_sweeps(lrstv_plan *plan, int *sweeps_host, int count, void *stream);
/* Copies a state block to / from caller device memory (N or 3N floats,
 * device-to-device, stream-ordered).  With lrstv_get_mu / lrstv_set_mu this
 * checkpoints and resumes an ADMM run (mu is kept in double precision, so a
 * resumed run repeats the uninterrupted one bit for bit). */
int lrstv_state_get(const lrstv_plan *plan, int block, float *dst, void *stream);
int lrstv_state_set(lrstv_plan *plan, int block, const float *src, void *stream);
int lrstv_get_mu(const lrstv_plan *plan, double *mu, int *iters);
int lrstv_set_mu(lrstv_plan *plan, double mu, int iters);

/* ----------------------------------------------------------- whole runs */
/* The problem statement Y -> (X = L, S) of eq. TDLRSTV (plain form):
 * lrstv_init, params.max_iter iterations, X := L and S copied out.  Device
 * buffers of N floats.  Returns after enqueueing, except that stats (if not
 * NULL) forces a synchronisation. */
int lrstv_plan_run(lrstv_plan *plan, const float *Y, float *X, float *S, lrstv_stats *stats,
                   void *stream);
/* Same with HOST buffers: copies Y in, runs, copies X and S out, and
 * synchronises `stream` before returning.  Pinned host memory gives
 * asynchronous copies; pageable memory works too. */
int lrstv_plan_run_host(lrstv_plan *plan, const float *Y_host, float *X_host, float *S_host,
                        lrstv_stats *stats, void *stream);
/* Autotuner (no counterpart in the paper): times `iters` iterations
 * (params.max_iter when 0) of the plan from the device cube Y for every
 * combination of the flags in `allowed` (a subset of LRSTV_FLAG_SIMT_GEMM |
 * LRSTV_FLAG_SIMT_DFT | LRSTV_FLAG_JACOBI_PER_SLICE | LRSTV_FLAG_JACOBI_PANEL16 |
 * LRSTV_FLAG_JACOBI_FIXED_ORDER | LRSTV_FLAG_WARM_START | LRSTV_FLAG_BF16X3; combinations params rejects, and
 * SIMT_DFT together with SIMT_GEMM, are skipped), each after
 * one untimed pass, with CUDA events on `stream`, and keeps the fastest in
 * the plan's params.flags.  These choices change the work (GEMM and DFT
 * engines, the Jacobi's schedule, panel width and starting basis), not the
 * result beyond
 * the FP32 bound; allowing LRSTV_FLAG_BF16X3 lets the tuner trade that bound
 * for the 3xBF16 one (see the flag).  *chosen and
 * *ms_out (may be NULL) receive the flags kept and their time in ms.  Leaves
 * the plan initialised from Y (lrstv_init) and synchronises `stream`.
 * ERR_ARG for a NULL plan or Y, iters < 0 or other bits in `allowed`; on any
 * CUDA error the plan's flags are restored. */
int lrstv_plan_autotune(lrstv_plan *plan, const float *Y, int iters, unsigned allowed,
                        unsigned *chosen, float *ms_out, void *stream);
/* One-shot form: creates a plan, runs it, destroys it (synchronises). */
int lrstv_denoise(const float *Y, int n1, int n2, int n3, const lrstv_params *params, float *X,
                  float *S, lrstv_stats *stats, void *stream);

/* ------------------------------------------------------------ batches */
/* A batch of independent cubes of possibly different shapes, run in
 * lockstep.  The cubes are kept in groups of one shape and one parameter set,
 * whose state the batch lays out as packed batches (block by block, the
 * group's cubes back to back).  Each ADMM step launches every kernel but the
 * Jacobi once per group, for all of its cubes, and ONE persistent Jacobi
 * launch that works through the Fourier slices of all cubes (largest first)
 * from a shared work list, so an uneven batch keeps every SM busy and a
 * step's launches grow with the number of groups, not of cubes.  Each cube
 * follows Algorithm 1 exactly as a single plan does (bit-identical results);
 * the paper treats one cube at a time, and batching is this library's
 * serving form.
 *  dims    3*ncubes ints: n1, n2, n3 of each cube.
 *  params  ncubes structs; mu0, rho, mu_max, max_iter and flags must agree
 *          (the cubes share one penalty schedule), tau, alpha, lambda and w
 *          may differ.  Parameters are fixed when the batch is created.
 * The batch owns one plan per cube (lrstv_batch_plan lends it for stats and
 * state export; do not destroy it or change its parameters), one allocation
 * per group and one small allocation for the work list.  Slices taller than
 * 256 rows (max(n1, n2)) take a separate Jacobi launch per group.  The
 * persistent launch is recorded in cube 0's profile (lrstv_profile_*), a
 * group's other launches in the profile of its first cube.  A cube whose plan
 * has the Tucker L-update (lrstv_plan_set_tucker) takes its own launches for
 * steps 1 and 2. */
typedef struct lrstv_batch lrstv_batch;
int lrstv_batch_create(int ncubes, const int *dims, const lrstv_params *params,
                       lrstv_batch **batch);
int lrstv_batch_destroy(lrstv_batch *batch);
int lrstv_batch_size(const lrstv_batch *batch, int *ncubes);
/* Number of groups (distinct shape and parameter sets) and, in group_of
 * (ncubes ints, may be NULL), each cube's group, numbered in order of first
 * appearance.  ERR_ARG for a NULL batch or ngroups. */
int lrstv_batch_groups(const lrstv_batch *batch, int *ngroups, int *group_of);
int lrstv_batch_plan(const lrstv_batch *batch, int i, lrstv_plan **plan);
/* Y: host array of ncubes device pointers (N_i floats each). */
int lrstv_batch_init(lrstv_batch *batch, const float *const *Y, void *stream);
int lrstv_batch_iterate(lrstv_batch *batch, int iters, void *stream);
/* lrstv_batch_init, max_iter iterations, X_i := L_i and S_i copied out (host
 * arrays of device pointers; X or S may be NULL).  With LRSTV_FLAG_GRAPH the
 * whole run is captured into one CUDA graph on first use and replayed while
 * the pointers and max_iter stay the same. */
int lrstv_batch_run(lrstv_batch *batch, const float *const *Y, float *const *X, float *const *S,
                    void *stream);

/* ---------------------------------------------------- standalone operators */
/* g_n = w_n D_n x, circular forward differences D_n x(v) = x(v + e_n) - x(v)
 * along mode n (Section III-A).  x: N floats, g: 3N floats. */
int lrstv_diff(const float *x, int n1, int n2, int n3, const float w[3], float *g, void *stream);
/* x = D_w^* g = sum_n w_n D_n^T g_n, D_n^T g(v) = g(v - e_n) - g(v). */
int lrstv_diff_adjoint(const float *g, int n1, int n2, int n3, const float w[3], float *x,
                       void *stream);
/* y = R_d(x) = sign(x) max(|x| - d, 0) elementwise (Section III-C, step 3;
 * the printed second case is read as x < -d).  In place allowed. */
int lrstv_soft_threshold(const float *x, size_t n, float d, float *y, void *stream);

/* Scratch the standalone Z-solve and t-SVT need, in bytes (caller-owned,
 * device memory, 256-byte aligned). */
int lrstv_zsolve_workspace_size(int n1, int n2, int n3, size_t *bytes);
int lrstv_tsvt_workspace_size(int n1, int n2, int n3, size_t *bytes);
/* Z = ifftn(fftn(T) / (mu (1 + P_z))), P_z = sum_n w_n^2 |fftn(D_n)|^2
 * (eq. Z_solution).  ERR_ARG if the workspace is too small. */
int lrstv_zsolve(const float *T, int n1, int n2, int n3, const float w[3], float mu, float *Z,
                 void *workspace, size_t workspace_bytes, void *stream);
/* t-SVT of a real cube (eq. E_solution with Theorem 4.2's t-SVD): DFT along
 * mode 3, singular values of every Fourier frontal slice soft-thresholded by
 * t, inverse DFT.  `sweeps_host` (may be NULL) receives the largest Jacobi
 * sweep count, negative if a slice hit the cap (0 if every slice's Frobenius
 * norm is at most t, so that no sweep was needed); passing it synchronises. */
int lrstv_tsvt(const float *A, int n1, int n2, int n3, float t, float *out, void *workspace,
               size_t workspace_bytes, int *sweeps_host, void *stream);

/* ------------------------------------------------- allocation-free t-SVT */
/* The paper has no counterpart to this call: it serves callers that cannot
 * allocate device memory when they call the library (a plug-in whose host
 * application owns the device memory pool, a process that reserves all of its
 * device memory up front, a loop that must never reach the allocator).
 *
 * lrstv_tsvt_noalloc computes the same t-SVT as lrstv_tsvt, but takes its
 * scratch from one fixed device array of LRSTV_NOALLOC_SCRATCH_BYTES (16 MiB)
 * that is part of the library: every GPU that loads liblrstv.so holds that
 * array until the process exits.  The call allocates nothing (no cudaMalloc,
 * cudaFree or allocating library routine).  The caller passes A and out
 * (device, N floats each) as for lrstv_tsvt.
 *  - Size limit: 2*h*n1*n2*8 + h*min(n1,n2)^2*8 + n3*8 + h*4 bytes (h =
 *    n3/2 + 1, each term rounded up to 256) must not exceed the array;
 *    larger cubes return LRSTV_ERR_SHAPE without touching the GPU.  Examples
 *    that fit: 64x64x31, 128x128x31, 100x100x80.
 *  - The call works in the calling thread's current device and context and
 *    looks up the array's device address there (cudaGetSymbolAddress) on
 *    every call, so it stays valid if the host application destroys its
 *    context and makes a new one.  Make the first call on a device before
 *    any stream capture.
 *  - Under CUDA's lazy module loading (the default; CUDA_MODULE_LOADING=LAZY)
 *    the library's device code, and with it the 16 MiB array, is loaded into
 *    a context only when first used: the FIRST call in each context loads
 *    the modules it needs, and that load does reach the driver's allocator
 *    (and can fail with LRSTV_ERR_CUDA when the device is full).  A caller
 *    that must not see that at run time makes one call during its set-up
 *    (any cube that fits, e.g. 8x8x4), or sets CUDA_MODULE_LOADING=EAGER so
 *    that everything is loaded with the context; every later call allocates
 *    nothing.
 *  - Every call on a device shares the one array and leaves the last call's
 *    contents in it; each call writes every scratch byte before reading it,
 *    so nothing has to start at zero.  Calls that overlap on the GPU (on two
 *    streams, or from two host threads) race on the array and give wrong
 *    results: order them on one stream.
 *  - sweeps_host as in lrstv_tsvt (passing it synchronises `stream`). */
#define LRSTV_NOALLOC_SCRATCH_BYTES (16u << 20)
int lrstv_tsvt_noalloc(const float *A, int n1, int n2, int n3, float t, float *out,
                       int *sweeps_host, void *stream);

/* ------------------------------------ unrolled, differentiable iteration */
/* K iterations of Algorithm 1 (Section III-C, printed F threshold tau/mu,
 * Gamma4 updated) on a batch of B cubes of one shape, with free scalars per
 * iteration, and the exact gradient of a loss on the final L with respect to
 * those scalars and to Y.  The paper runs the iteration with fixed tau,
 * alpha, lambda and a geometric mu; here theta_k = (tau_k, alpha_k,
 * lambda_k, mu_k) for k = 0..K-1 are inputs (an unrolled solver whose scalars
 * are learned), and iteration k runs with mu = mu_k and no penalty update.
 * The start is the plan's: L = Z = Y, everything else zero.
 *
 * lrstv_unroll_create   allocates one device arena holding every iterate
 *   (K + 1 states of 17 B N floats, the per-iteration checkpoints), the SVD
 *   factors of every Fourier slice of every E-update (K x 3 B (n3/2+1)
 *   slices; one iteration's with LRSTV_FLAG_UNROLL_RECOMPUTE, which reruns
 *   each E-update's SVDs in the backward pass) and the scratch of both
 *   passes; lrstv_unroll_bytes reports its size.  w: weights of D_w (NULL =
 *   1, 1, 1).  flags: any of LRSTV_FLAG_SIMT_GEMM, LRSTV_FLAG_SIMT_DFT,
 *   LRSTV_FLAG_JACOBI_PER_SLICE, LRSTV_FLAG_JACOBI_PANEL16, LRSTV_FLAG_WARM_START (iteration
 *   k > 0 starts its Jacobi SVDs from iteration k-1's singular vectors, as a
 *   plan does), LRSTV_FLAG_UNROLL_RECOMPUTE.  iters in 1..4096.
 * lrstv_unroll_forward  Y: device, B cubes back to back (B N floats).
 *   theta: HOST array of K x 4 doubles (tau, alpha, lambda, mu per
 *   iteration; all finite and >= 0, mu > 0), copied during the call.
 *   X: device, B N floats (may be NULL): L after the K iterations.
 * lrstv_unroll_backward dX: device, B N floats: dLoss/dX.  dtheta: DEVICE
 *   array of K x 4 doubles, overwritten with dLoss/dtheta (same order as
 *   theta).  dY: device, B N floats (may be NULL): dLoss/dY.  Uses the last
 *   forward's theta and iterates; LRSTV_ERR_STATE before any forward.
 *   The soft-threshold masks are taken where the forward took them, and a
 *   voxel exactly on a threshold counts as cut.
 * lrstv_unroll_stats    (synchronises `stream`) unconverged: Fourier slices
 *   of the last forward whose Jacobi SVD hit its sweep cap; gemm_errors: 1 if
 *   a tensor-core GEMM's bounded wait ran out (either pointer may be NULL).
 * A forward or backward pass of one handle must not overlap another call of
 * that handle on the GPU. */
typedef struct lrstv_unroll lrstv_unroll;
int lrstv_unroll_create(int n1, int n2, int n3, int batch, int iters, const float w[3],
                        unsigned flags, lrstv_unroll **unroll);
int lrstv_unroll_destroy(lrstv_unroll *unroll);
int lrstv_unroll_bytes(const lrstv_unroll *unroll, size_t *bytes);
int lrstv_unroll_forward(lrstv_unroll *unroll, const float *Y, const double *theta, float *X,
                         void *stream);
int lrstv_unroll_backward(lrstv_unroll *unroll, const float *dX, double *dtheta, float *dY,
                          void *stream);
int lrstv_unroll_stats(lrstv_unroll *unroll, int *unconverged, int *gemm_errors, void *stream);

#ifdef __cplusplus
}
#endif
#endif
