/*
 * lrstv_oracle.c -- FP64 CPU oracle of the plain-LRSTV ADMM iteration
 * (arXiv 2204.12879, Section III-C and Algorithm 1).
 *
 * TEST INFRASTRUCTURE ONLY: the reference the CUDA path is checked against.
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline and
 * reference legs may load it.  It shares no code with the CUDA library.
 *
 * Deliberately plain: naive O(n^2) DFTs along each mode (no FFT), a full
 * complex 3-D spectrum (no half-spectrum trick), every Fourier slice
 * thresholded on its own (no conjugate-symmetry shortcut), and a one-sided
 * (Hestenes) Jacobi SVD per slice.  OpenMP only splits independent outputs, so
 * results do not depend on the thread count.
 *
 * Readings of the paper where it is silent or inconsistent (all selectable
 * where they change results):
 *  - Plain LRSTV: the Tucker constraint is dropped, so the HOOI step of the
 *    L-update (eq. X_solution) with full ranks is the identity and
 *    L = (Y - S + Z + (Gamma1 - Gamma2)/mu) / 2.
 *  - F threshold: tau/mu as printed (eq. F_solution); ORC_FLAG_F_THRESH_EXACT
 *    gives tau/(2 mu), the exact minimiser of the printed subproblem.
 *  - Update order: Algorithm 1, L -> Z -> F -> E -> S -> multipliers -> mu,
 *    so the F-update reads the previous E.
 *  - Gamma4 is updated like the other multipliers, Gamma4 += mu (E - F);
 *    ORC_FLAG_NO_GAMMA4 keeps the printed multiplier list (Gamma1..3 only).
 *  - The soft-threshold's second case reads x < -Delta.
 *  - D_n are circular forward differences; D_1 runs along mode 1.
 *  - t-SVT thresholds every Fourier frontal slice's singular values by the
 *    same alpha/mu (Theorem 4.2 with an unnormalised mode-3 DFT).
 */
#include "lrstv_oracle.h"

#include <complex.h>
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORC_PI 3.14159265358979323846264338327950288

static size_t vol(int n1, int n2, int n3) { return (size_t)n1 * (size_t)n2 * (size_t)n3; }
static size_t at(int n1, int n2, int i, int j, int k) {
  return (size_t)i + (size_t)n1 * ((size_t)j + (size_t)n2 * (size_t)k);
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---------------------------------------------------------------- D_n ---- */
/* D_n x(v) = x(v + e_n) - x(v), periodic boundary (Section III-A, the
 * circulant difference matrix of Theorem 4.1). */
void orc_diff(const double *x, int n1, int n2, int n3, const double *w, double *g) {
  size_t N = vol(n1, n2, n3);
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < n3; ++k)
    for (int j = 0; j < n2; ++j)
      for (int i = 0; i < n1; ++i) {
        size_t v = at(n1, n2, i, j, k);
        double xv = x[v];
        g[v] = w[0] * (x[at(n1, n2, (i + 1) % n1, j, k)] - xv);
        g[N + v] = w[1] * (x[at(n1, n2, i, (j + 1) % n2, k)] - xv);
        g[2 * N + v] = w[2] * (x[at(n1, n2, i, j, (k + 1) % n3)] - xv);
      }
}

/* D_n^T g(v) = g(v - e_n) - g(v): the transpose of the circulant above. */
void orc_diff_adjoint(const double *g, int n1, int n2, int n3, const double *w, double *x) {
  size_t N = vol(n1, n2, n3);
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < n3; ++k)
    for (int j = 0; j < n2; ++j)
      for (int i = 0; i < n1; ++i) {
        size_t v = at(n1, n2, i, j, k);
        double s = 0.0;
        s += w[0] * (g[at(n1, n2, (i + n1 - 1) % n1, j, k)] - g[v]);
        s += w[1] * (g[N + at(n1, n2, i, (j + n2 - 1) % n2, k)] - g[N + v]);
        s += w[2] * (g[2 * N + at(n1, n2, i, j, (k + n3 - 1) % n3)] - g[2 * N + v]);
        x[v] = s;
      }
}

/* ---------------------------------------------------------------- DFT ---- */
/* y[u] = sum_t x[t] exp(sign 2 pi i u t / n), scaled by 1/n when sign = +1.
 * Applied along one mode of a complex cube; every output is a direct sum. */
void orc_dft_axis(double *a_, int n1, int n2, int n3, int axis, int sign) {
  cplx *a = (cplx *)a_;
  int dims[3] = {n1, n2, n3};
  int n = dims[axis];
  size_t stride = axis == 0 ? 1 : (axis == 1 ? (size_t)n1 : (size_t)n1 * n2);
  size_t nfib = vol(n1, n2, n3) / (size_t)n;
  cplx *tw = (cplx *)malloc(sizeof(cplx) * (size_t)n);
  for (int m = 0; m < n; ++m) {
    double ang = 2.0 * ORC_PI * (double)m / (double)n;
    tw[m] = cos(ang) + (double)sign * sin(ang) * I;
  }
  double scale = sign > 0 ? 1.0 / (double)n : 1.0;
#pragma omp parallel
  {
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)n);
#pragma omp for schedule(static)
    for (size_t f = 0; f < nfib; ++f) {
      /* fiber f: the base index enumerates the other two modes */
      size_t base;
      if (axis == 0) base = f * (size_t)n1;
      else if (axis == 1) base = (f % (size_t)n1) + (f / (size_t)n1) * (size_t)n1 * n2;
      else base = f;
      for (int t = 0; t < n; ++t) tmp[t] = a[base + (size_t)t * stride];
      for (int u = 0; u < n; ++u) {
        cplx acc = 0.0;
        for (int t = 0; t < n; ++t) acc += tmp[t] * tw[((size_t)u * (size_t)t) % (size_t)n];
        a[base + (size_t)u * stride] = acc * scale;
      }
    }
    free(tmp);
  }
  free(tw);
}

void orc_dft3(double *a, int n1, int n2, int n3, int sign) {
  orc_dft_axis(a, n1, n2, n3, 0, sign);
  orc_dft_axis(a, n1, n2, n3, 1, sign);
  orc_dft_axis(a, n1, n2, n3, 2, sign);
}

/* ----------------------------------------------------------- Z-update ---- */
/* P_z = sum_n w_n^2 |fftn(D_n)|^2 (eq. Z_solution): the point-spread array of
 * D_n (-1 at the origin, +1 one step back along mode n, so that convolving
 * with it gives x(v + e_n) - x(v)) is transformed with the 3-D DFT. */
void orc_pz(int n1, int n2, int n3, const double *w, double *pz) {
  size_t N = vol(n1, n2, n3);
  int dims[3] = {n1, n2, n3};
  double *psf = (double *)malloc(sizeof(double) * 2 * N);
  for (size_t v = 0; v < N; ++v) pz[v] = 0.0;
  for (int n = 0; n < 3; ++n) {
    memset(psf, 0, sizeof(double) * 2 * N);
    int c[3] = {0, 0, 0};
    psf[0] = -1.0;
    c[n] = (dims[n] - 1) % dims[n];
    size_t v1 = at(n1, n2, c[0], c[1], c[2]);
    psf[2 * v1] += 1.0;
    orc_dft3(psf, n1, n2, n3, -1);
    for (size_t v = 0; v < N; ++v) {
      double re = psf[2 * v], im = psf[2 * v + 1];
      pz[v] += w[n] * w[n] * (re * re + im * im);
    }
  }
  free(psf);
}

/* Solve mu (I + D_w^* D_w) Z = T by the 3-D DFT (eq. Z_solution). */
void orc_zsolve(const double *T, int n1, int n2, int n3, const double *w, double mu, double *Z) {
  size_t N = vol(n1, n2, n3);
  double *a = (double *)malloc(sizeof(double) * 2 * N);
  double *pz = (double *)malloc(sizeof(double) * N);
  orc_pz(n1, n2, n3, w, pz);
  for (size_t v = 0; v < N; ++v) { a[2 * v] = T[v]; a[2 * v + 1] = 0.0; }
  orc_dft3(a, n1, n2, n3, -1);
  for (size_t v = 0; v < N; ++v) {
    double d = mu + mu * pz[v];
    a[2 * v] /= d;
    a[2 * v + 1] /= d;
  }
  orc_dft3(a, n1, n2, n3, +1);
  for (size_t v = 0; v < N; ++v) Z[v] = a[2 * v];
  free(pz);
  free(a);
}

/* ------------------------------------------------------ soft threshold ---- */
/* R_d(x) (Section III-C, step 3), with the second case read as x < -d. */
double orc_soft(double x, double d) {
  if (x > d) return x - d;
  if (x < -d) return x + d;
  return 0.0;
}

/* ------------------------------------------------------------ SVT ------- */
/* One-sided (Hestenes) Jacobi on the columns of W (nr x nc, nr >= nc),
 * accumulating the same unitary column operations in V (nc x nc).  A pair
 * (p, q) is rotated until |w_p^H w_q| <= tol sqrt(|w_p|^2 |w_q|^2). */
static int hestenes(cplx *W, int nr, int nc, cplx *V) {
  const int max_sweeps = 80;
  const double tol = (double)nr * DBL_EPSILON;
  /* A column whose squared norm is below (nr eps)^2 ||W||_F^2 is rounding
   * residue: its direction cannot be resolved and its singular value is zero
   * to working precision, so it takes part in no rotation. */
  double fro2 = 0.0;
  for (size_t r = 0; r < (size_t)nr * nc; ++r)
    fro2 += creal(W[r]) * creal(W[r]) + cimag(W[r]) * cimag(W[r]);
  const double negl = tol * tol * fro2;
  for (int i = 0; i < nc; ++i)
    for (int j = 0; j < nc; ++j) V[(size_t)i + (size_t)nc * j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 1; sweep <= max_sweeps; ++sweep) {
    int rotated = 0;
    for (int p = 0; p < nc - 1; ++p)
      for (int q = p + 1; q < nc; ++q) {
        cplx *wp = W + (size_t)nr * p, *wq = W + (size_t)nr * q;
        double alpha = 0.0, beta = 0.0;
        cplx gamma = 0.0;
        for (int r = 0; r < nr; ++r) {
          alpha += creal(wp[r]) * creal(wp[r]) + cimag(wp[r]) * cimag(wp[r]);
          beta += creal(wq[r]) * creal(wq[r]) + cimag(wq[r]) * cimag(wq[r]);
          gamma += conj(wp[r]) * wq[r];
        }
        double ag = cabs(gamma);
        if (alpha <= negl || beta <= negl) continue;
        if (ag == 0.0 || ag <= tol * sqrt(alpha * beta)) continue;
        rotated = 1;
        /* 2x2 Hermitian [[alpha, gamma], [conj(gamma), beta]]: remove the
         * phase of gamma, then the real symmetric Schur rotation. */
        double zeta = (beta - alpha) / (2.0 * ag);
        double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t);
        double s = c * t;
        cplx e = conj(gamma) / ag;
        for (int r = 0; r < nr; ++r) {
          cplx a = wp[r], b = e * wq[r];
          wp[r] = c * a - s * b;
          wq[r] = s * a + c * b;
        }
        cplx *vp = V + (size_t)nc * p, *vq = V + (size_t)nc * q;
        for (int r = 0; r < nc; ++r) {
          cplx a = vp[r], b = e * vq[r];
          vp[r] = c * a - s * b;
          vq[r] = s * a + c * b;
        }
      }
    if (!rotated) return sweep;
  }
  return -max_sweeps;
}

/* Copies A (m x n) into the working matrix W = A (m >= n) or W = A^H. */
static void to_work(const cplx *A, int m, int n, cplx *W) {
  if (m >= n) {
    memcpy(W, A, sizeof(cplx) * (size_t)m * n);
  } else {
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < n; ++j) W[(size_t)j + (size_t)n * i] = conj(A[(size_t)i + (size_t)m * j]);
  }
}

/* SVT_t(A) = U max(Sigma - t, 0) V^H (eq. E_solution), in place.  With
 * W V = U Sigma from Jacobi: SVT_t(W) = sum_i max(1 - t/sigma_i, 0) w_i v_i^H. */
int orc_svt_matrix(double *A_, int m, int n, double t) {
  cplx *A = (cplx *)A_;
  int nr = m >= n ? m : n, nc = m >= n ? n : m;
  cplx *W = (cplx *)malloc(sizeof(cplx) * (size_t)nr * nc);
  cplx *V = (cplx *)malloc(sizeof(cplx) * (size_t)nc * nc);
  double *g = (double *)malloc(sizeof(double) * (size_t)nc);
  to_work(A, m, n, W);
  int sweeps = hestenes(W, nr, nc, V);
  for (int i = 0; i < nc; ++i) {
    double s2 = 0.0;
    for (int r = 0; r < nr; ++r) {
      cplx x = W[(size_t)r + (size_t)nr * i];
      s2 += creal(x) * creal(x) + cimag(x) * cimag(x);
    }
    double sigma = sqrt(s2);
    g[i] = sigma > t ? 1.0 - t / sigma : 0.0;
  }
  for (int r = 0; r < nr; ++r)
    for (int c = 0; c < nc; ++c) {
      cplx acc = 0.0;
      for (int i = 0; i < nc; ++i)
        acc += g[i] * W[(size_t)r + (size_t)nr * i] * conj(V[(size_t)c + (size_t)nc * i]);
      /* R(r, c) of the working orientation; undo the transpose if taken */
      if (m >= n) A[(size_t)r + (size_t)m * c] = acc;
      else A[(size_t)c + (size_t)m * r] = conj(acc);
    }
  free(g);
  free(V);
  free(W);
  return sweeps;
}

/* Combines two sweep counts: negative (cap hit) wins, else the larger. */
static int merge_sweeps(int a, int b) {
  if (a < 0 || b < 0) return a < b ? a : b;
  return a > b ? a : b;
}

static int cmp_desc(const void *a, const void *b) {
  double x = *(const double *)a, y = *(const double *)b;
  return (x < y) - (x > y);
}

int orc_singular_values(const double *A_, int m, int n, double *sigma) {
  const cplx *A = (const cplx *)A_;
  int nr = m >= n ? m : n, nc = m >= n ? n : m;
  cplx *W = (cplx *)malloc(sizeof(cplx) * (size_t)nr * nc);
  cplx *V = (cplx *)malloc(sizeof(cplx) * (size_t)nc * nc);
  to_work(A, m, n, W);
  int sweeps = hestenes(W, nr, nc, V);
  for (int i = 0; i < nc; ++i) {
    double s2 = 0.0;
    for (int r = 0; r < nr; ++r) {
      cplx x = W[(size_t)r + (size_t)nr * i];
      s2 += creal(x) * creal(x) + cimag(x) * cimag(x);
    }
    sigma[i] = sqrt(s2);
  }
  qsort(sigma, (size_t)nc, sizeof(double), cmp_desc);
  free(V);
  free(W);
  return sweeps;
}

/* t-SVT (eq. E_solution with the t-SVD of Theorem 4.2): DFT along mode 3,
 * SVT of every frontal slice with threshold t, inverse DFT. */
int orc_tsvt(const double *A, int n1, int n2, int n3, double t, double *out) {
  size_t N = vol(n1, n2, n3), P = (size_t)n1 * n2;
  double *a = (double *)malloc(sizeof(double) * 2 * N);
  int *sw = (int *)malloc(sizeof(int) * (size_t)n3);
  for (size_t v = 0; v < N; ++v) { a[2 * v] = A[v]; a[2 * v + 1] = 0.0; }
  orc_dft_axis(a, n1, n2, n3, 2, -1);
#pragma omp parallel for schedule(dynamic, 1)
  for (int k = 0; k < n3; ++k) sw[k] = orc_svt_matrix(a + 2 * P * (size_t)k, n1, n2, t);
  orc_dft_axis(a, n1, n2, n3, 2, +1);
  for (size_t v = 0; v < N; ++v) out[v] = a[2 * v];
  int worst = 0;
  for (int k = 0; k < n3; ++k) worst = merge_sweeps(worst, sw[k]);
  free(sw);
  free(a);
  return worst;
}

/* --------------------------------------------------------------- ADMM ---- */
#define BLK(st, b) ((st) + (size_t)(b) * N)

/* Initialisation (left empty by Algorithm 1): L = Z = Y, everything else 0. */
void orc_init(const double *Y, int n1, int n2, int n3, double *st) {
  size_t N = vol(n1, n2, n3);
  memset(st, 0, sizeof(double) * N * ORC_NSTATE);
  memcpy(BLK(st, ORC_Y), Y, sizeof(double) * N);
  memcpy(BLK(st, ORC_L), Y, sizeof(double) * N);
  memcpy(BLK(st, ORC_Z), Y, sizeof(double) * N);
}

/* Step 1 (eq. X_solution, full Tucker ranks). */
void orc_step_l(double *st, int n1, int n2, int n3, const double *p, double mu) {
  size_t N = vol(n1, n2, n3);
  (void)p;
  const double *Y = BLK(st, ORC_Y), *S = BLK(st, ORC_S), *Z = BLK(st, ORC_Z);
  const double *G1 = BLK(st, ORC_G1), *G2 = BLK(st, ORC_G2);
  double *L = BLK(st, ORC_L);
#pragma omp parallel for schedule(static)
  for (size_t v = 0; v < N; ++v) L[v] = 0.5 * (Y[v] - S[v] + Z[v] + (G1[v] - G2[v]) / mu);
}

/* Step 2 (eq. Z_solution): T_z = mu L + mu D_w^*(F) + Gamma2 - D_w^*(Gamma3). */
void orc_step_z(double *st, int n1, int n2, int n3, const double *p, double mu) {
  size_t N = vol(n1, n2, n3);
  const double *w = p + ORC_P_W1;
  double *T = (double *)malloc(sizeof(double) * N);
  double *aF = (double *)malloc(sizeof(double) * N);
  double *aG = (double *)malloc(sizeof(double) * N);
  orc_diff_adjoint(BLK(st, ORC_F), n1, n2, n3, w, aF);
  orc_diff_adjoint(BLK(st, ORC_G3), n1, n2, n3, w, aG);
  const double *L = BLK(st, ORC_L), *G2 = BLK(st, ORC_G2);
  for (size_t v = 0; v < N; ++v) T[v] = mu * L[v] + mu * aF[v] + G2[v] - aG[v];
  orc_zsolve(T, n1, n2, n3, w, mu, BLK(st, ORC_Z));
  free(aG);
  free(aF);
  free(T);
}

/* Group soft threshold (the prox of d ||.||_2 on R^m): x scaled by
 * max(1 - d / ||x||_2, 0), zero when ||x||_2 <= d. */
void orc_group_soft(double *x, int m, double d) {
  double s = 0.0;
  for (int i = 0; i < m; ++i) s += x[i] * x[i];
  const double nrm = sqrt(s);
  const double g = nrm > d ? 1.0 - d / nrm : 0.0;
  for (int i = 0; i < m; ++i) x[i] *= g;
}

/* Step 3 (eq. F_solution): F = R_{tau/mu}((T1 + T2)/2),
 * T1 = D_w Z + Gamma3/mu, T2 = E + Gamma4/mu.  Isotropic LRSTV (eq. CRSSTV_iso,
 * with the per-pixel 2-norm of the isotropic TV of Section II-B and
 * tau_n = (tau w_n)^2): the soft threshold becomes the group threshold of the
 * 3-vector (F_1, F_2, F_3) at each voxel. */
void orc_step_f(double *st, int n1, int n2, int n3, const double *p, double mu, int flags) {
  size_t N = vol(n1, n2, n3);
  double *g = (double *)malloc(sizeof(double) * 3 * N);
  orc_diff(BLK(st, ORC_Z), n1, n2, n3, p + ORC_P_W1, g);
  double thr = (flags & ORC_FLAG_F_THRESH_EXACT) ? p[ORC_P_TAU] / (2.0 * mu) : p[ORC_P_TAU] / mu;
  double *F = BLK(st, ORC_F);
  const double *E = BLK(st, ORC_E), *G3 = BLK(st, ORC_G3), *G4 = BLK(st, ORC_G4);
  if (flags & ORC_FLAG_ISO_TV) {
#pragma omp parallel for schedule(static)
    for (size_t v = 0; v < N; ++v) {
      double x[3];
      for (int n = 0; n < 3; ++n) {
        const size_t u = v + (size_t)n * N;
        x[n] = 0.5 * ((g[u] + G3[u] / mu) + (E[u] + G4[u] / mu));
      }
      orc_group_soft(x, 3, thr);
      for (int n = 0; n < 3; ++n) F[v + (size_t)n * N] = x[n];
    }
    free(g);
    return;
  }
#pragma omp parallel for schedule(static)
  for (size_t v = 0; v < 3 * N; ++v) {
    double t1 = g[v] + G3[v] / mu, t2 = E[v] + G4[v] / mu;
    F[v] = orc_soft(0.5 * (t1 + t2), thr);
  }
  free(g);
}

/* Step 4 (eq. E_solution): E_n = t-SVT(F_n - Gamma4_n/mu, alpha/mu). */
int orc_step_e(double *st, int n1, int n2, int n3, const double *p, double mu) {
  size_t N = vol(n1, n2, n3);
  double *B = (double *)malloc(sizeof(double) * N);
  int worst = 0;
  for (int n = 0; n < 3; ++n) {
    const double *F = BLK(st, ORC_F + n), *G4 = BLK(st, ORC_G4 + n);
    for (size_t v = 0; v < N; ++v) B[v] = F[v] - G4[v] / mu;
    worst = merge_sweeps(worst, orc_tsvt(B, n1, n2, n3, p[ORC_P_ALPHA] / mu, BLK(st, ORC_E + n)));
  }
  free(B);
  return worst;
}

/* Step 5 (eq. S_solution): S = R_{lambda/mu}(Y - L + Gamma1/mu). */
void orc_step_s(double *st, int n1, int n2, int n3, const double *p, double mu) {
  size_t N = vol(n1, n2, n3);
  const double *Y = BLK(st, ORC_Y), *L = BLK(st, ORC_L), *G1 = BLK(st, ORC_G1);
  double *S = BLK(st, ORC_S);
  double thr = p[ORC_P_LAMBDA] / mu;
#pragma omp parallel for schedule(static)
  for (size_t v = 0; v < N; ++v) S[v] = orc_soft(Y[v] - L[v] + G1[v] / mu, thr);
}

/* Step 6 (eq. Multipliers), plus Gamma4 += mu (E - F). */
void orc_step_dual(double *st, int n1, int n2, int n3, const double *p, double mu, int flags) {
  size_t N = vol(n1, n2, n3);
  double *g = (double *)malloc(sizeof(double) * 3 * N);
  orc_diff(BLK(st, ORC_Z), n1, n2, n3, p + ORC_P_W1, g);
  const double *Y = BLK(st, ORC_Y), *L = BLK(st, ORC_L), *S = BLK(st, ORC_S);
  const double *Z = BLK(st, ORC_Z), *F = BLK(st, ORC_F), *E = BLK(st, ORC_E);
  double *G1 = BLK(st, ORC_G1), *G2 = BLK(st, ORC_G2), *G3 = BLK(st, ORC_G3), *G4 = BLK(st, ORC_G4);
#pragma omp parallel for schedule(static)
  for (size_t v = 0; v < N; ++v) {
    G1[v] += mu * (Y[v] - L[v] - S[v]);
    G2[v] += mu * (L[v] - Z[v]);
  }
#pragma omp parallel for schedule(static)
  for (size_t v = 0; v < 3 * N; ++v) {
    G3[v] += mu * (g[v] - F[v]);
    if (!(flags & ORC_FLAG_NO_GAMMA4)) G4[v] += mu * (E[v] - F[v]);
  }
  free(g);
}

/* Step 7: mu := min(rho mu, mu_max). */
double orc_step_mu(const double *p, double mu) {
  double m = p[ORC_P_RHO] * mu;
  return m < p[ORC_P_MUMAX] ? m : p[ORC_P_MUMAX];
}

/* Convergence check of Algorithm 1. */
double orc_residual(const double *st, int n1, int n2, int n3, double *res) {
  size_t N = vol(n1, n2, n3);
  const double *Y = BLK(st, ORC_Y), *L = BLK(st, ORC_L), *S = BLK(st, ORC_S), *Z = BLK(st, ORC_Z);
  double r0 = 0.0, r1 = 0.0;
  for (size_t v = 0; v < N; ++v) {
    double a = fabs(Y[v] - L[v] - S[v]), b = fabs(L[v] - Z[v]);
    if (a > r0) r0 = a;
    if (b > r1) r1 = b;
  }
  if (res) { res[0] = r0; res[1] = r1; }
  return r0 > r1 ? r0 : r1;
}

int orc_iterate(double *st, int n1, int n2, int n3, const double *p, double *mu,
                int iters, int flags, double *res_out) {
  int worst = 0;
  for (int it = 0; it < iters; ++it) {
    double m = *mu;
    orc_step_l(st, n1, n2, n3, p, m);
    orc_step_z(st, n1, n2, n3, p, m);
    orc_step_f(st, n1, n2, n3, p, m, flags);
    worst = merge_sweeps(worst, orc_step_e(st, n1, n2, n3, p, m));
    orc_step_s(st, n1, n2, n3, p, m);
    orc_step_dual(st, n1, n2, n3, p, m, flags);
    *mu = orc_step_mu(p, m);
    if (res_out) orc_residual(st, n1, n2, n3, res_out + 2 * (size_t)it);
  }
  return worst;
}
