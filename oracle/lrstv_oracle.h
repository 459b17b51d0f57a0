/*
 * lrstv_oracle.h -- FP64 CPU oracle of the plain-LRSTV ADMM iteration.
 *
 * TEST INFRASTRUCTURE ONLY.  This header and lrstv_oracle.c are the slow,
 * obviously-correct reference that the CUDA path is checked against.  Only
 * tests/, __graft_entry__.smoke() and the cpu_baseline / reference legs of
 * bench.py may load it.  It shares no code, header, table or constant with the
 * CUDA library (include/lrstv.h, paper_2204_12879_gb300/csrc/).
 *
 * Paper: "Low-rank Meets Sparseness: An Integrated Spatial-Spectral Total
 * Variation Approach to Hyperspectral Denoising", arXiv 2204.12879.
 *
 * Cube layout: element (i, j, k) of an n1 x n2 x n3 cube sits at
 * i + n1*(j + n2*k)  (mode 1 fastest, frontal slices contiguous).
 * Complex arrays are interleaved (re, im) pairs of doubles.
 *
 * ADMM state: one buffer of ORC_NSTATE*N doubles, blocks in this order
 * (the block index times N is the offset):
 *   0 Y (observation O)   1 L   2 Z   3 S   4 Gamma1   5 Gamma2
 *   6..8 F_1..F_3   9..11 E_1..E_3   12..14 Gamma3_1..3   15..17 Gamma4_1..3
 *
 * Parameter vector (doubles): ORC_P_* indices below.
 */
#ifndef LRSTV_ORACLE_H
#define LRSTV_ORACLE_H
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORC_P_TAU = 0, ORC_P_ALPHA, ORC_P_LAMBDA, ORC_P_W1, ORC_P_W2, ORC_P_W3,
  ORC_P_MU0, ORC_P_RHO, ORC_P_MUMAX, ORC_P_EPS, ORC_NPARAM
};

enum {
  ORC_Y = 0, ORC_L, ORC_Z, ORC_S, ORC_G1, ORC_G2,
  ORC_F = 6, ORC_E = 9, ORC_G3 = 12, ORC_G4 = 15, ORC_NSTATE = 18
};

/* flags */
#define ORC_FLAG_F_THRESH_EXACT 1 /* F threshold tau/(2 mu) instead of the printed tau/mu */
#define ORC_FLAG_NO_GAMMA4      2 /* literal multiplier list: Gamma4 never updated      */
#define ORC_FLAG_ISO_TV         4 /* isotropic LRSTV (eq. CRSSTV_iso): F thresholded per voxel
                                     as the 3-vector (F_1, F_2, F_3), by its 2-norm          */

/* Circular forward differences g_n = w_n D_n x, n = 1..3; g holds 3N doubles. */
void orc_diff(const double *x, int n1, int n2, int n3, const double *w, double *g);
/* Adjoint: x = sum_n w_n D_n^T g_n. */
void orc_diff_adjoint(const double *g, int n1, int n2, int n3, const double *w, double *x);

/* Naive DFT of a complex cube along one mode (axis 0, 1 or 2), in place.
 * sign = -1: forward, unnormalised.  sign = +1: inverse, scaled by 1/n_axis. */
void orc_dft_axis(double *a, int n1, int n2, int n3, int axis, int sign);
/* 3-D DFT (fftn / ifftn) of a complex cube, in place. */
void orc_dft3(double *a, int n1, int n2, int n3, int sign);

/* P_z = sum_n w_n^2 |fftn(D_n)|^2 as an N-sized real array. */
void orc_pz(int n1, int n2, int n3, const double *w, double *pz);
/* Z = ifftn(fftn(T) / (mu (1 + P_z))). */
void orc_zsolve(const double *T, int n1, int n2, int n3, const double *w, double mu, double *Z);

/* Soft threshold R_d(x) = sign(x) max(|x| - d, 0). */
double orc_soft(double x, double d);
/* Group soft threshold of x (m entries) in place: x max(1 - d/||x||_2, 0). */
void orc_group_soft(double *x, int m, double d);

/* SVT of one complex m x n column-major matrix, in place (one-sided Jacobi).
 * Returns the number of sweeps used (negative if the sweep cap was hit). */
int orc_svt_matrix(double *A, int m, int n, double t);
/* Singular values of a complex m x n column-major matrix (descending). */
int orc_singular_values(const double *A, int m, int n, double *sigma);
/* t-SVT of a real cube: threshold t on every Fourier frontal slice. */
int orc_tsvt(const double *A, int n1, int n2, int n3, double t, double *out);

/* ADMM (Algorithm 1 with the plain-LRSTV L-step). st: ORC_NSTATE*N doubles. */
void orc_init(const double *Y, int n1, int n2, int n3, double *st);
void orc_step_l(double *st, int n1, int n2, int n3, const double *p, double mu);
void orc_step_z(double *st, int n1, int n2, int n3, const double *p, double mu);
void orc_step_f(double *st, int n1, int n2, int n3, const double *p, double mu, int flags);
int  orc_step_e(double *st, int n1, int n2, int n3, const double *p, double mu);
void orc_step_s(double *st, int n1, int n2, int n3, const double *p, double mu);
void orc_step_dual(double *st, int n1, int n2, int n3, const double *p, double mu, int flags);
double orc_step_mu(const double *p, double mu);
/* max(||Y-L-S||_inf, ||L-Z||_inf) and the two parts in res[0], res[1]. */
double orc_residual(const double *st, int n1, int n2, int n3, double *res);
/* Runs `iters` iterations from state st and penalty *mu.  res_out (may be
 * NULL) receives 2 residuals per iteration.  Returns the largest Jacobi sweep
 * count used, negative if any slice hit the sweep cap. */
int orc_iterate(double *st, int n1, int n2, int n3, const double *p, double *mu,
                int iters, int flags, double *res_out);

int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
