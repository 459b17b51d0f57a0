"""FP64 reference of the TDLRSTV L-update: the Tucker projection of the
L-subproblem's target by HOOI (Section III-C, step 1, eq. X_solution with the
Tucker-3 model of eq. LRTAmodel).

TEST INFRASTRUCTURE ONLY (see the package docstring).  numpy, float64;
library eigen/SVD routines serve as steps.  Cubes are (n1, n2, n3) arrays.

Readings (the paper names HOOI but not its schedule):
 - ranks (r1, r2, r3) are given; the paper sets r1 = 0.8 n1, r2 = 0.8 n2 and
   tunes r3;
 - each ADMM iteration runs ONE HOOI sweep (factors updated in the order
   U1, U2, U3, each from the current others), starting from the previous
   ADMM iteration's factors; the first ADMM iteration starts from the
   truncated HOSVD of its target;
 - U_n holds the r_n leading eigenvectors of the mode-n Gram matrix of the
   target multiplied by the other factors' transposes (the leading left
   singular vectors of that unfolding);
 - L = X x1 U1 U1^T x2 U2 U2^T x3 U3 U3^T (core, then expansion).
"""
from __future__ import annotations

import numpy as np

__all__ = ["unfold", "mode_product", "leading_eigvecs", "hosvd", "hooi_sweep", "project",
           "tucker_l_update", "TuckerState"]


def unfold(X, n):
    """Mode-n unfolding: rows indexed by mode n, columns by the other modes."""
    return np.moveaxis(np.asarray(X), n, 0).reshape(X.shape[n], -1)


def mode_product(X, M, n):
    """X x_n M: contracts mode n of X with the columns of M (M is m x n_n)."""
    Y = np.tensordot(M, np.moveaxis(X, n, 0), axes=(1, 0))
    return np.moveaxis(Y, 0, n)


def leading_eigvecs(G, r):
    """The r eigenvectors of the symmetric matrix G with the largest
    eigenvalues (columns, in decreasing order)."""
    w, V = np.linalg.eigh(G)
    return V[:, ::-1][:, :r]


def hosvd(X, ranks):
    """Truncated HOSVD factors: leading eigenvectors of every mode's Gram."""
    return [leading_eigvecs(unfold(X, n) @ unfold(X, n).T, ranks[n]) for n in range(3)]


def hooi_sweep(X, U, ranks):
    """One HOOI sweep: U_n <- leading eigenvectors of the mode-n Gram of
    X multiplied by the other (current) factors' transposes, n = 1, 2, 3."""
    U = list(U)
    for n in range(3):
        Z = X
        for m in range(3):
            if m != n:
                Z = mode_product(Z, U[m].T, m)
        Zn = unfold(Z, n)
        U[n] = leading_eigvecs(Zn @ Zn.T, ranks[n])
    return U


def project(X, U):
    """X x1 U1 U1^T x2 U2 U2^T x3 U3 U3^T."""
    C = X
    for n in range(3):
        C = mode_product(C, U[n].T, n)
    L = C
    for n in range(3):
        L = mode_product(L, U[n], n)
    return L


def tucker_l_update(X, U_prev, ranks):
    """The L-update: one HOOI sweep from U_prev (or from the truncated HOSVD
    of X when U_prev is None), then the projection.  Returns (L, U)."""
    U = hosvd(X, ranks) if U_prev is None else U_prev
    U = hooi_sweep(X, U, ranks)
    return project(X, U), U


class TuckerState:
    """Algorithm 1 with the Tucker L-update on the C oracle's state: the
    target 1/2 (Y - S + Z + (Gamma1 - Gamma2)/mu) is formed here, projected
    by tucker_l_update, and every other step runs in the C oracle."""

    def __init__(self, orc, Y, params, ranks, flags=0):
        self.st = orc.State(Y, params, flags=flags)
        self.ranks = tuple(int(r) for r in ranks)
        self.U = None

    def step_l(self):
        s = self.st
        T = 0.5 * (s.get("Y") - s.get("S") + s.get("Z") + (s.get("G1") - s.get("G2")) / s.mu)
        L, self.U = tucker_l_update(T, self.U, self.ranks)
        s.set("L", L)

    def iterate(self, iters):
        s = self.st
        for _ in range(iters):
            self.step_l()
            s.step_z()
            s.step_f()
            s.step_e()
            s.step_s()
            s.step_dual()
            s.step_mu()
            s.iters += 1

    @property
    def X(self):
        return self.st.X
