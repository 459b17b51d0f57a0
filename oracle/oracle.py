"""ctypes front end of the FP64 C oracle (``lrstv_oracle.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Each function cites
the passage of arXiv 2204.12879 whose computation the C routine performs.
Arrays are numpy float64 / complex128 in the cube layout
``(i, j, k) -> i + n1*(j + n2*k)``, i.e. numpy arrays of shape (n1, n2, n3)
in Fortran order, or flat vectors in that order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

__all__ = [
    "build_oracle", "lib", "Params", "diff", "diff_adjoint", "dft_axis", "dft3",
    "pz", "zsolve", "soft", "group_soft", "svt_matrix", "singular_values", "tsvt",
    "State", "NSTATE", "BLOCKS", "num_threads", "mpsnr",
    "FLAG_F_THRESH_EXACT", "FLAG_NO_GAMMA4", "FLAG_ISO_TV",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lrstv_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liblrstv_oracle.so")
_lock = threading.Lock()
_lib = None

FLAG_F_THRESH_EXACT = 1
FLAG_NO_GAMMA4 = 2
FLAG_ISO_TV = 4

NSTATE = 18
BLOCKS = {"Y": 0, "L": 1, "Z": 2, "S": 3, "G1": 4, "G2": 5,
          "F": 6, "E": 9, "G3": 12, "G4": 15}


def build_oracle(force: bool = False) -> str:
    """Compiles the oracle with gcc (FP64, OpenMP, no FMA contraction)."""
    with _lock:
        if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < max(
                os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "lrstv_oracle.h"))):
            os.makedirs(os.path.dirname(_OUT), exist_ok=True)
            tmp = _OUT + f".tmp{os.getpid()}"
            subprocess.check_call([
                "gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                "-std=gnu11", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _OUT)
    return _OUT


def load_library(path: str):
    """Loads an oracle shared library and declares its C signatures."""
    L = ctypes.CDLL(path)
    if True:
        D = ctypes.POINTER(ctypes.c_double)
        i = ctypes.c_int
        d = ctypes.c_double
        sig = {
            "orc_diff": (None, [D, i, i, i, D, D]),
            "orc_diff_adjoint": (None, [D, i, i, i, D, D]),
            "orc_dft_axis": (None, [D, i, i, i, i, i]),
            "orc_dft3": (None, [D, i, i, i, i]),
            "orc_pz": (None, [i, i, i, D, D]),
            "orc_zsolve": (None, [D, i, i, i, D, d, D]),
            "orc_soft": (d, [d, d]),
            "orc_group_soft": (None, [D, i, d]),
            "orc_svt_matrix": (i, [D, i, i, d]),
            "orc_singular_values": (i, [D, i, i, D]),
            "orc_tsvt": (i, [D, i, i, i, d, D]),
            "orc_init": (None, [D, i, i, i, D]),
            "orc_step_l": (None, [D, i, i, i, D, d]),
            "orc_step_z": (None, [D, i, i, i, D, d]),
            "orc_step_f": (None, [D, i, i, i, D, d, i]),
            "orc_step_e": (i, [D, i, i, i, D, d]),
            "orc_step_s": (None, [D, i, i, i, D, d]),
            "orc_step_dual": (None, [D, i, i, i, D, d, i]),
            "orc_step_mu": (d, [D, d]),
            "orc_residual": (d, [D, i, i, i, D]),
            "orc_iterate": (i, [D, i, i, i, D, D, i, i, D]),
            "orc_num_threads": (i, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = load_library(build_oracle())
    return _lib


def _p(a: np.ndarray):
    if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("oracle arrays must be contiguous float64")
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _flat(x) -> np.ndarray:
    """Cube (n1, n2, n3) -> flat float64 vector in the i + n1 (j + n2 k) order."""
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1, order="F"))


def _cube(v: np.ndarray, shape) -> np.ndarray:
    return np.asarray(v).reshape(shape, order="F")


def num_threads() -> int:
    return lib().orc_num_threads()


class Params:
    """The scalars of Algorithm 1: tau (gradient L1), alpha (gradient TNN),
    lambda (sparse noise), weights w_1..w_3 of D_w, the penalty schedule
    mu0 / rho / mu_max and the stopping tolerance eps (Section III-C)."""

    def __init__(self, tau=0.001, alpha=0.2, lam=None, w=(1.0, 1.0, 1.0), mu0=1e-2,
                 rho=1.5, mu_max=1e6, eps=1e-6, n1=None, n2=None, C=1.0):
        if lam is None:
            # lambda = C / sqrt(M N), M N the spatial size (Section IV-D)
            lam = C / np.sqrt(float(n1 * n2)) if n1 else 0.1
        self.tau, self.alpha, self.lam = float(tau), float(alpha), float(lam)
        self.w = tuple(float(x) for x in w)
        self.mu0, self.rho, self.mu_max, self.eps = float(mu0), float(rho), float(mu_max), float(eps)

    def vector(self) -> np.ndarray:
        return np.array([self.tau, self.alpha, self.lam, *self.w, self.mu0, self.rho,
                         self.mu_max, self.eps], dtype=np.float64)


def diff(x, w=(1.0, 1.0, 1.0)):
    """w_n D_n x for n = 1..3 (circular forward differences, Section III-A).
    Returns an array of shape (3, n1, n2, n3)."""
    x = np.asarray(x, dtype=np.float64)
    n1, n2, n3 = x.shape
    g = np.empty(3 * x.size)
    lib().orc_diff(_p(_flat(x)), n1, n2, n3, _p(np.asarray(w, np.float64)), _p(g))
    return np.stack([_cube(g[n * x.size:(n + 1) * x.size], x.shape) for n in range(3)])


def diff_adjoint(g, w=(1.0, 1.0, 1.0)):
    """sum_n w_n D_n^T g_n, the adjoint D_w^* of eq. Z_solution."""
    g = np.asarray(g, dtype=np.float64)
    shape = g.shape[1:]
    flat = np.concatenate([_flat(g[n]) for n in range(3)])
    x = np.empty(flat.size // 3)
    lib().orc_diff_adjoint(_p(flat), *shape, _p(np.asarray(w, np.float64)), _p(x))
    return _cube(x, shape)


def dft_axis(a, axis, sign=-1):
    """Naive DFT of a complex cube along one mode (sign=+1: inverse with 1/n)."""
    a = np.asarray(a, dtype=np.complex128)
    v = np.ascontiguousarray(a.reshape(-1, order="F")).view(np.float64).copy()
    lib().orc_dft_axis(_p(v), *a.shape, int(axis), int(sign))
    return v.view(np.complex128).reshape(a.shape, order="F")


def dft3(a, sign=-1):
    """fftn (sign=-1) / ifftn (sign=+1) of eq. Z_solution, by direct sums."""
    a = np.asarray(a, dtype=np.complex128)
    v = np.ascontiguousarray(a.reshape(-1, order="F")).view(np.float64).copy()
    lib().orc_dft3(_p(v), *a.shape, int(sign))
    return v.view(np.complex128).reshape(a.shape, order="F")


def pz(shape, w=(1.0, 1.0, 1.0)):
    """P_z = sum_n w_n^2 |fftn(D_n)|^2 (eq. Z_solution)."""
    out = np.empty(int(np.prod(shape)))
    lib().orc_pz(*shape, _p(np.asarray(w, np.float64)), _p(out))
    return _cube(out, shape)


def zsolve(T, mu, w=(1.0, 1.0, 1.0)):
    """Z = ifftn(fftn(T) / (mu (1 + P_z))) (eq. Z_solution)."""
    T = np.asarray(T, dtype=np.float64)
    Z = np.empty(T.size)
    lib().orc_zsolve(_p(_flat(T)), *T.shape, _p(np.asarray(w, np.float64)), float(mu), _p(Z))
    return _cube(Z, T.shape)


def soft(x, d):
    """R_d(x) = sign(x) max(|x| - d, 0) (Section III-C, step 3)."""
    f = lib().orc_soft
    return np.vectorize(lambda t: f(float(t), float(d)))(np.asarray(x, np.float64))


def group_soft(x, d):
    """The prox of d ||.||_2 applied to each row of x (the isotropic
    F-update's group threshold, eq. CRSSTV_iso)."""
    x = np.array(x, dtype=np.float64, ndmin=2)
    out = np.empty_like(x)
    for k in range(x.shape[0]):
        row = np.ascontiguousarray(x[k])
        lib().orc_group_soft(_p(row), row.size, float(d))
        out[k] = row
    return out


def svt_matrix(A, t):
    """SVT_t of one complex matrix by one-sided Jacobi (eq. E_solution).
    Returns (result, sweeps)."""
    A = np.asarray(A, dtype=np.complex128)
    m, n = A.shape
    v = np.ascontiguousarray(A.reshape(-1, order="F")).view(np.float64).copy()
    sw = lib().orc_svt_matrix(_p(v), m, n, float(t))
    return v.view(np.complex128).reshape((m, n), order="F"), sw


def singular_values(A):
    A = np.asarray(A, dtype=np.complex128)
    m, n = A.shape
    v = np.ascontiguousarray(A.reshape(-1, order="F")).view(np.float64).copy()
    s = np.empty(min(m, n))
    lib().orc_singular_values(_p(v), m, n, _p(s))
    return s


def tsvt(A, t):
    """t-SVT of a real cube with threshold t on each Fourier frontal slice
    (eq. E_solution, Theorem 4.2).  Returns (result, sweeps)."""
    A = np.asarray(A, dtype=np.float64)
    out = np.empty(A.size)
    sw = lib().orc_tsvt(_p(_flat(A)), *A.shape, float(t), _p(out))
    return _cube(out, A.shape), sw


class State:
    """ADMM state of Algorithm 1 (plain LRSTV) in one FP64 buffer:
    Y, L, Z, S, Gamma1, Gamma2, F_1..3, E_1..3, Gamma3_1..3, Gamma4_1..3."""

    def __init__(self, Y, params: Params, flags: int = 0):
        Y = np.asarray(Y, dtype=np.float64)
        self.shape = Y.shape
        self.N = Y.size
        self.p = params.vector()
        self.flags = int(flags)
        self.mu = float(params.mu0)
        self.buf = np.zeros(NSTATE * self.N)
        lib().orc_init(_p(_flat(Y)), *self.shape, _p(self.buf))
        self.iters = 0

    # -- access -------------------------------------------------------------
    def get(self, name, n=None):
        b = BLOCKS[name] + (n or 0)
        return _cube(self.buf[b * self.N:(b + 1) * self.N].copy(), self.shape)

    def set(self, name, value, n=None):
        b = BLOCKS[name] + (n or 0)
        self.buf[b * self.N:(b + 1) * self.N] = _flat(value)

    def block(self, b):
        return _cube(self.buf[b * self.N:(b + 1) * self.N].copy(), self.shape)

    def copy(self):
        c = object.__new__(State)
        c.__dict__.update(self.__dict__)
        c.buf = self.buf.copy()
        c.p = self.p.copy()
        return c

    # -- steps of Algorithm 1 ----------------------------------------------
    def step_l(self):
        lib().orc_step_l(_p(self.buf), *self.shape, _p(self.p), self.mu)

    def step_z(self):
        lib().orc_step_z(_p(self.buf), *self.shape, _p(self.p), self.mu)

    def step_f(self):
        lib().orc_step_f(_p(self.buf), *self.shape, _p(self.p), self.mu, self.flags)

    def step_e(self):
        return lib().orc_step_e(_p(self.buf), *self.shape, _p(self.p), self.mu)

    def step_s(self):
        lib().orc_step_s(_p(self.buf), *self.shape, _p(self.p), self.mu)

    def step_dual(self):
        lib().orc_step_dual(_p(self.buf), *self.shape, _p(self.p), self.mu, self.flags)

    def step_mu(self):
        self.mu = lib().orc_step_mu(_p(self.p), self.mu)

    def residual(self):
        r = np.zeros(2)
        lib().orc_residual(_p(self.buf), *self.shape, _p(r))
        return r

    def step_theta(self, tau, alpha, lam, mu):
        """One iteration of Algorithm 1 with explicit scalars (tau, alpha,
        lambda, mu) for this iteration and no penalty update: the iteration
        of an unrolled solver whose per-iteration scalars are free."""
        self.p[0], self.p[1], self.p[2] = float(tau), float(alpha), float(lam)
        self.mu = float(mu)
        self.step_l()
        self.step_z()
        self.step_f()
        sw = self.step_e()
        self.step_s()
        self.step_dual()
        self.iters += 1
        return sw

    def iterate(self, iters):
        """Runs `iters` iterations; returns (residuals (iters, 2), sweeps)."""
        res = np.zeros(2 * max(iters, 1))
        mu = ctypes.c_double(self.mu)
        sw = lib().orc_iterate(_p(self.buf), *self.shape, _p(self.p), ctypes.byref(mu),
                               int(iters), self.flags, _p(res))
        self.mu = mu.value
        self.iters += iters
        return res[:2 * iters].reshape(iters, 2), sw

    @property
    def X(self):
        """The denoised cube, X := L (Algorithm 1, Ensure)."""
        return self.get("L")


def mpsnr(x, clean):
    """Mean over bands of 10 log10(1 / MSE_band), data on [0, 1] (Section IV-A)."""
    x = np.asarray(x, np.float64)
    clean = np.asarray(clean, np.float64)
    mse = ((x - clean) ** 2).reshape(-1, x.shape[-1], order="F").mean(axis=0)
    return float(np.mean(10.0 * np.log10(1.0 / np.maximum(mse, 1e-300))))
