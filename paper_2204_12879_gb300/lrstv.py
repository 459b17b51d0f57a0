"""Thin ctypes binding of liblrstv.so (include/lrstv.h).

Argument marshalling only: every step of the denoiser runs in the library's
CUDA kernels.  torch supplies device memory and streams.  There is no CPU
fallback: without the compiled library (or without a CUDA device) every call
raises.

Cubes are torch float32 CUDA tensors of N = n1*n2*n3 elements in the order
i + n1*(j + n2*k) (mode 1 fastest).  A tensor of shape (n3, n2, n1) in the
default C order has exactly that layout; flat tensors work too.
"""
from __future__ import annotations

import ctypes
import os

from . import builder as _build

__all__ = [
    "Params", "Stats", "Profile", "Plan", "Batch", "Unroll", "load", "status_string", "kernel_name", "LrstvError",
    "lrstv_diff", "lrstv_diff_adjoint", "lrstv_soft_threshold", "lrstv_zsolve", "lrstv_tsvt",
    "lrstv_tsvt_noalloc", "lrstv_peak_probe", "PEAK_UNITS",
    "lrstv_denoise", "BLOCK", "FLAG_F_THRESH_EXACT", "FLAG_NO_GAMMA4", "FLAG_GRAPH",
    "FLAG_STRICT", "FLAG_SIMT_GEMM", "FLAG_WARM_START", "FLAG_ISO_TV", "FLAG_BF16X3",
    "FLAG_SIMT_DFT", "FLAG_JACOBI_PER_SLICE", "FLAG_JACOBI_PANEL16", "FLAG_UNROLL_RECOMPUTE",
    "FLAG_JACOBI_FIXED_ORDER",
    "EXPORTED",
]

FLAG_F_THRESH_EXACT = 1
FLAG_NO_GAMMA4 = 2
FLAG_GRAPH = 4
FLAG_STRICT = 8
FLAG_SIMT_GEMM = 16
FLAG_WARM_START = 32
FLAG_ISO_TV = 64
FLAG_BF16X3 = 128
FLAG_SIMT_DFT = 256
FLAG_JACOBI_PER_SLICE = 512
FLAG_JACOBI_PANEL16 = 1024
FLAG_UNROLL_RECOMPUTE = 2048
FLAG_JACOBI_FIXED_ORDER = 4096

BLOCK = {"Y": 0, "L": 1, "Z": 2, "S": 3, "G1": 4, "G2": 5, "F": 6, "E": 7, "G3": 8, "G4": 9,
         "TZ": 10}
_TRIPLE = {"F", "E", "G3", "G4"}


class LrstvError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__(f"{fn}: {status_string(code)} (status {code})")
        self.code = code


class Params(ctypes.Structure):
    """lrstv_params: tau, alpha, lambda, w[3], mu0, rho, mu_max, eps, max_iter, flags."""
    _fields_ = [("tau", ctypes.c_float), ("alpha", ctypes.c_float), ("lam", ctypes.c_float),
                ("w", ctypes.c_float * 3), ("mu0", ctypes.c_float), ("rho", ctypes.c_float),
                ("mu_max", ctypes.c_float), ("eps", ctypes.c_float), ("max_iter", ctypes.c_int),
                ("flags", ctypes.c_uint)]

    @classmethod
    def make(cls, n1, n2, tau=0.001, alpha=0.2, lam=None, C=1.0, w=(1.0, 1.0, 1.0), mu0=1e-2,
             rho=1.5, mu_max=1e6, eps=1e-6, max_iter=20, flags=0):
        """Defaults of this library: lambda = C / sqrt(n1 n2) (Section IV-D)."""
        if lam is None:
            lam = C / (float(n1 * n2) ** 0.5)
        p = cls()
        p.tau, p.alpha, p.lam = tau, alpha, lam
        p.w[0], p.w[1], p.w[2] = w
        p.mu0, p.rho, p.mu_max, p.eps = mu0, rho, mu_max, eps
        p.max_iter, p.flags = int(max_iter), int(flags)
        return p


class Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("res_inf", ctypes.c_float * 2), ("mu", ctypes.c_float),
                ("jacobi_unconverged", ctypes.c_int), ("jacobi_max_sweeps", ctypes.c_int),
                ("gemm_errors", ctypes.c_int)]

    def as_dict(self):
        return {"iters": self.iters, "res_inf": [self.res_inf[0], self.res_inf[1]], "mu": self.mu,
                "jacobi_unconverged": self.jacobi_unconverged,
                "jacobi_max_sweeps": self.jacobi_max_sweeps, "gemm_errors": self.gemm_errors}


class Profile(ctypes.Structure):
    """lrstv_profile: per-kernel launches and summed CUDA-event milliseconds,
    and the Jacobi work counters."""
    _fields_ = [("launches", ctypes.c_int * 16), ("ms", ctypes.c_double * 16),
                ("jacobi_pairs", ctypes.c_ulonglong), ("jacobi_rotations", ctypes.c_ulonglong)]

    def as_dict(self):
        out = {}
        for k in range(16):
            if self.launches[k]:
                out[kernel_name(k)] = {"launches": self.launches[k], "ms": self.ms[k]}
        return out


_P = ctypes.c_void_p
_I = ctypes.c_int
_F = ctypes.c_float
_SZ = ctypes.c_size_t
# name -> argtypes (every entry point returns int status unless listed in _RESTYPE)
_SIGS = {
    "lrstv_status_string": [_I],
    "lrstv_max_spatial": [],
    "lrstv_check_bounded_wait": [ctypes.c_longlong, _I, ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "lrstv_peak_probe": [_I, ctypes.c_longlong, ctypes.POINTER(ctypes.c_double),
                         ctypes.POINTER(ctypes.c_double)],
    "lrstv_plan_create": [_I, _I, _I, ctypes.POINTER(Params), ctypes.POINTER(_P)],
    "lrstv_plan_destroy": [_P],
    "lrstv_plan_bytes": [_P, ctypes.POINTER(_SZ)],
    "lrstv_plan_set_params": [_P, ctypes.POINTER(Params)],
    "lrstv_init": [_P, _P, _P],
    "lrstv_step_l_tz": [_P, _P],
    "lrstv_step_z": [_P, _P],
    "lrstv_step_fs_dual": [_P, _P],
    "lrstv_step_e": [_P, _P],
    "lrstv_step_mu": [_P],
    "lrstv_iterate": [_P, _I, _P],
    "lrstv_get_stats": [_P, ctypes.POINTER(Stats), _P],
    "lrstv_get_slice_sweeps": [_P, ctypes.POINTER(_I), _I, _P],
    "lrstv_plan_set_tucker": [_P, ctypes.POINTER(_I)],
    "lrstv_plan_tucker_factor": [_P, _I, _P, _P],
    "lrstv_state_get": [_P, _I, _P, _P],
    "lrstv_state_set": [_P, _I, _P, _P],
    "lrstv_get_mu": [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I)],
    "lrstv_set_mu": [_P, ctypes.c_double, _I],
    "lrstv_plan_run": [_P, _P, _P, _P, ctypes.POINTER(Stats), _P],
    "lrstv_plan_run_host": [_P, _P, _P, _P, ctypes.POINTER(Stats), _P],
    "lrstv_plan_autotune": [_P, _P, _I, ctypes.c_uint, ctypes.POINTER(ctypes.c_uint),
                            ctypes.POINTER(_F), _P],
    "lrstv_denoise": [_P, _I, _I, _I, ctypes.POINTER(Params), _P, _P, ctypes.POINTER(Stats), _P],
    "lrstv_diff": [_P, _I, _I, _I, ctypes.POINTER(_F), _P, _P],
    "lrstv_diff_adjoint": [_P, _I, _I, _I, ctypes.POINTER(_F), _P, _P],
    "lrstv_soft_threshold": [_P, _SZ, _F, _P, _P],
    "lrstv_zsolve_workspace_size": [_I, _I, _I, ctypes.POINTER(_SZ)],
    "lrstv_tsvt_workspace_size": [_I, _I, _I, ctypes.POINTER(_SZ)],
    "lrstv_zsolve": [_P, _I, _I, _I, ctypes.POINTER(_F), _F, _P, _P, _SZ, _P],
    "lrstv_tsvt": [_P, _I, _I, _I, _F, _P, _P, _SZ, ctypes.POINTER(_I), _P],
    "lrstv_tsvt_noalloc": [_P, _I, _I, _I, _F, _P, ctypes.POINTER(_I), _P],
    "lrstv_batch_create": [_I, ctypes.POINTER(_I), ctypes.POINTER(Params), ctypes.POINTER(_P)],
    "lrstv_batch_destroy": [_P],
    "lrstv_batch_size": [_P, ctypes.POINTER(_I)],
    "lrstv_batch_groups": [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "lrstv_batch_plan": [_P, _I, ctypes.POINTER(_P)],
    "lrstv_batch_init": [_P, ctypes.POINTER(_P), _P],
    "lrstv_batch_iterate": [_P, _I, _P],
    "lrstv_batch_run": [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P), _P],
    "lrstv_unroll_create": [_I, _I, _I, _I, _I, ctypes.POINTER(_F), ctypes.c_uint,
                            ctypes.POINTER(_P)],
    "lrstv_unroll_destroy": [_P],
    "lrstv_unroll_bytes": [_P, ctypes.POINTER(_SZ)],
    "lrstv_unroll_forward": [_P, _P, ctypes.POINTER(ctypes.c_double), _P, _P],
    "lrstv_unroll_backward": [_P, _P, _P, _P, _P],
    "lrstv_unroll_stats": [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), _P],
    "lrstv_kernel_name": [_I],
    "lrstv_profile_enable": [_P, _I],
    "lrstv_profile_read": [_P, ctypes.POINTER(Profile)],
}
_RESTYPE = {"lrstv_status_string": ctypes.c_char_p, "lrstv_kernel_name": ctypes.c_char_p}
EXPORTED = sorted(_SIGS)

_lib = None


def load(build_if_missing: bool = True):
    """Loads liblrstv.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError("liblrstv.so is not built; run paper_2204_12879_gb300.build()")
        L = ctypes.CDLL(path)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = _RESTYPE.get(name, ctypes.c_int)
        _lib = L
    return _lib


def status_string(code: int) -> str:
    return load().lrstv_status_string(int(code)).decode()


def kernel_name(k: int) -> str:
    return load().lrstv_kernel_name(int(k)).decode()


def _call(name, *args):
    rc = getattr(load(), name)(*args)
    if rc != 0:
        raise LrstvError(name, rc)
    return rc


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("liblrstv needs a CUDA device; there is no CPU path")
    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, n=None):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 \
            or not t.is_contiguous():
        raise TypeError("expected a contiguous float32 CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"expected {n} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _w(w):
    return (ctypes.c_float * 3)(*[float(x) for x in w])


def _empty(n, device=None):
    torch = _torch()
    return torch.empty(int(n), dtype=torch.float32, device=device or "cuda")


class Plan:
    """An lrstv_plan: device state of one n1 x n2 x n3 ADMM run."""

    def __init__(self, n1, n2, n3, params: Params):
        _torch()
        self.shape = (int(n1), int(n2), int(n3))
        self.N = n1 * n2 * n3
        self.params = params
        h = ctypes.c_void_p()
        _call("lrstv_plan_create", int(n1), int(n2), int(n3), ctypes.byref(params), ctypes.byref(h))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().lrstv_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def nbytes(self):
        b = ctypes.c_size_t()
        _call("lrstv_plan_bytes", self._h, ctypes.byref(b))
        return b.value

    def set_params(self, params: Params):
        _call("lrstv_plan_set_params", self._h, ctypes.byref(params))
        self.params = params

    def init(self, Y, stream=None):
        _call("lrstv_init", self._h, _dev(Y, self.N), _stream(stream))

    def step_l_tz(self, stream=None):
        _call("lrstv_step_l_tz", self._h, _stream(stream))

    def step_z(self, stream=None):
        _call("lrstv_step_z", self._h, _stream(stream))

    def step_fs_dual(self, stream=None):
        _call("lrstv_step_fs_dual", self._h, _stream(stream))

    def step_e(self, stream=None):
        _call("lrstv_step_e", self._h, _stream(stream))

    def step_mu(self):
        _call("lrstv_step_mu", self._h)

    def iterate(self, iters, stream=None):
        _call("lrstv_iterate", self._h, int(iters), _stream(stream))

    def stats(self, stream=None) -> Stats:
        s = Stats()
        _call("lrstv_get_stats", self._h, ctypes.byref(s), _stream(stream))
        return s

    def set_tucker(self, ranks):
        """Full TDLRSTV: Tucker (HOOI) L-update with multilinear ranks
        (r1, r2, r3); None or (0, 0, 0) restores the plain L-update."""
        arr = None if ranks is None else (_I * 3)(*[int(r) for r in ranks])
        _call("lrstv_plan_set_tucker", self._h, arr)

    def tucker_factor(self, mode, rank, stream=None):
        """U_{mode+1} of the last Tucker L-update as an (n, rank) float32 CUDA
        tensor (orthonormal columns)."""
        torch = _torch()
        n = self.shape[mode]
        out = torch.empty(rank * n, dtype=torch.float32, device="cuda")
        _call("lrstv_plan_tucker_factor", self._h, int(mode), ctypes.c_void_p(out.data_ptr()),
              _stream(stream))
        return out.view(rank, n).t()

    def slice_sweeps(self, stream=None):
        """Per-slice Jacobi sweep counts of the last E-step, shape (3, n3//2 + 1)."""
        import numpy as np
        h = self.shape[2] // 2 + 1
        out = np.zeros(3 * h, dtype=np.int32)
        _call("lrstv_get_slice_sweeps", self._h, out.ctypes.data_as(ctypes.POINTER(_I)), 3 * h,
              _stream(stream))
        return out.reshape(3, h)

    def get(self, name, stream=None):
        n = 3 * self.N if name in _TRIPLE else self.N
        out = _empty(n)
        _call("lrstv_state_get", self._h, BLOCK[name], _dev(out), _stream(stream))
        return out

    def set(self, name, value, stream=None):
        n = 3 * self.N if name in _TRIPLE else self.N
        _call("lrstv_state_set", self._h, BLOCK[name], _dev(value, n), _stream(stream))

    @property
    def mu(self):
        m, it = ctypes.c_double(), ctypes.c_int()
        _call("lrstv_get_mu", self._h, ctypes.byref(m), ctypes.byref(it))
        return m.value, it.value

    def set_mu(self, mu, iters):
        _call("lrstv_set_mu", self._h, float(mu), int(iters))

    def profile_enable(self, on=True):
        _call("lrstv_profile_enable", self._h, 1 if on else 0)

    def profile_read(self) -> Profile:
        p = Profile()
        _call("lrstv_profile_read", self._h, ctypes.byref(p))
        return p

    def run(self, Y, X=None, S=None, stats=False, stream=None):
        """lrstv_plan_run on device tensors; returns (X, S[, Stats])."""
        X = _empty(self.N) if X is None else X
        S = _empty(self.N) if S is None else S
        st = Stats()
        _call("lrstv_plan_run", self._h, _dev(Y, self.N), _dev(X, self.N), _dev(S, self.N),
              ctypes.byref(st) if stats else None, _stream(stream))
        return (X, S, st) if stats else (X, S)

    def autotune(self, Y, iters=0, allowed=None, stream=None):
        """lrstv_plan_autotune: keeps the fastest combination of the allowed
        flags (default: SIMT_GEMM, SIMT_DFT, JACOBI_PER_SLICE, JACOBI_PANEL16
        and WARM_START;
        FLAG_BF16X3 may be added, which trades the FP32 bound for the 3xBF16
        one) for this plan and cube.
        Returns (flags kept, their time in ms); leaves the plan initialised
        from Y."""
        if allowed is None:
            allowed = (FLAG_SIMT_GEMM | FLAG_SIMT_DFT | FLAG_JACOBI_PER_SLICE |
                       FLAG_JACOBI_PANEL16 | FLAG_WARM_START)
        chosen = ctypes.c_uint()
        ms = _F()
        _call("lrstv_plan_autotune", self._h, _dev(Y, self.N), int(iters), int(allowed),
              ctypes.byref(chosen), ctypes.byref(ms), _stream(stream))
        return int(chosen.value), float(ms.value)

    def run_host(self, Y, X, S, stats=False, stream=None):
        """lrstv_plan_run_host on host float32 buffers (numpy arrays or pinned
        CPU tensors, N contiguous elements each); synchronises."""
        st = Stats()
        _call("lrstv_plan_run_host", self._h, _host_ptr(Y, self.N), _host_ptr(X, self.N),
              _host_ptr(S, self.N), ctypes.byref(st) if stats else None, _stream(stream))
        return st


class _BorrowedPlan(Plan):
    """A plan owned by a batch: usable for stats and state export, never freed here."""

    def __init__(self, handle, shape, params):
        self.shape = tuple(shape)
        self.N = shape[0] * shape[1] * shape[2]
        self.params = params
        self._borrowed = handle

    @property
    def _h(self):
        return self._borrowed

    def close(self):
        pass


class Batch:
    """An lrstv_batch: independent cubes of uneven shapes run in lockstep,
    one launch per kernel and group of equal shapes and parameters, with one
    persistent Jacobi launch per E-step."""

    def __init__(self, shapes, params):
        _torch()
        self.shapes = [tuple(int(x) for x in sh) for sh in shapes]
        n = len(self.shapes)
        if isinstance(params, Params):
            params = [params] * n
        self.params = list(params)
        dims = (ctypes.c_int * (3 * n))(*[x for sh in self.shapes for x in sh])
        parr = (Params * n)(*self.params)
        h = ctypes.c_void_p()
        _call("lrstv_batch_create", n, dims, parr, ctypes.byref(h))
        self._h = h
        self.n = n

    def close(self):
        if getattr(self, "_h", None):
            load().lrstv_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def groups(self):
        """(number of groups, list of each cube's group)."""
        ng = ctypes.c_int()
        gof = (ctypes.c_int * self.n)()
        _call("lrstv_batch_groups", self._h, ctypes.byref(ng), gof)
        return ng.value, list(gof)

    def plan(self, i) -> Plan:
        h = ctypes.c_void_p()
        _call("lrstv_batch_plan", self._h, int(i), ctypes.byref(h))
        return _BorrowedPlan(h, self.shapes[i], self.params[i])

    @staticmethod
    def _ptrs(ts, shapes):
        arr = (ctypes.c_void_p * len(ts))()
        for i, (t, sh) in enumerate(zip(ts, shapes)):
            arr[i] = _dev(t, sh[0] * sh[1] * sh[2]).value
        return arr

    def init(self, Ys, stream=None):
        _call("lrstv_batch_init", self._h, self._ptrs(Ys, self.shapes), _stream(stream))

    def iterate(self, iters, stream=None):
        _call("lrstv_batch_iterate", self._h, int(iters), _stream(stream))

    def run(self, Ys, Xs=None, Ss=None, stream=None):
        """lrstv_batch_run; returns (Xs, Ss) lists of device tensors."""
        Xs = [_empty(sh[0] * sh[1] * sh[2]) for sh in self.shapes] if Xs is None else Xs
        Ss = [_empty(sh[0] * sh[1] * sh[2]) for sh in self.shapes] if Ss is None else Ss
        _call("lrstv_batch_run", self._h, self._ptrs(Ys, self.shapes),
              self._ptrs(Xs, self.shapes), self._ptrs(Ss, self.shapes), _stream(stream))
        return Xs, Ss


class Unroll:
    """An lrstv_unroll: K iterations of Algorithm 1 with per-iteration scalars
    theta_k = (tau, alpha, lambda, mu) on B cubes of one shape, and the
    gradient of a loss on the final L with respect to theta and Y.

    Y and X are B cubes back to back (a (B, n3, n2, n1) tensor in C order).
    theta is a host (K, 4) float64 array; its gradient comes back as a
    (K, 4) float64 CUDA tensor.  A backward pass uses the iterates of the
    handle's last forward pass."""

    def __init__(self, shape, batch, iters, w=(1.0, 1.0, 1.0), flags=0):
        self.shape = tuple(int(x) for x in shape)
        self.batch, self.iters = int(batch), int(iters)
        self.N = self.shape[0] * self.shape[1] * self.shape[2]
        h = ctypes.c_void_p()
        _call("lrstv_unroll_create", *self.shape, self.batch, self.iters, _w(w),
              int(flags), ctypes.byref(h))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().lrstv_unroll_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def nbytes(self):
        b = ctypes.c_size_t()
        _call("lrstv_unroll_bytes", self._h, ctypes.byref(b))
        return b.value

    def forward(self, Y, theta, X=None, stream=None):
        import numpy as np
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
        if th.shape != (self.iters, 4):
            raise ValueError(f"theta must be ({self.iters}, 4)")
        n = self.batch * self.N
        X = _empty(n, Y.device).view(Y.shape) if X is None else X
        _call("lrstv_unroll_forward", self._h, _dev(Y, n),
              th.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _dev(X, n), _stream(stream))
        return X

    def backward(self, dX, want_dY=True, stream=None):
        """Returns (dtheta (K, 4) float64 CUDA tensor, dY or None)."""
        torch = _torch()
        n = self.batch * self.N
        dth = torch.empty((self.iters, 4), dtype=torch.float64, device=dX.device)
        dY = _empty(n, dX.device).view(dX.shape) if want_dY else None
        _call("lrstv_unroll_backward", self._h, _dev(dX, n), ctypes.c_void_p(dth.data_ptr()),
              _dev(dY, n) if dY is not None else None, _stream(stream))
        return dth, dY

    def stats(self, stream=None):
        """(Fourier slices whose Jacobi hit its sweep cap in the last forward,
        tensor-core GEMM wait timeouts); synchronises."""
        a, b = ctypes.c_int(), ctypes.c_int()
        _call("lrstv_unroll_stats", self._h, ctypes.byref(a), ctypes.byref(b), _stream(stream))
        return a.value, b.value


def _host_ptr(a, n):
    import numpy as np
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.is_cuda or a.dtype != torch.float32 or not a.is_contiguous() or a.numel() != n:
                raise TypeError("expected a contiguous float32 CPU tensor of N elements")
            return ctypes.c_void_p(a.data_ptr())
    except ImportError:
        pass
    if not (isinstance(a, np.ndarray) and a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]
            and a.size == n):
        raise TypeError("expected a contiguous float32 host array of N elements")
    return ctypes.c_void_p(a.ctypes.data)


def lrstv_diff(x, shape, w=(1.0, 1.0, 1.0), out=None, stream=None):
    """w_n D_n x for n = 1..3 (3N floats)."""
    n1, n2, n3 = shape
    out = _empty(3 * x.numel()) if out is None else out
    _call("lrstv_diff", _dev(x, n1 * n2 * n3), n1, n2, n3, _w(w), _dev(out, 3 * x.numel()),
          _stream(stream))
    return out


def lrstv_diff_adjoint(g, shape, w=(1.0, 1.0, 1.0), out=None, stream=None):
    n1, n2, n3 = shape
    N = n1 * n2 * n3
    out = _empty(N) if out is None else out
    _call("lrstv_diff_adjoint", _dev(g, 3 * N), n1, n2, n3, _w(w), _dev(out, N), _stream(stream))
    return out


def lrstv_soft_threshold(x, d, out=None, stream=None):
    out = _empty(x.numel()) if out is None else out
    _call("lrstv_soft_threshold", _dev(x), x.numel(), float(d), _dev(out, x.numel()),
          _stream(stream))
    return out


def _workspace(fn, shape):
    b = ctypes.c_size_t()
    _call(fn, *shape, ctypes.byref(b))
    torch = _torch()
    return torch.empty(max(int(b.value), 1), dtype=torch.uint8, device="cuda"), b.value


def lrstv_zsolve(T, shape, mu, w=(1.0, 1.0, 1.0), out=None, workspace=None, stream=None):
    """Z = ifftn(fftn(T) / (mu (1 + P_z)))."""
    n1, n2, n3 = shape
    N = n1 * n2 * n3
    out = _empty(N) if out is None else out
    ws, nb = workspace if workspace is not None else _workspace("lrstv_zsolve_workspace_size", shape)
    _call("lrstv_zsolve", _dev(T, N), n1, n2, n3, _w(w), float(mu), _dev(out, N),
          ctypes.c_void_p(ws.data_ptr()), nb, _stream(stream))
    return out


def lrstv_tsvt(A, shape, t, out=None, workspace=None, sweeps=False, stream=None):
    """t-SVT with threshold t on each Fourier frontal slice; returns out (and
    the worst Jacobi sweep count when sweeps=True)."""
    n1, n2, n3 = shape
    N = n1 * n2 * n3
    out = _empty(N) if out is None else out
    ws, nb = workspace if workspace is not None else _workspace("lrstv_tsvt_workspace_size", shape)
    sw = ctypes.c_int(0)
    _call("lrstv_tsvt", _dev(A, N), n1, n2, n3, float(t), _dev(out, N),
          ctypes.c_void_p(ws.data_ptr()), nb, ctypes.byref(sw) if sweeps else None, _stream(stream))
    return (out, sw.value) if sweeps else out


def lrstv_tsvt_noalloc(A, shape, t, out, sweeps=False, stream=None):
    """lrstv_tsvt_noalloc: the t-SVT with the library's fixed device scratch
    array instead of a workspace (for callers that cannot allocate).  `out`
    must be given; nothing is allocated."""
    n1, n2, n3 = shape
    N = n1 * n2 * n3
    sw = ctypes.c_int(0)
    _call("lrstv_tsvt_noalloc", _dev(A, N), n1, n2, n3, float(t), _dev(out, N),
          ctypes.byref(sw) if sweeps else None, _stream(stream))
    return (out, sw.value) if sweeps else out


def lrstv_check_bounded_wait(tries, arrive=False):
    """lrstv_check_bounded_wait: returns (timed_out, lanes_freed)."""
    _torch()
    t, n = _I(), _I()
    _call("lrstv_check_bounded_wait", int(tries), 1 if arrive else 0, ctypes.byref(t),
          ctypes.byref(n))
    return t.value, n.value


PEAK_UNITS = {"fp32_fma": 0, "fp32_fma2": 1, "tf32_mma": 2, "bf16_mma": 3}


def lrstv_peak_probe(unit, work):
    """lrstv_peak_probe: one throughput probe on the current device; unit is a
    key of PEAK_UNITS.  Returns (TFLOP/s, ms of the timed launch)."""
    _torch()
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _call("lrstv_peak_probe", PEAK_UNITS[unit], int(work), ctypes.byref(tf), ctypes.byref(ms))
    return tf.value, ms.value


def lrstv_denoise(Y, shape, params: Params, stream=None):
    """One-shot lrstv_denoise: returns (X, S, Stats)."""
    n1, n2, n3 = shape
    N = n1 * n2 * n3
    X, S, st = _empty(N), _empty(N), Stats()
    _call("lrstv_denoise", _dev(Y, N), n1, n2, n3, ctypes.byref(params), _dev(X, N), _dev(S, N),
          ctypes.byref(st), _stream(stream))
    return X, S, st
