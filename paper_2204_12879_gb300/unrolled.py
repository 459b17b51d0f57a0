"""Differentiable unrolled plain-LRSTV (torch.autograd front end of lrstv_unroll).

K iterations of Algorithm 1 (Section III-C) on a batch of cubes, with the
scalars of every iteration -- tau (gradient sparsity), alpha (gradient tensor
nuclear norm), lambda (sparse noise) and the penalty mu -- as learnable
parameters.  Forward and backward both run in liblrstv's kernels
(``lrstv_unroll_forward`` / ``lrstv_unroll_backward``); this module only
marshals tensors.  The module keeps the scalars as logarithms so that every
optimiser step leaves them positive, as the iteration requires.
"""
from __future__ import annotations

import math

import torch

from . import lrstv as _lr

__all__ = ["UnrolledLRSTVFunction", "UnrolledLRSTV", "default_theta"]


def default_theta(n1, n2, iters, tau=1e-3, alpha=0.2, lam=None, C=1.0, mu0=1e-2, rho=1.5,
                  mu_max=1e6):
    """The plain solver's scalars as a K x 4 list: fixed tau, alpha, lambda =
    C / sqrt(n1 n2) (Section IV-D) and the geometric penalty schedule
    mu_k = min(rho^k mu0, mu_max)."""
    lam = C / math.sqrt(n1 * n2) if lam is None else lam
    out, mu = [], float(mu0)
    for _ in range(iters):
        out.append([float(tau), float(alpha), float(lam), mu])
        mu = min(float(rho) * mu, float(mu_max))
    return out


class UnrolledLRSTVFunction(torch.autograd.Function):
    """X = unrolled LRSTV(Y, theta) through an lrstv_unroll handle.

    Y: (B, n3, n2, n1) float32 CUDA tensor; theta: (K, 4) float64 tensor on
    any device.  The handle keeps the iterates of its last forward pass, so a
    backward pass must come before the same handle's next forward pass."""

    @staticmethod
    def forward(ctx, Y, theta, handle):
        th = theta.detach().to("cpu", torch.float64).numpy()
        X = handle.forward(Y.contiguous(), th)
        ctx.handle = handle
        ctx.theta_meta = (theta.device, theta.dtype)
        return X

    @staticmethod
    def backward(ctx, gX):
        dth, dY = ctx.handle.backward(gX.contiguous(), want_dY=ctx.needs_input_grad[0])
        dev, dt = ctx.theta_meta
        return dY, dth.to(dev, dt), None


class UnrolledLRSTV(torch.nn.Module):
    """K unrolled iterations with 4 K learnable scalars (log tau, log alpha,
    log lambda, log mu per iteration), initialised to the plain solver's
    schedule (default_theta).  forward(Y) -> X for a (B, n3, n2, n1) float32
    CUDA batch of the shape given here."""

    def __init__(self, n1, n2, n3, batch, iters=10, w=(1.0, 1.0, 1.0), flags=0, **theta_kw):
        super().__init__()
        self.shape = (int(n1), int(n2), int(n3))
        self.batch, self.iters = int(batch), int(iters)
        th = torch.tensor(default_theta(n1, n2, iters, **theta_kw), dtype=torch.float64)
        self.log_theta = torch.nn.Parameter(th.log())
        self.handle = _lr.Unroll(self.shape, batch, iters, w=w, flags=flags)

    def theta(self):
        return self.log_theta.exp()

    def forward(self, Y):
        return UnrolledLRSTVFunction.apply(Y, self.theta(), self.handle)
