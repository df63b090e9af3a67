"""Differentiable Drell-Yan cross section: ``torch.autograd.Function`` over the
library's adjoint kernel.

Forward: one stage of ``itmx`` VEGAS iterations on the context's current grid,
held fixed (typically adapted first by warm-up stages, as in the two-stage
runs of Section 3.2), giving sigma(theta) for theta = (M_Z, Gamma_Z,
sin^2 theta_W, a, b).  Backward: the same iterations again, from the same
iteration counter -- so over exactly the same events -- through the
hand-written reverse sweep of the event weight (``vegas_adjoint``); the weights
are recomputed, not stored.  The gradient is that of the frozen-grid
estimator with the inverse-variance combination weights held fixed.
"""
from __future__ import annotations

import numpy as np
import torch

from . import vegas as v
from .workloads import DY_GRAD_INDEX, DY_PARAMS


def _params_with(theta: np.ndarray, base) -> np.ndarray:
    p = np.array(base, dtype=np.float64)
    for k, idx in enumerate(DY_GRAD_INDEX):
        p[idx] = theta[k]
    return p


class _DYSigma(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, integ: "DrellYanIntegral"):
        th = theta.detach().to("cpu", torch.float64).numpy()
        params = _params_with(th, integ.base_params)
        state = integ.g.state()
        I, e, _, _, _ = integ.g.iterate(integ.ncall, integ.itmx, v.VEGAS_DY, params)
        ctx.integ = integ
        ctx.state = state
        ctx.params = params
        ctx.after = integ.g.state()
        integ.last_error = e
        return theta.new_tensor(I)

    @staticmethod
    def backward(ctx, grad_out):
        integ = ctx.integ
        now = integ.g.state()
        integ.g.restore(ctx.state)  # same iteration counter: same events
        grad, grad_err, _, _, _ = integ.g.adjoint(integ.ncall, integ.itmx, ctx.params)
        integ.g.restore(now)
        integ.last_grad_err = grad_err
        g = torch.as_tensor(grad, dtype=grad_out.dtype, device=grad_out.device)
        return grad_out * g, None


class DrellYanIntegral:
    """sigma(theta) of the LO Drell-Yan integrand as a differentiable function.

    ``warmup(ncall, itmx)`` adapts the grid; afterwards the grid is frozen and
    every call ``integ(theta)`` integrates with it."""

    def __init__(self, ndim: int = 4, nbins: int = 100, seed: int = 1234, *, ncall: int = 100_000,
                 itmx: int = 5, precision: str = "fp64", base_params=DY_PARAMS):
        self.g = v.Vegas(ndim, nbins, seed, precision=precision)
        self.ncall, self.itmx = ncall, itmx
        self.base_params = tuple(base_params)
        self.last_error = None
        self.last_grad_err = None

    def warmup(self, ncall: int, itmx: int, theta=None):
        p = self.base_params if theta is None else _params_with(np.asarray(theta, float),
                                                               self.base_params)
        self.g.set(v.VEGAS_OPT_ADAPT, 1)
        out = self.g.iterate(ncall, itmx, v.VEGAS_DY, p)
        self.g.set(v.VEGAS_OPT_ADAPT, 0)
        return out

    def __call__(self, theta: torch.Tensor) -> torch.Tensor:
        self.g.set(v.VEGAS_OPT_ADAPT, 0)
        return _DYSigma.apply(theta, self)

    def close(self):
        self.g.close()
