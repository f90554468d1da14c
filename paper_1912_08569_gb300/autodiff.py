"""The swap-potential energy as a differentiable torch function (GPU path).

``energy(model, x, theta)`` returns U(x; theta) for positions x [n, 3]
(float64, CUDA, user order) and theta = (lambda, eps, sigma) of the reactive
type pair.  Its backward gives dU/dx = -F and dU/dtheta from the library's
kernels (swp_compute_forces, swp_param_grad).  The force returned by that
backward is itself differentiable with respect to theta (through dF/dtheta
from swp_param_grad), so a loss built from forces obtained by
``torch.autograd.grad(U, x, create_graph=True)`` -- a force-matching fit --
back-propagates to theta ("double backward").  ``forces(model, x, theta)``
returns the same forces directly, differentiable with respect to theta.

Not provided: second derivatives with respect to positions (a force-dependent
loss gives theta its gradient; x receives none through the forces).

The energy and forces follow Eq. 2b, Eq. pot and Eq. 3bp (one reactive type
pair, unshifted form); the derivative formulas are in the header of the
parameter-derivative kernels.
"""
from __future__ import annotations

import numpy as np

from . import _abi as A


class SwapModel:
    """A SwapSystem whose reactive pair (ti, tj) takes (lambda, eps, sigma)
    from a tensor at every evaluation; the other coefficients stay as given."""

    def __init__(self, system, pairs, types, react=(0, 1), mass=None):
        import torch

        self.torch = torch
        self.s = system
        self.pairs = {k: dict(v) for k, v in pairs.items()}
        self.react = tuple(react)
        if self.pairs[self.react].get("kind") != 2:
            raise ValueError("react must name the swap pair")
        dev = system.device
        self.types = torch.as_tensor(np.asarray(types, dtype=np.int32), device=dev)
        self.mass = None if mass is None else torch.as_tensor(np.asarray(mass, dtype=np.float64), device=dev)

    def _set_theta(self, theta):
        lam, eps, sig = [float(v) for v in theta.detach().cpu().tolist()]
        p = self.pairs[self.react]
        ti, tj = self.react
        A.swp_set_pair(self.s.ctx, ti, tj, 2, eps, sig, p.get("n", 6), p.get("rcut", 0.0), lam, 0,
                       p.get("rbond", 0.0) or 0.0)

    def evaluate(self, x, theta, want_grad=True):
        """(U, F [n, 3], dU/dtheta [3], dF/dtheta [3, n, 3]) at x, theta (float64, device)."""
        t = self.torch
        self._set_theta(theta)
        xd = x.detach().to(dtype=t.float64).contiguous()
        self.s.set_state(xd, None, self.types, self.mass)
        self.s.compute_forces()
        th = A.swp_read_thermo(self.s.ctx)
        U = th.U2 + th.U3
        n = self.s.n
        F = t.empty((n, 3), dtype=t.float64, device=x.device)
        A.swp_read_forces(self.s.ctx, F, A.SWP_DEVICE)
        if not want_grad:
            return U, F, None, None
        dF = t.empty((3, n, 3), dtype=t.float64, device=x.device)
        dU = A.swp_param_grad(self.s.ctx, self.react[0], self.react[1], dF)
        return U, F, t.as_tensor(dU, dtype=t.float64, device=x.device), dF


def _functions():
    import torch

    class _Forces(torch.autograd.Function):
        @staticmethod
        def forward(ctx, x, theta, F, dF):
            ctx.save_for_backward(dF)
            return F.clone()

        @staticmethod
        def backward(ctx, gF):
            (dF,) = ctx.saved_tensors
            gtheta = torch.einsum("knc,nc->k", dF, gF)
            return None, gtheta, None, None

    class _Energy(torch.autograd.Function):
        @staticmethod
        def forward(ctx, x, theta, model):
            U, F, dU, dF = model.evaluate(x, theta)
            ctx.save_for_backward(x, theta, F, dU, dF)
            return torch.tensor(U, dtype=torch.float64, device=x.device)

        @staticmethod
        def backward(ctx, gU):
            x, theta, F, dU, dF = ctx.saved_tensors
            gx = -gU * _Forces.apply(x, theta, F, dF)
            return gx, gU * dU, None

    return _Energy, _Forces


_FN = None


def _fn():
    global _FN
    if _FN is None:
        _FN = _functions()
    return _FN


def energy(model: SwapModel, x, theta):
    """U(x; theta) as a 0-dim float64 tensor (differentiable in x and theta)."""
    return _fn()[0].apply(x, theta, model)


def forces(model: SwapModel, x, theta):
    """F(x; theta) [n, 3] float64, differentiable with respect to theta."""
    U, F, dU, dF = model.evaluate(x, theta)
    return _fn()[1].apply(x, theta, F, dF)
