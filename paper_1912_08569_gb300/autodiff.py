"""The swap-potential energy as a differentiable torch function (GPU path).

``energy(model, x, theta)`` returns U(x; theta) for positions x [n, 3]
(float64, CUDA, user order) and theta = (lambda, eps, sigma) of the reactive
type pair.  Its backward gives dU/dx = -F and dU/dtheta from the library's
kernels, which one call (swp_eval_grad) enqueues together with the energy:
theta, x and every result stay in device memory and nothing waits for the
device, so a fit over many snapshots runs at the pace of its kernels.  Errors
the device latches (a list row longer than the list buffer allows, a
non-finite force) surface at the next ``SwapModel.check()`` or any other
synchronising call of the system.  The force returned by that
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
    from a tensor at every evaluation; the other coefficients stay as given.
    Evaluations replace the system's state (zero velocities, unit masses)."""

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

    def evaluate(self, x, theta, want_grad=True):
        """(U [], F [n, 3], dU/dtheta [3], dF/dtheta [3, n, 3]) at x, theta as
        float64 device tensors, enqueued on the system's stream (no sync)."""
        t = self.torch
        dev = self.s.device
        n = self.s.n
        th = theta.detach().to(device=dev, dtype=t.float64).contiguous()
        xd = x.detach().to(device=dev, dtype=t.float64).contiguous()
        U = t.empty((), dtype=t.float64, device=dev)
        F = t.empty((n, 3), dtype=t.float64, device=dev)
        dU = t.empty(3, dtype=t.float64, device=dev) if want_grad else None
        dF = t.empty((3, n, 3), dtype=t.float64, device=dev) if want_grad else None
        A.swp_eval_grad(self.s.ctx, self.react[0], self.react[1], th, xd, self.types, U, F, dU, dF)
        return U, F, dU, dF

    def evaluate_batch(self, X, theta):
        """The same for snapshots X [S, n, 3] (one list of types): U [S],
        F [S, n, 3], dU/dtheta [S, 3], dF/dtheta [S, 3, n, 3], one evaluation
        per snapshot enqueued into the slices of the outputs (no sync)."""
        t = self.torch
        dev = self.s.device
        S, n = X.shape[0], self.s.n
        th = theta.detach().to(device=dev, dtype=t.float64).contiguous()
        Xd = X.detach().to(device=dev, dtype=t.float64).contiguous()
        U = t.empty(S, dtype=t.float64, device=dev)
        F = t.empty((S, n, 3), dtype=t.float64, device=dev)
        dU = t.empty((S, 3), dtype=t.float64, device=dev)
        dF = t.empty((S, 3, n, 3), dtype=t.float64, device=dev)
        ctx, ti, tj, ty = self.s.ctx, self.react[0], self.react[1], self.types
        for k in range(S):
            A.swp_eval_grad(ctx, ti, tj, th, Xd[k], ty, U[k], F[k], dU[k], dF[k])
        return U, F, dU, dF

    def check(self):
        """Waits for the evaluations so far and raises if the device latched an error."""
        A.swp_sync(self.s.ctx)


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
            return U

        @staticmethod
        def backward(ctx, gU):
            x, theta, F, dU, dF = ctx.saved_tensors
            gx = _Forces.apply(x, theta, F, dF) * (-gU)
            return gx, gU * dU, None

    # snapshots in one Function: X [S, n, 3], U [S], dF [S, 3, n, 3]
    class _ForcesBatch(torch.autograd.Function):
        @staticmethod
        def forward(ctx, X, theta, F, dF):
            ctx.save_for_backward(dF)
            return F.clone()

        @staticmethod
        def backward(ctx, gF):
            (dF,) = ctx.saved_tensors
            gtheta = torch.einsum("sknc,snc->k", dF, gF)
            return None, gtheta, None, None

    class _EnergyBatch(torch.autograd.Function):
        @staticmethod
        def forward(ctx, X, theta, model):
            U, F, dU, dF = model.evaluate_batch(X, theta)
            ctx.save_for_backward(X, theta, F, dU, dF)
            return U

        @staticmethod
        def backward(ctx, gU):
            X, theta, F, dU, dF = ctx.saved_tensors
            gX = _ForcesBatch.apply(X, theta, F, dF) * (-gU)[:, None, None]
            return gX, (gU[:, None] * dU).sum(0), None

    return _Energy, _Forces, _EnergyBatch, _ForcesBatch


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


def energy_batch(model: SwapModel, X, theta):
    """U(X_s; theta) for snapshots X [S, n, 3] (the model's types) as a float64
    tensor [S], differentiable in X and theta like ``energy``: one autograd
    node for the whole batch, so a fit over many snapshots pays the Python
    cost of autograd once, not per snapshot."""
    return _fn()[2].apply(X, theta, model)
