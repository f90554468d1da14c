"""The autograd wiring of ``autodiff.energy`` / ``autodiff.forces`` on CPU.

A fake model returns U, F = -dU/dx, dU/dtheta and dF/dtheta of a toy energy
that torch can differentiate itself; the Functions must then give the same
gradients as plain autograd through the toy formula, including the double
backward of a force-matching loss.  (The GPU kernels behind the real model are
checked against the oracle in test_gpu_autodiff.py.)
"""
import pytest

torch = pytest.importorskip("torch")

from paper_1912_08569_gb300 import autodiff  # noqa: E402


def _toy_u(x, th):
    # U = th0 * sum |x|^2 / 2 + th1 * sum(x) + th2 * sum(x^4) / 4
    return th[0] * (x * x).sum() / 2 + th[1] * x.sum() + th[2] * (x ** 4).sum() / 4


class ToyModel:
    def evaluate(self, x, theta, want_grad=True):
        x = x.detach().to(torch.float64)
        th = theta.detach().to(torch.float64)
        U = _toy_u(x, th)  # a 0-dim tensor, like the real model's device scalar
        F = -(th[0] * x + th[1] + th[2] * x ** 3)
        dU = torch.stack([(x * x).sum() / 2, x.sum(), (x ** 4).sum() / 4])
        dF = torch.stack([-x, -torch.ones_like(x), -(x ** 3)])
        return U, F, dU, dF

    def evaluate_batch(self, X, theta):
        out = [self.evaluate(x, theta) for x in X]
        return tuple(torch.stack([o[k] for o in out]) for k in range(4))


def test_energy_backward_gives_minus_forces_and_dU_dtheta():
    g = torch.Generator().manual_seed(1)
    x0 = torch.randn(50, 3, generator=g, dtype=torch.float64)
    th0 = torch.tensor([1.3, -0.4, 0.7], dtype=torch.float64)
    x = x0.clone().requires_grad_(True)
    th = th0.clone().requires_grad_(True)
    autodiff.energy(ToyModel(), x, th).backward()
    xr = x0.clone().requires_grad_(True)
    tr = th0.clone().requires_grad_(True)
    _toy_u(xr, tr).backward()
    torch.testing.assert_close(x.grad, xr.grad, rtol=1e-13, atol=1e-13)
    torch.testing.assert_close(th.grad, tr.grad, rtol=1e-13, atol=1e-13)


def test_force_matching_double_backward_matches_autograd():
    g = torch.Generator().manual_seed(2)
    snaps = [torch.randn(40, 3, generator=g, dtype=torch.float64) for _ in range(3)]
    th0 = torch.tensor([0.9, 0.2, 0.5], dtype=torch.float64)
    ref = [-(1.0 * x + 0.1 + 0.3 * x ** 3) for x in snaps]  # target forces at another theta
    model = ToyModel()

    th = th0.clone().requires_grad_(True)
    loss = 0.0
    for x, Fr in zip(snaps, ref):
        xr = x.clone().requires_grad_(True)
        (gx,) = torch.autograd.grad(autodiff.energy(model, xr, th), xr, create_graph=True)
        loss = loss + ((-gx - Fr) ** 2).mean()
    loss.backward()

    tr = th0.clone().requires_grad_(True)
    loss2 = 0.0
    for x, Fr in zip(snaps, ref):
        xr = x.clone().requires_grad_(True)
        (gx,) = torch.autograd.grad(_toy_u(xr, tr), xr, create_graph=True)
        loss2 = loss2 + ((-gx - Fr) ** 2).mean()
    loss2.backward()
    assert loss.item() == pytest.approx(loss2.item(), rel=1e-13)
    torch.testing.assert_close(th.grad, tr.grad, rtol=1e-12, atol=1e-14)

    # the same gradient through autodiff.forces
    t3 = th0.clone().requires_grad_(True)
    loss3 = sum(((autodiff.forces(model, x, t3) - Fr) ** 2).mean() for x, Fr in zip(snaps, ref))
    loss3.backward()
    torch.testing.assert_close(t3.grad, tr.grad, rtol=1e-12, atol=1e-14)


def test_energy_batch_matches_per_snapshot_functions():
    """energy_batch (one autograd node for all snapshots) gives the loss and the
    gradient of the per-snapshot form."""
    g = torch.Generator().manual_seed(3)
    X0 = torch.randn(4, 30, 3, generator=g, dtype=torch.float64)
    th0 = torch.tensor([0.9, 0.2, 0.5], dtype=torch.float64)
    R = torch.stack([-(1.0 * x + 0.1 + 0.3 * x ** 3) for x in X0])
    model = ToyModel()
    th = th0.clone().requires_grad_(True)
    X = X0.clone().requires_grad_(True)
    U = autodiff.energy_batch(model, X, th)
    (gX,) = torch.autograd.grad(U.sum(), X, create_graph=True)
    loss = ((gX + R) ** 2).mean()
    loss.backward()
    tr = th0.clone().requires_grad_(True)
    loss2 = 0.0
    for x, r in zip(X0, R):
        xr = x.clone().requires_grad_(True)
        (gx,) = torch.autograd.grad(_toy_u(xr, tr), xr, create_graph=True)
        loss2 = loss2 + ((gx + r) ** 2).mean()
    (loss2 / len(X0)).backward()
    assert loss.item() == pytest.approx(loss2.item() / len(X0), rel=1e-13)
    torch.testing.assert_close(th.grad, tr.grad, rtol=1e-12, atol=1e-14)
    torch.testing.assert_close(U, torch.stack([_toy_u(x, th0) for x in X0]), rtol=1e-13, atol=1e-13)
