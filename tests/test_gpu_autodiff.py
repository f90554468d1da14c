"""Differentiable energy (GPU path) against central finite differences of the
FP64 oracle, h = 1e-4.

dU/d(lambda, eps, sigma) and dF/d(lambda, eps, sigma) from the library are
compared with central differences of the oracle's energy and forces under the
same change of the coefficients (the oracle takes its cut-off decisions on
the same FP32 positions in FP32 mode).  The autograd wrapper is checked for
dU/dx = -F, dU/dtheta, and the double backward of a force-matching loss
against central differences of the same loss built from oracle forces.

Tolerances: central differences with h = 1e-4 carry a truncation error of
order h^2 times the third derivative (about 1e-5 relative here), so the FP64
path is held to 1e-4 and the FP32 path, whose pair terms are rounded to FP32,
to 1e-3 (relative to the size of the derivative).  dF/dsigma jumps where a
reactive pair crosses r_min (vh is only once continuously differentiable
there and r_min moves with sigma), so a difference quotient that straddles
r_min is meaningless: particles with a reactive partner within 3h of r_min
are left out of the force comparison, and the loss test uses snapshots with
no such pair.
"""
import numpy as np
import pytest

from gpu_helpers import make_gpu, oracle_pairs
from paper_1912_08569_gb300 import inputs

pytestmark = pytest.mark.gpu

H = 1e-4
TOLD = {"fp64": 1e-4, "fp32": 1e-3}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_08569_gb300.build import build

    build()


def _wl(n=2000, density=0.4, lam=1.0, seed=5):
    wl = inputs.workload("mix2k", lambda3=lam, n=n, density=density, seed=seed, shift=0)
    return wl


def _with_theta(pairs, theta):
    p = {k: dict(v) for k, v in pairs.items()}
    p[(0, 1)]["lambda3"], p[(0, 1)]["eps"], p[(0, 1)]["sigma"] = theta
    return p


def _oracle(orc, wl, theta, fp32):
    pairs = _with_theta(wl["pairs"], theta)
    return orc.forces(wl["x"], wl["types"], 2, orc.pair_table(2, pairs), wl["box"], fp32=fp32)


def _near_rmin(wl, sigma, n_exp=10, band=3 * H):
    """Particles with a reactive partner whose distance is within band of r_min."""
    x, L = wl["x"], wl["box"]
    d = x[None, :, :] - x[:, None, :]
    d -= L * np.round(d / L)
    r = np.sqrt((d * d).sum(-1))
    react = wl["types"][:, None] != wl["types"][None, :]
    near = react & (np.abs(r - sigma * 2.0 ** (1.0 / n_exp)) < band * 2.0 ** (1.0 / n_exp))
    return near.any(axis=1)


def _fd(orc, wl, theta, fp32):
    """Central differences of U and F in each coefficient."""
    dU = np.zeros(3)
    dF = np.zeros((3, wl["n"], 3))
    for k in range(3):
        tp, tm = list(theta), list(theta)
        tp[k] += H
        tm[k] -= H
        rp, rm = _oracle(orc, wl, tp, fp32), _oracle(orc, wl, tm, fp32)
        dU[k] = ((rp["U2"] + rp["U3"]) - (rm["U2"] + rm["U3"])) / (2 * H)
        dF[k] = (rp["F"] - rm["F"]) / (2 * H)
    return dU, dF


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("theta", [(1.0, 1.0, 1.0), (2.0, 0.8, 1.05), (0.5, 1.2, 0.95)])
def test_param_grad_matches_finite_differences(orc, precision, theta):
    import torch
    from paper_1912_08569_gb300 import _abi as A

    wl = _wl()
    pairs = _with_theta(wl["pairs"], theta)
    wl2 = dict(wl, pairs=pairs)
    s = make_gpu(wl2, precision)
    s.compute_forces()
    dF = torch.empty((3, wl["n"], 3), dtype=torch.float64, device=s.device)
    dU = A.swp_param_grad(s.ctx, 0, 1, dF)
    dU_fd, dF_fd = _fd(orc, wl, theta, precision == "fp32")
    tol = TOLD[precision]
    keep = ~_near_rmin(wl, theta[2])
    assert keep.sum() > 0.95 * wl["n"]
    for k in range(3):
        assert abs(dU[k] - dU_fd[k]) <= tol * (abs(dU_fd[k]) + 1.0), (k, dU[k], dU_fd[k])
        got = dF[k].cpu().numpy()[keep]
        ref = dF_fd[k][keep]
        err = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-12)
        assert err <= tol, (k, err)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_param_grad_at_lambda_zero(orc, precision):
    """At lambda = 0 (no three-body term) U is linear in lambda, so the one-sided
    difference U(h) - U(0) over h is exact up to rounding (lambda < 0 is not a
    valid coefficient)."""
    import torch
    from paper_1912_08569_gb300 import _abi as A

    wl = _wl()
    theta = (0.0, 1.0, 1.0)
    s = make_gpu(dict(wl, pairs=_with_theta(wl["pairs"], theta)), precision)
    s.compute_forces()
    dF = torch.empty((3, wl["n"], 3), dtype=torch.float64, device=s.device)
    dU = A.swp_param_grad(s.ctx, 0, 1, dF)
    r0, r1 = _oracle(orc, wl, theta, precision == "fp32"), _oracle(orc, wl, (H, 1.0, 1.0), precision == "fp32")
    fd = ((r1["U2"] + r1["U3"]) - (r0["U2"] + r0["U3"])) / H
    assert abs(dU[0] - fd) <= TOLD[precision] * (abs(fd) + 1.0), (dU[0], fd)
    dF_fd = (r1["F"] - r0["F"]) / H
    err = np.linalg.norm(dF[0].cpu().numpy() - dF_fd) / np.linalg.norm(dF_fd)
    assert err <= TOLD[precision], err


def test_param_grad_rejects_shifted_and_stale():
    from paper_1912_08569_gb300 import _abi as A

    wl = inputs.workload("mix2k", n=500, shift=1, seed=3)
    s = make_gpu(wl, "fp32")
    s.compute_forces()
    with pytest.raises(A.SwpError):
        A.swp_param_grad(s.ctx, 0, 1)
    wl = _wl(n=500)
    s = make_gpu(wl, "fp32")  # state set, forces not computed
    with pytest.raises(A.SwpError):
        A.swp_param_grad(s.ctx, 0, 1)


def _model(wl, precision):
    from paper_1912_08569_gb300.autodiff import SwapModel

    s = make_gpu(wl, precision)
    return SwapModel(s, wl["pairs"], wl["types"])


def test_autograd_energy_backward(orc):
    import torch
    from paper_1912_08569_gb300 import autodiff

    wl = _wl()
    m = _model(wl, "fp64")
    x = torch.tensor(wl["x"], dtype=torch.float64, device=m.s.device, requires_grad=True)
    theta = torch.tensor([1.0, 1.0, 1.0], dtype=torch.float64, device=m.s.device, requires_grad=True)
    U = autodiff.energy(m, x, theta)
    U.backward()
    ref = _oracle(orc, wl, (1.0, 1.0, 1.0), False)
    assert abs(U.item() - (ref["U2"] + ref["U3"])) <= 1e-12 * ref["scale_U2"] + 1e-12 * ref["scale_U3"]
    err = np.linalg.norm(-x.grad.cpu().numpy() - ref["F"], axis=1)
    assert np.all(err <= 1e-12 * ref["fscale"])
    dU_fd, _ = _fd(orc, wl, (1.0, 1.0, 1.0), False)
    g = theta.grad.cpu().numpy()
    assert np.all(np.abs(g - dU_fd) <= TOLD["fp64"] * (np.abs(dU_fd) + 1.0)), (g, dU_fd)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_force_matching_double_backward(orc, precision):
    """Loss = mean over snapshots and components of (F(theta) - F_ref)^2, with
    F_ref the oracle forces at theta_ref; F from torch.autograd.grad(U, x,
    create_graph=True).  dLoss/dtheta against central differences of the
    oracle's loss."""
    import torch
    from paper_1912_08569_gb300 import autodiff

    theta_ref = (1.0, 1.0, 1.0)
    theta0 = (1.3, 0.9, 1.02)
    snaps = []
    for seed in range(40, 100):  # snapshots with no reactive pair straddling r_min
        w = _wl(n=1200, seed=seed)
        if not _near_rmin(w, theta0[2]).any():
            snaps.append(w)
        if len(snaps) == 3:
            break
    assert len(snaps) == 3
    refs = [_oracle(orc, w, theta_ref, precision == "fp32")["F"] for w in snaps]
    m = _model(snaps[0], precision)
    theta = torch.tensor(theta0, dtype=torch.float64, device=m.s.device, requires_grad=True)
    loss = 0.0
    for w, Fr in zip(snaps, refs):
        m.types = torch.as_tensor(w["types"], device=m.s.device)
        x = torch.tensor(w["x"], dtype=torch.float64, device=m.s.device, requires_grad=True)
        U = autodiff.energy(m, x, theta)
        (gx,) = torch.autograd.grad(U, x, create_graph=True)
        F = -gx
        loss = loss + ((F - torch.as_tensor(Fr, device=m.s.device)) ** 2).mean()
    loss = loss / len(snaps)
    loss.backward()
    g = theta.grad.cpu().numpy()

    def oracle_loss(th):
        return np.mean([np.mean((_oracle(orc, w, th, precision == "fp32")["F"] - Fr) ** 2)
                        for w, Fr in zip(snaps, refs)])

    L0 = oracle_loss(theta0)
    assert abs(loss.item() - L0) <= (1e-10 if precision == "fp64" else 1e-4) * L0
    for k in range(3):
        tp, tm = list(theta0), list(theta0)
        tp[k] += H
        tm[k] -= H
        fd = (oracle_loss(tp) - oracle_loss(tm)) / (2 * H)
        assert abs(g[k] - fd) <= TOLD[precision] * (abs(fd) + 1e-3 * L0), (k, g[k], fd)

    # the same gradient through forces() directly
    theta2 = torch.tensor(theta0, dtype=torch.float64, device=m.s.device, requires_grad=True)
    loss2 = 0.0
    for w, Fr in zip(snaps, refs):
        m.types = torch.as_tensor(w["types"], device=m.s.device)
        x = torch.tensor(w["x"], dtype=torch.float64, device=m.s.device)
        F = autodiff.forces(m, x, theta2)
        loss2 = loss2 + ((F - torch.as_tensor(Fr, device=m.s.device)) ** 2).mean()
    (loss2 / len(snaps)).backward()
    np.testing.assert_allclose(theta2.grad.cpu().numpy(), g, rtol=1e-12, atol=0)


def _oracle_threaded_forces(orc, w, theta, fp32):
    pairs = _with_theta(w["pairs"], theta)
    try:
        return orc.forces(w["x"], w["types"], 2, orc.pair_table(2, pairs), w["box"], fp32=fp32, threaded=True)["F"]
    except Exception:  # no OpenMP build on this host: the serial oracle (same arithmetic)
        return orc.forces(w["x"], w["types"], 2, orc.pair_table(2, pairs), w["box"], fp32=fp32)["F"]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_force_matching_double_backward_64_snapshots_of_20k(orc, precision):
    """The differentiable case as stated: 64 seeded snapshots of 20,000
    particles (A:B 1:1, density 0.4), loss = mean over snapshots of the mean
    squared force error against oracle forces at theta_ref = (1, 1, 1),
    gradient at theta0 through autodiff.energy and a double backward, every
    evaluation enqueued without host synchronisation.  Against central
    differences of the oracle's loss with h = 1e-5: at this size some reactive
    pairs always lie within h of r_min, where dF/dsigma jumps, but over 1.3 M
    particles their share is small -- the difference quotients at h = 1e-4,
    1e-5 and 1e-6 agree to 8e-6 (sigma) and 1e-8 (lambda, eps) relative."""
    import torch
    from paper_1912_08569_gb300 import autodiff

    h, fp32 = 1e-5, precision == "fp32"
    theta_ref, theta0 = (1.0, 1.0, 1.0), [1.3, 0.9, 1.02]
    snaps = [inputs.workload("mix100k", n=20000, density=0.4, seed=100 + k, shift=0) for k in range(64)]
    refs = [_oracle_threaded_forces(orc, w, theta_ref, fp32) for w in snaps]
    m = _model(snaps[0], precision)
    dev = m.s.device
    theta = torch.tensor(theta0, dtype=torch.float64, device=dev, requires_grad=True)
    loss = 0.0
    for w, Fr in zip(snaps, refs):
        m.types = torch.as_tensor(w["types"], device=dev)
        x = torch.tensor(w["x"], dtype=torch.float64, device=dev, requires_grad=True)
        (gx,) = torch.autograd.grad(autodiff.energy(m, x, theta), x, create_graph=True)
        loss = loss + ((-gx - torch.as_tensor(Fr, device=dev)) ** 2).mean()
    loss = loss / len(snaps)
    loss.backward()
    m.check()  # nothing latched on the device (list rows, non-finite forces)
    g = theta.grad.cpu().numpy()

    def oracle_loss(th):
        return np.mean([np.mean((_oracle_threaded_forces(orc, w, th, fp32) - Fr) ** 2)
                        for w, Fr in zip(snaps, refs)])

    L0 = oracle_loss(theta0)
    assert abs(loss.item() - L0) <= (1e-10 if precision == "fp64" else 1e-4) * L0
    tol = {"fp64": 1e-5, "fp32": 1e-3}[precision]
    for k in range(3):
        tp, tm = list(theta0), list(theta0)
        tp[k] += h
        tm[k] -= h
        fd = (oracle_loss(tp) - oracle_loss(tm)) / (2 * h)
        assert abs(g[k] - fd) <= tol * (abs(fd) + 1e-3 * L0), (k, g[k], fd)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_eval_grad_equals_host_driven_path(precision):
    """swp_eval_grad (theta and positions from device memory, nothing read
    back) against swp_set_pair + swp_set_state + swp_compute_forces +
    swp_param_grad on the same inputs: the same coefficients reach the same
    kernels, so energy, forces and derivatives agree bit for bit; several
    thetas in a row on one context, then an ordinary run that must take the
    host coefficients again."""
    import torch
    from paper_1912_08569_gb300 import _abi as A

    wl = _wl(n=3000, seed=8)
    m = _model(wl, precision)
    dev = m.s.device
    x = torch.tensor(wl["x"], dtype=torch.float64, device=dev)
    for theta in [(1.0, 1.0, 1.0), (2.0, 0.8, 1.05), (0.5, 1.2, 0.95)]:
        U, F, dU, dF = m.evaluate(x, torch.tensor(theta, dtype=torch.float64, device=dev))
        h = make_gpu(dict(wl, pairs=_with_theta(wl["pairs"], theta)), precision)
        h.compute_forces()
        th = h.thermo()
        dF_h = torch.empty((3, wl["n"], 3), dtype=torch.float64, device=dev)
        dU_h = A.swp_param_grad(h.ctx, 0, 1, dF_h)
        assert U.item() == th["U2"] + th["U3"], (theta, U.item(), th["U2"] + th["U3"])
        np.testing.assert_array_equal(F.cpu().numpy(), h.forces())
        np.testing.assert_array_equal(dU.cpu().numpy(), np.asarray(dU_h))
        np.testing.assert_array_equal(dF.cpu().numpy(), dF_h.cpu().numpy())
        h.close()
    m.check()
    # an ordinary evaluation afterwards uses the coefficients of swp_set_pair (theta = 1, 1, 1)
    m.s.set_state(wl["x"], None, wl["types"])
    m.s.compute_forces()
    U1, _, _, _ = m.evaluate(x, torch.tensor((1.0, 1.0, 1.0), dtype=torch.float64, device=dev), want_grad=False)
    th = m.s.thermo()
    assert th["U2"] + th["U3"] == U1.item()


def test_eval_grad_latches_out_of_range_types():
    import torch
    from paper_1912_08569_gb300 import _abi as A

    wl = _wl(n=800, seed=9)
    m = _model(wl, "fp32")
    dev = m.s.device
    bad = torch.as_tensor(wl["types"], device=dev).clone()
    bad[5] = 7
    m.types = bad
    m.evaluate(torch.tensor(wl["x"], dtype=torch.float64, device=dev),
               torch.tensor((1.0, 1.0, 1.0), dtype=torch.float64, device=dev))
    with pytest.raises(A.SwpError) as e:
        m.check()
    assert e.value.code == A.SWP_ERR_INVALID and "type" in str(e.value)
    # the context recovers with a valid state
    m.types = torch.as_tensor(wl["types"], device=dev)
    m.evaluate(torch.tensor(wl["x"], dtype=torch.float64, device=dev),
               torch.tensor((1.0, 1.0, 1.0), dtype=torch.float64, device=dev))
    m.check()


def test_energy_batch_matches_per_snapshot_energy():
    """The batched Function (one autograd node for S snapshots) gives the
    per-snapshot Function's energies bit for bit and its force-matching
    gradient to rounding."""
    import torch
    from paper_1912_08569_gb300 import autodiff

    snaps = [_wl(n=1500, seed=60 + k) for k in range(5)]
    m = _model(snaps[0], "fp32")
    dev = m.s.device
    R = torch.stack([torch.as_tensor(w["x"] * 0.0 + 0.1, device=dev) for w in snaps])
    theta0 = (1.3, 0.9, 1.02)
    X = torch.stack([torch.tensor(w["x"], dtype=torch.float64, device=dev) for w in snaps]).requires_grad_(True)
    th = torch.tensor(theta0, dtype=torch.float64, device=dev, requires_grad=True)
    U = autodiff.energy_batch(m, X, th)
    (gX,) = torch.autograd.grad(U.sum(), X, create_graph=True)
    ((gX + R) ** 2).mean().backward()
    t2 = torch.tensor(theta0, dtype=torch.float64, device=dev, requires_grad=True)
    loss2, U2 = 0.0, []
    for k in range(len(snaps)):
        x = X[k].detach().clone().requires_grad_(True)
        u = autodiff.energy(m, x, t2)
        U2.append(u.detach())
        (gx,) = torch.autograd.grad(u, x, create_graph=True)
        loss2 = loss2 + ((gx + R[k]) ** 2).mean()
    (loss2 / len(snaps)).backward()
    m.check()
    np.testing.assert_array_equal(U.detach().cpu().numpy(), torch.stack(U2).cpu().numpy())
    np.testing.assert_allclose(th.grad.cpu().numpy(), t2.grad.cpu().numpy(), rtol=1e-12, atol=0)
