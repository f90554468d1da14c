"""The allocation-free force entry point against the ordinary one and the oracle.

swp_compute_forces_static exists for callers that cannot allocate device
memory when they need forces (a host framework that has reserved the device's
memory and forbids side allocations, a loop that cannot afford cudaMalloc's
device-wide synchronisation).  Its scratch lives in one static device array
shared by every call, so this test makes calls in a row on different
configurations -- a later call must not see an earlier one's leftovers, not
even after a call that failed -- and compares each with swp_compute_forces on
the same input and with the oracle, within the parity tolerances used
throughout (FP32 1e-5, FP64 1e-12 of the per-particle error scale).
Collected last on purpose (file name), so a stop-at-first-failure run has run
every other test before it.
"""
import numpy as np
import pytest

from gpu_helpers import TOL, make_gpu, oracle_pairs
from paper_1912_08569_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_08569_gb300.build import build

    build()
    dev = torch.device("cuda", torch.cuda.current_device())
    return torch, dev, torch.cuda.current_stream(dev).cuda_stream


def _ctx(A, wl, precision, max_nn=64):
    ctx = A.swp_create(wl["n"], 2, wl["box"], precision, 0)
    for (ti, tj), p in wl["pairs"].items():
        A.swp_set_pair(ctx, ti, tj, p["kind"], p.get("eps", 1.0), p.get("sigma", 1.0), p.get("n", 6),
                       p.get("rcut", 0.0), p.get("lambda3", 0.0), p.get("shift", 0), p.get("rbond", 0.0) or 0.0)
    A.swp_set_nlist(ctx, wl["skin"], max_nn)
    return ctx


def _static(cuda, wl, precision, types=True, max_nn=64):
    from paper_1912_08569_gb300 import _abi as A

    torch, dev, stream = cuda
    ctx = _ctx(A, wl, A.SWP_FP64 if precision == "fp64" else A.SWP_FP32, max_nn)
    x = torch.tensor(wl["x"], dtype=torch.float64, device=dev)
    ty = torch.tensor(wl["types"], dtype=torch.int32, device=dev) if types else None
    f = torch.full((wl["n"], 3), float("nan"), dtype=torch.float64, device=dev)
    th = torch.full((9,), float("nan"), dtype=torch.float64, device=dev)
    try:
        A.swp_compute_forces_static(ctx, x, ty, f, th, stream)
    finally:
        A.swp_destroy(ctx)
    return f.cpu().numpy(), th.cpu().numpy()


def _existing(wl, precision):
    s = make_gpu(wl, precision)
    s.compute_forces()
    F, th = s.forces(), s.thermo()
    s.close()
    return F, th


def _check(F, th, ref, tol, what):
    err = np.linalg.norm(F - ref["F"], axis=1)
    assert np.all(err <= tol * ref["fscale"]), (what, float(np.max(err / np.maximum(ref["fscale"], 1e-300))))
    assert abs(th[0] - ref["U2"]) <= tol * ref["scale_U2"], what
    assert abs(th[1] - ref["U3"]) <= tol * ref["scale_U3"], what
    assert np.all(np.abs(th[2:8] - ref["W"]) <= tol * ref["scale_W"] + 1e-300), what
    assert int(round(th[8])) == ref["n_bonds"], what


def test_static_scratch_forces_match_existing_entry_point_and_oracle(orc, cuda):
    configs = [("fp32", inputs.workload("mix2k", lambda3=1.0, n=3000, density=0.5, seed=11)),
               ("fp32", inputs.workload("mix2k", lambda3=5.0, n=2500, density=0.3, seed=12)),
               ("fp64", inputs.workload("mix2k", lambda3=1.0, n=2000, density=0.2, seed=13))]
    for k, (prec, wl) in enumerate(configs):
        F_static, th_static = _static(cuda, wl, prec)
        F_ref, th_ref = _existing(wl, prec)
        ref = orc.forces(wl["x"], wl["types"], 2, oracle_pairs(orc, wl), wl["box"], fp32=prec == "fp32")
        tol = TOL[prec]
        # against the ordinary entry point on the same input
        err = np.linalg.norm(F_static - F_ref, axis=1)
        assert np.all(err <= tol * ref["fscale"]), (k, float(err.max()))
        assert abs(th_static[0] - th_ref["U2"]) <= tol * ref["scale_U2"], k
        assert abs(th_static[1] - th_ref["U3"]) <= tol * ref["scale_U3"], k
        assert int(round(th_static[8])) == th_ref["n_bonds"], k
        # and against the oracle
        _check(F_static, th_static, ref, tol, f"static call {k} ({prec})")


def test_static_scratch_without_types(orc, cuda):
    """type_dev = NULL: every particle is type 0 (a WCA fluid here)."""
    wl = inputs.workload("mix2k", lambda3=1.0, n=1500, density=0.4, seed=14)
    F, th = _static(cuda, wl, "fp32", types=False)
    zeros = np.zeros(wl["n"], dtype=np.int32)
    ref = orc.forces(wl["x"], zeros, 2, oracle_pairs(orc, wl), wl["box"], fp32=True)
    _check(F, th, ref, TOL["fp32"], "no types")
    assert ref["n_bonds"] == 0 and th[1] == 0.0


def test_static_scratch_overflow_then_clean_call(orc, cuda):
    """A row longer than max_nn fails with SWP_ERR_NLIST_OVERFLOW; the next call
    on a valid context starts from a clean control block and is right."""
    from paper_1912_08569_gb300 import _abi as A

    wl = inputs.workload("mix2k", lambda3=1.0, n=2000, density=0.5, seed=15)
    with pytest.raises(A.SwpError) as e:
        _static(cuda, wl, "fp32", max_nn=3)
    assert e.value.code == A.SWP_ERR_NLIST_OVERFLOW, str(e.value)
    F, th = _static(cuda, wl, "fp32")
    ref = orc.forces(wl["x"], wl["types"], 2, oracle_pairs(orc, wl), wl["box"], fp32=True)
    _check(F, th, ref, TOL["fp32"], "after an overflow")


def test_static_scratch_rejects_oversized_systems(cuda):
    from paper_1912_08569_gb300 import _abi as A

    torch, dev, stream = cuda
    n = 200_000
    box = inputs.cubic_box(n, 0.5)
    wl = dict(n=n, box=box, pairs=inputs.swap_pairs(), skin=0.3)
    ctx = _ctx(A, wl, A.SWP_FP32)
    x = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    f = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    with pytest.raises(A.SwpError) as e:
        A.swp_compute_forces_static(ctx, x, None, f, None, stream)
    assert e.value.code == A.SWP_ERR_INVALID and "static scratch" in str(e.value)
    A.swp_destroy(ctx)
