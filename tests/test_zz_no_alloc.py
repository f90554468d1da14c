"""The allocation-free force entry point against the ordinary one.

swp_compute_forces_static exists for callers that cannot allocate device
memory when they need forces (a host framework that has reserved the device's
memory, code driven from inside a stream capture, a loop that cannot afford
cudaMalloc's device-wide synchronisation).  Its scratch lives in one static
device array shared by every call, so this test makes two calls in a row on
different configurations -- the second must not see the first's leftovers --
and compares each with swp_compute_forces on the same input, within the FP32
parity tolerance used throughout (1e-5 of the per-particle error scale).
Collected last on purpose (file name), so a stop-at-first-failure run has run
every other test before it.
"""
import numpy as np
import pytest

from gpu_helpers import TOL, make_gpu, oracle_pairs
from paper_1912_08569_gb300 import inputs

pytestmark = pytest.mark.gpu


def _forces_existing(wl):
    s = make_gpu(wl, "fp32")
    s.compute_forces()
    F, th = s.forces(), s.thermo()
    s.close()
    return F, th


def test_static_scratch_forces_match_existing_entry_point(orc):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_08569_gb300 import _abi as A
    from paper_1912_08569_gb300.build import build

    build()
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev).cuda_stream
    configs = [inputs.workload("mix2k", lambda3=1.0, n=3000, density=0.5, seed=11),
               inputs.workload("mix2k", lambda3=5.0, n=2500, density=0.3, seed=12)]
    for k, wl in enumerate(configs):
        ctx = A.swp_create(wl["n"], 2, wl["box"], A.SWP_FP32, 0)
        for (ti, tj), p in wl["pairs"].items():
            A.swp_set_pair(ctx, ti, tj, p["kind"], p.get("eps", 1.0), p.get("sigma", 1.0),
                           p.get("n", 6), p.get("rcut", 0.0), p.get("lambda3", 0.0),
                           p.get("shift", 0), p.get("rbond", 0.0) or 0.0)
        A.swp_set_nlist(ctx, wl["skin"], 64)
        x = torch.tensor(wl["x"], dtype=torch.float64, device=dev)
        ty = torch.tensor(wl["types"], dtype=torch.int32, device=dev)
        f = torch.full((wl["n"], 3), float("nan"), dtype=torch.float64, device=dev)
        th = torch.full((9,), float("nan"), dtype=torch.float64, device=dev)
        A.swp_compute_forces_static(ctx, x, ty, f, th, stream)
        F_static = f.cpu().numpy()
        th_static = th.cpu().numpy()
        A.swp_destroy(ctx)

        F_ref, th_ref = _forces_existing(wl)
        scale = orc.forces(wl["x"], wl["types"], 2, oracle_pairs(orc, wl), wl["box"], fp32=True)
        err = np.linalg.norm(F_static - F_ref, axis=1)
        assert np.all(err <= TOL["fp32"] * scale["fscale"]), (k, float(err.max()))
        assert abs(th_static[0] - th_ref["U2"]) <= TOL["fp32"] * scale["scale_U2"], k
        assert abs(th_static[1] - th_ref["U3"]) <= TOL["fp32"] * scale["scale_U3"], k
        assert np.all(np.abs(th_static[2:8] - th_ref["W"]) <= TOL["fp32"] * scale["scale_W"]), k
        assert int(round(th_static[8])) == th_ref["n_bonds"], k


def test_static_scratch_rejects_oversized_systems():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_08569_gb300 import _abi as A

    n = 200_000
    box = inputs.cubic_box(n, 0.5)
    ctx = A.swp_create(n, 2, box, A.SWP_FP32, 0)
    for (ti, tj), p in inputs.swap_pairs().items():
        A.swp_set_pair(ctx, ti, tj, p["kind"], p.get("eps", 1.0), p.get("sigma", 1.0), p.get("n", 6),
                       p.get("rcut", 0.0), p.get("lambda3", 0.0), 0, p.get("rbond", 0.0) or 0.0)
    A.swp_set_nlist(ctx, 0.3, 64)
    dev = torch.device("cuda", torch.cuda.current_device())
    x = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    f = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    with pytest.raises(A.SwpError) as e:
        A.swp_compute_forces_static(ctx, x, None, f, None, torch.cuda.current_stream(dev).cuda_stream)
    assert e.value.code == A.SWP_ERR_INVALID and "static scratch" in str(e.value)
    A.swp_destroy(ctx)
