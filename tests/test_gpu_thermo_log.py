"""The thermo log against per-launch reads: a record of the energies, virial,
kinetic energy and bond count of every logged step, written by the step
kernel itself (the step kernel sums those terms only on logged steps and on
the last step of each launch).

A run of m steps in one launch with a record every step must give, step by
step, what m one-step launches report through swp_read_thermo: the
trajectories are the same bit for bit (launch boundaries do not change the
dynamics), and so are the block partials and their reduction (same order).
Checked in the FP32 resident step, the FP32 two-barrier step and the FP64
step, with the interval, the ring's wrap-around across launches and the
argument errors.
"""
import numpy as np
import pytest

from gpu_helpers import make_gpu
from paper_1912_08569_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_08569_gb300.build import build

    build()


def _wl(seed=21, n=3000):
    wl = inputs.workload("mix2k", lambda3=1.0, n=n, density=0.5, seed=seed)
    wl["seed"] = 77
    return wl


def _per_step(wl, precision, nsteps, resident):
    s = make_gpu(wl, precision)
    s.set_resident(resident)
    rows = []
    for _ in range(nsteps):
        s.run(1, wl["dt"], 0.1, 1.0)
        th = s.thermo()
        rows.append((th["step"], th["U2"], th["U3"], th["K"], *th["W"], th["n_bonds"]))
    s.close()
    return np.array(rows)


@pytest.mark.parametrize("precision,resident", [("fp32", True), ("fp32", False), ("fp64", False)])
def test_log_every_step_matches_one_step_launches(precision, resident):
    wl, nsteps = _wl(), 60
    s = make_gpu(wl, precision)
    s.set_resident(resident)
    s.set_thermo_log(1, 128)
    s.run(nsteps, wl["dt"], 0.1, 1.0)
    log = s.thermo_log()
    th = s.thermo()
    if precision == "fp32" and resident:
        assert th["resident_steps"] == nsteps
    s.close()
    ref = _per_step(wl, precision, nsteps, resident)
    np.testing.assert_array_equal(log["step"], np.arange(1, nsteps + 1))
    np.testing.assert_array_equal(log["step"], ref[:, 0])
    np.testing.assert_array_equal(log["n_bonds"], ref[:, 10].astype(np.int64))
    got = np.column_stack([log["U2"], log["U3"], log["K"], log["W"]])
    scale = np.abs(ref[:, 1:10]).max(axis=0) + 1e-300
    assert np.all(np.abs(got - ref[:, 1:10]) <= 1e-13 * scale), np.abs(got - ref[:, 1:10]).max(axis=0) / scale
    # the launch's last step is also its thermo record, bit for bit
    assert (log["U2"][-1], log["U3"][-1], log["K"][-1]) == (th["U2"], th["U3"], th["K"])
    np.testing.assert_array_equal(log["W"][-1], th["W"])


def test_log_interval_and_ring_wrap():
    wl = _wl(seed=22)
    s = make_gpu(wl, "fp32")
    s.set_thermo_log(5, 4)
    s.run(50, wl["dt"], 0.1, 1.0)
    np.testing.assert_array_equal(s.thermo_log()["step"], [35, 40, 45, 50])
    s.run(12, wl["dt"], 0.1, 1.0)  # steps 51..62: records at 55 and 60, across the ring's end
    log = s.thermo_log()
    np.testing.assert_array_equal(log["step"], [45, 50, 55, 60])
    assert np.all(np.isfinite(log["U2"])) and np.all(log["K"] > 0)
    # set_state starts the log (and the step count) afresh
    s.set_state(wl["x"], wl["v"], wl["types"], wl["mass"])
    s.run(3, wl["dt"], 0.1, 1.0)
    assert len(s.thermo_log()["step"]) == 0
    s.run(2, wl["dt"], 0.1, 1.0)
    np.testing.assert_array_equal(s.thermo_log()["step"], [5])
    s.close()


def test_log_argument_errors():
    import torch
    from paper_1912_08569_gb300 import _abi as A

    wl = _wl(seed=23, n=500)
    s = make_gpu(wl, "fp32")
    with pytest.raises(RuntimeError):
        s.thermo_log()  # none set
    nb = A.swp_thermo_log_bytes(s.ctx, 8)
    assert nb > 0 and A.swp_thermo_log_bytes(s.ctx, 0) == 0
    ring = torch.empty(nb + 512, dtype=torch.uint8, device=s.device)
    for every, cap, ptr, nbytes in [(-1, 8, ring.data_ptr(), nb), (1, 0, ring.data_ptr(), nb),
                                    (1, 8, None, nb), (1, 8, ring.data_ptr() + 8, nb),
                                    (1, 8, ring.data_ptr(), nb - 1)]:
        with pytest.raises(A.SwpError) as e:
            A.swp_set_thermo_log(s.ctx, every, cap, ptr, nbytes)
        assert e.value.code == A.SWP_ERR_INVALID
    A.swp_set_thermo_log(s.ctx, 2, 8, ring.data_ptr(), nb)
    s.run(4, wl["dt"], 0.1, 1.0)
    rec = torch.empty((8, 10), dtype=torch.float64, device=s.device)
    stp = torch.empty(8, dtype=torch.int64, device=s.device)
    assert A.swp_thermo_log(s.ctx, rec, stp, 1) == 1  # the newest record only
    assert int(stp[0]) == 4
    A.swp_set_thermo_log(s.ctx, 0)
    with pytest.raises(A.SwpError):
        A.swp_thermo_log(s.ctx, rec, stp, 8)
    s.close()
