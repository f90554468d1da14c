"""The resident step (one grid barrier per step, each block's neighbourhood in
shared memory) against the two-barrier step and against the oracle, and the
bounded device waits.

The resident mode changes where the data of a step live and how many barriers
separate its phases, not its arithmetic: forces and trajectories must be equal
bit for bit to those of the two-barrier path (same per-entry operations, same
summation orders), the energies and virial equal within the rounding of their
sums, and the forces at the end of a run equal the oracle's at the positions
reached, within the FP32 tolerance (Eq. 2b, Eq. 3bp through S_i).
"""
import numpy as np
import pytest

from gpu_helpers import TOL, assert_forces_match, assert_thermo_match, make_gpu, oracle_pairs
from paper_1912_08569_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_08569_gb300.build import build

    build()


def _wl(n, density, lam, seed=3, kT=0.1, shift=0):
    wl = inputs.workload("mix2k", lambda3=lam, n=n, density=density, seed=seed, shift=shift)
    wl["v"] = inputs.maxwell_velocities(n, kT, 1.0, seed=seed + 1)
    return wl


def _run_pair(wl, nsteps, kT, gamma):
    a = make_gpu(wl, "fp32")
    b = make_gpu(wl, "fp32")
    b.set_resident(False)
    for s in (a, b):
        s.run(nsteps, 0.001, kT, gamma)
    return a, b


@pytest.mark.parametrize("n,density,lam,gamma", [
    (151, 0.3, 1.0, 1.0),      # fewer particles than blocks: most blocks own one or none
    (2000, 0.3, 1.0, 0.0),     # NVE
    (20000, 0.5, 5.0, 1.0),
    (60013, 0.4, 0.0, 1.0),    # ragged; lambda = 0 still forms S
])
def test_resident_equals_two_barrier_path(orc, n, density, lam, gamma):
    wl = _wl(n, density, lam)
    a, b = _run_pair(wl, 300, 0.1, gamma)
    ta, tb = a.thermo(), b.thermo()
    assert ta["resident_steps"] == 300 and tb["resident_steps"] == 0
    assert ta["n_rebuilds"] == tb["n_rebuilds"]
    xa, va, ia = a.state()
    xb, vb, ib = b.state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(ia, ib)
    assert np.array_equal(a.forces(), b.forces())
    ref = orc.forces(xa, wl["types"], 2, oracle_pairs(orc, wl), wl["box"], fp32=True)
    assert_forces_match(a.forces(), ref, TOL["fp32"], f"resident n={n}")
    # the energies and virial of the last step: the same quantities, summed in another grouping
    assert_thermo_match(ta, ref, TOL["fp32"], "resident thermo")
    assert_thermo_match(tb, ref, TOL["fp32"], "two-barrier thermo")
    assert ta["K"] == pytest.approx(tb["K"], rel=1e-6)
    a.close()
    b.close()


def test_resident_at_full_size_matches_oracle(orc):
    """The 100k-particle FP32 workload (N = 100,000, density 0.5, lambda = 1,
    BAOAB kT = 0.05): 200 resident steps through list rebuilds, then every force
    against the oracle at the positions reached."""
    wl = inputs.workload("mix100k", lambda3=1.0)
    s = make_gpu(wl, "fp32")
    s.run(200, wl["dt"], wl["kT"], wl["gamma"])
    th = s.thermo()
    assert th["resident_steps"] == 200
    x, _, _ = s.state()
    ref = orc.forces(x, wl["types"], 2, oracle_pairs(orc, wl), wl["box"], fp32=True)
    assert_forces_match(s.forces(), ref, TOL["fp32"], "mix100k resident")
    assert_thermo_match(th, ref, TOL["fp32"], "mix100k resident")
    s.close()


def test_resident_falls_back_when_the_halo_does_not_fit(orc):
    """A dense system on a small grid: 1,000 particles per block at density 0.7
    have about 2,400 halo particles and 20,000 local entries, beyond the
    shared-memory capacity (3,072 and 16,384), so every block agrees to take
    the two-barrier path, and the run is still right."""
    wl = _wl(24000, 0.7, 1.0, seed=8)
    s = make_gpu(wl, "fp32")
    s.set_grid(24)
    s.run(100, 0.001, 0.1, 1.0)
    th = s.thermo()
    assert th["resident_steps"] == 0
    x, _, _ = s.state()
    ref = orc.forces(x, wl["types"], 2, oracle_pairs(orc, wl), wl["box"], fp32=True)
    assert_forces_match(s.forces(), ref, TOL["fp32"], "fallback")
    assert th["step"] == 100
    s.close()


def test_withheld_arrival_times_out_and_the_context_recovers(orc):
    """Failure detection without a fault: one block's arrival at the first grid
    barrier is withheld, every other block's wait runs out after 1 ms, the call
    reports SWP_ERR_TIMEOUT, and after a new state the context computes the
    oracle's forces again."""
    import torch

    from paper_1912_08569_gb300 import _abi as A

    wl = _wl(2000, 0.3, 1.0, seed=6)
    s = make_gpu(wl, "fp32")
    s.compute_forces()
    s.set_timeout(1_000_000)
    A.swp_set_withhold_arrival(s.ctx, 1)
    with pytest.raises(A.SwpError) as e:
        s.run(100, 0.001, 0.1, 1.0)
    assert e.value.code == A.SWP_ERR_TIMEOUT, str(e.value)
    torch.cuda.synchronize()  # nothing is left running
    s.set_timeout(2_000_000_000)
    s.set_state(wl["x"], wl["v"], wl["types"], wl["mass"])
    s.compute_forces()
    ref = orc.forces(wl["x"], wl["types"], 2, oracle_pairs(orc, wl), wl["box"], fp32=True)
    assert_forces_match(s.forces(), ref, TOL["fp32"], "after recovery")
    s.run(20, 0.001, 0.1, 1.0)  # the request was consumed by the failed launch
    assert s.thermo()["step"] == 20
    s.close()
