"""The FP64 plain-method case as stated: 2,000 particles (1,000 A + 1,000 B,
only A-B pairs bond, A-A and B-B WCA sigma = 1), cubic periodic box at number
density 0.2, random positions with minimum separation 0.9, Eq. 2b with eps = 1,
sigma = 1, n = 10, cut-off 1.5 used unshifted (the paper's literal form),
lambda = 1; one energy and force evaluation, then 1,000 velocity-Verlet steps
at dt = 0.001 from Maxwell velocities at kT = 0.1.

The GPU's FP64 path is held to the oracle at 1e-12 of the error scales for the
evaluation, and step by step along the trajectory: the total energy
U2 + U3 + K of every step against the oracle's record of the same step (read
after each of 1,000 one-step launches, and from the step kernel's thermo log
of one 1,000-step launch).  In the
unshifted form the energy jumps (v(1.5) = -0.068 for n = 10) whenever a pair
crosses the cut-off, on both sides at the same step; the two trajectories stay
within a few 1e-14 of each other over the 1,000 steps (fixed-point against
FP64 position updates, amplified by the dynamics), far from any pair sitting
that close to a threshold, so every record must agree to the FP64 tolerance.
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


def test_config1_fp64_evaluation_and_nve_record(orc):
    wl = inputs.workload("mix2k", lambda3=1.0)  # N = 2,000, density 0.2, unshifted, NVE, kT = 0.1
    assert wl["n"] == 2000 and wl["density"] == 0.2 and wl["pairs"][(0, 1)]["shift"] == 0
    assert (wl["types"] == 0).sum() == 1000
    tab = oracle_pairs(orc, wl)
    s = make_gpu(wl, "fp64")
    s.compute_forces()
    ref = orc.forces(wl["x"], wl["types"], 2, tab, wl["box"])
    assert_forces_match(s.forces(), ref, TOL["fp64"], "config 1 evaluation")
    assert_thermo_match(s.thermo(), ref, TOL["fp64"], "config 1 evaluation")

    nsteps, dt = 1000, wl["dt"]
    rec = np.zeros((nsteps, 4))
    for k in range(nsteps):
        s.run(1, dt)
        th = s.thermo()
        rec[k] = th["U2"], th["U3"], th["K"], th["n_bonds"]
    assert s.thermo()["step"] == nsteps
    # the same record from the step kernel's thermo log, in one 1,000-step launch
    s2 = make_gpu(wl, "fp64")
    s2.set_thermo_log(1, nsteps)
    s2.run(nsteps, dt)
    log = s2.thermo_log()
    s2.close()
    np.testing.assert_array_equal(log["step"], np.arange(1, nsteps + 1))
    np.testing.assert_array_equal(log["n_bonds"], rec[:, 3])
    np.testing.assert_allclose(np.column_stack([log["U2"], log["U3"], log["K"]]), rec[:, :3], rtol=0,
                               atol=1e-13 * (ref["scale_U2"] + ref["scale_U3"]))
    xo, vo, imo, tho = orc.run(wl["x"], wl["v"], wl["types"], wl["mass"], wl["tags"], 2, tab, wl["box"], dt,
                               nsteps)
    E_gpu = rec[:, 0] + rec[:, 1] + rec[:, 2]
    E_orc = tho[:, 0] + tho[:, 1] + tho[:, 2]
    scale = ref["scale_U2"] + ref["scale_U3"] + np.abs(tho[:, 2]).max()
    dev = np.abs(E_gpu - E_orc)
    assert dev.max() <= TOL["fp64"] * scale, (int(dev.argmax()), dev.max(), scale)
    np.testing.assert_array_equal(rec[:, 3], tho[:, 9])  # bond counts, step by step
    # the unshifted form's energy is not conserved: pairs crossing r_cut make it jump
    jumps = np.abs(np.diff(E_orc))
    assert jumps.max() > 1e-3, "expected cut-off crossings in 1,000 steps"
    x, v, img = s.state()
    assert np.abs((x + img * wl["box"]) - (xo + imo * wl["box"])).max() <= 1e-11
    assert np.abs(v - vo).max() <= 1e-10
    s.close()
