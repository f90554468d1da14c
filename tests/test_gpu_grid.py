"""Step kernel on fewer blocks than SMs (swp_set_grid) against the FP64 oracle.

Requests below ten blocks run on ten (one block per thermo quantity reduced
in parallel); a block of a small grid walks its particles in several
sub-chunks.  Each grid must give the oracle's forces, thermo record and
trajectories at the usual tolerances, and a change of grid between runs must
rebuild the list and carry on.
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


def _min_image(d, box):
    return d - box * np.round(d / box)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("grid", [1, 10, 11, 33, 76])
def test_forces_on_small_grids(orc, precision, grid):
    wl = inputs.workload("mix2k", lambda3=2.0, n=3001, density=0.5, seed=4)
    s = make_gpu(wl, precision)
    s.set_grid(grid)
    s.compute_forces()
    ref = orc.forces(wl["x"], wl["types"], 2, oracle_pairs(orc, wl), wl["box"], fp32=precision == "fp32")
    assert_forces_match(s.forces(), ref, TOL[precision], f"grid={grid}")
    assert_thermo_match(s.thermo(), ref, TOL[precision], f"grid={grid}")


@pytest.mark.parametrize("grid", [10, 17])
def test_trajectory_with_rebuilds_on_small_grids(orc, grid):
    wl = inputs.workload("mix2k", lambda3=1.0, n=1500, density=0.3, seed=2, shift=1)
    wl["v"] = inputs.maxwell_velocities(1500, 1.0, 1.0, seed=9)
    wl["skin"] = 0.08
    dt, kT, nsteps = 0.001, 1.0, 300
    s = make_gpu(wl, "fp64")
    s.set_grid(grid)
    s.run(nsteps, dt, kT, 1.0)
    x, v, img = s.state()
    th = s.thermo()
    assert th["n_rebuilds"] >= 5
    xo, vo, imo, tho = orc.run(wl["x"], wl["v"], wl["types"], wl["mass"], wl["tags"], 2, oracle_pairs(orc, wl),
                               wl["box"], dt, nsteps, kT=kT, gamma=1.0, seed=wl["seed"], fp32=False)
    assert np.abs((x + img * wl["box"]) - (xo + imo * wl["box"])).max() <= 1e-8
    assert np.abs(v - vo).max() <= 1e-6
    assert th["K"] == pytest.approx(tho[-1, 2], rel=1e-10)


def test_dumbbell_small_grid_matches_full_grid():
    """The paper's timing system (n = 100 dumbbells) on ten blocks and on every
    SM: the same trajectory up to the order of floating-point sums."""
    wl = inputs.dumbbell_workload(seed=3, kT=0.03, n_a=600, n_b=400, rcut=1.15)
    out = []
    for grid in (10, 0):
        s = make_gpu(wl, "fp64")
        s.set_grid(grid)
        s.run(400, 0.001, 0.03, 1.0)
        x, v, img = s.state()
        out.append((x + img * wl["box"], v, s.thermo()))
        s.close()
    (xa, va, ta), (xb, vb, tb) = out
    assert np.abs(xa - xb).max() <= 1e-9
    assert np.abs(va - vb).max() <= 1e-7
    assert ta["n_bonds"] == tb["n_bonds"]
    assert ta["U2"] == pytest.approx(tb["U2"], rel=1e-9, abs=1e-9)


def test_grid_change_between_runs(orc):
    wl = inputs.workload("mix2k", lambda3=1.0, n=2500, density=0.4, seed=6)
    a = make_gpu(wl, "fp64")
    a.run(60, 0.001, 0.1, 1.0)
    b = make_gpu(wl, "fp64")
    b.run(25, 0.001, 0.1, 1.0)
    b.set_grid(12)
    b.run(35, 0.001, 0.1, 1.0)
    xa, va, ia = a.state()
    xb, vb, ib = b.state()
    assert np.abs(_min_image(xa - xb, wl["box"])).max() <= 1e-10
    assert np.abs(va - vb).max() <= 1e-8
    assert a.thermo()["step"] == b.thermo()["step"] == 60


def test_negative_grid_is_rejected():
    from paper_1912_08569_gb300 import _abi as A

    wl = inputs.workload("mix2k", n=300, seed=1)
    s = make_gpu(wl, "fp32")
    with pytest.raises(A.SwpError):
        s.set_grid(-1)
