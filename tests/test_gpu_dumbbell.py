"""The paper's own model on the GPU path against the oracle: the dumbbell
mixture of section "Effect of swaps" (600 A + 400 B at density 0.125, A-B swap
pair with exponent n = 100, lambda = 1; A-A and B-B WCA), at the two cut-offs
of the Supplementary's performance runs (r_c = 1.3 and 1.15).

n = 100 takes paths the n = 10 mixture never reaches: (sigma/r)^n by the
general repeated-squaring loop (n/2 = 50), and an extremely stiff bond (the
curvature of Eq. 2b at r_min is about 2 n^2 eps / r_min^2).  Checked element by
element: forces, energies, virial and bond count at the start and after 2,000
BAOAB steps of the GPU dynamics (FP32 and FP64), and a 50-step BAOAB trajectory
against the oracle's integrator from the same inputs (same Philox noise).
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


def _dumbbell(rcut, seed=5, kT=0.03):
    wl = inputs.dumbbell_workload(seed=seed, kT=kT, rcut=rcut)
    wl["seed"] = 4242
    return wl


def _min_image(d, box):
    return d - box * np.round(d / box)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("rcut", [1.3, 1.15])
def test_dumbbell_forces_match_oracle(orc, precision, rcut):
    wl = _dumbbell(rcut)
    s = make_gpu(wl, precision)
    s.compute_forces()
    tab = oracle_pairs(orc, wl)
    ref = orc.forces(wl["x"], wl["types"], 2, tab, wl["box"], fp32=precision == "fp32")
    assert ref["n_bonds"] >= 400  # every B starts bonded to its own A (a few also to a neighbour's)
    assert_forces_match(s.forces(), ref, TOL[precision], f"dumbbell start r_c={rcut}")
    assert_thermo_match(s.thermo(), ref, TOL[precision], f"dumbbell start r_c={rcut}")
    # after the dynamics has explored the bond wells (thermal approaches inside r_min)
    s.run(2000, wl["dt"], wl["kT"], wl["gamma"])
    x, _, _ = s.state()
    ref = orc.forces(x, wl["types"], 2, tab, wl["box"], fp32=precision == "fp32")
    assert_forces_match(s.forces(), ref, TOL[precision], f"dumbbell after 2000 steps r_c={rcut}")
    assert_thermo_match(s.thermo(), ref, TOL[precision], f"dumbbell after 2000 steps r_c={rcut}")
    s.close()


# 50 steps of the stiff n = 100 bond (about 1.5 oscillation periods): FP32 a
# few quanta of the 32-bit box-fraction positions and the FP32 force rounding
# carried through the oscillation; FP64 likewise at its own precision
TRAJ = {"fp32": dict(x=2e-6, v=2e-4), "fp64": dict(x=1e-10, v=1e-8)}


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("rcut", [1.3, 1.15])
def test_dumbbell_trajectory_matches_oracle(orc, precision, rcut):
    wl = _dumbbell(rcut, seed=9)
    nsteps = 50
    s = make_gpu(wl, precision)
    s.run(nsteps, wl["dt"], wl["kT"], wl["gamma"])
    x, v, img = s.state()
    th = s.thermo()
    xo, vo, imo, tho = orc.run(wl["x"], wl["v"], wl["types"], wl["mass"], wl["tags"], 2, oracle_pairs(orc, wl),
                               wl["box"], wl["dt"], nsteps, kT=wl["kT"], gamma=wl["gamma"], seed=wl["seed"],
                               fp32=precision == "fp32")
    dx = np.abs((x + img * wl["box"]) - (xo + imo * wl["box"])).max()
    dv = np.abs(v - vo).max()
    assert dx <= TRAJ[precision]["x"], dx
    assert dv <= TRAJ[precision]["v"], dv
    ref = orc.forces(xo, wl["types"], 2, oracle_pairs(orc, wl), wl["box"], fp32=precision == "fp32")
    tol = max(TOL[precision], 1e3 * TRAJ[precision]["x"])
    assert abs(th["U2"] - tho[-1, 0]) <= tol * ref["scale_U2"]
    assert abs(th["U3"] - tho[-1, 1]) <= tol * ref["scale_U3"]
    assert th["n_bonds"] == int(tho[-1, 9])
    s.close()
