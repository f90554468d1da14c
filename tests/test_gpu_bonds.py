"""Harmonic bonds (the vitrimer network's chains) on the GPU path against the
oracle: forces, energies (the bond energy is reported inside U2), virial and
bond-swap counts of a small vitrimer network, and short trajectories, in
FP32 and FP64, with the tolerances of the pair-term tests.
"""
import numpy as np
import pytest

from gpu_helpers import TOL, assert_forces_match, make_gpu, oracle_pairs
from paper_1912_08569_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_08569_gb300.build import build

    build()


def _wl(n=5500, seed=2, kT=0.5):
    return inputs.vitrimer_workload(n, seed=seed, kT=kT)


def _gpu(wl, precision, **kw):
    s = make_gpu(wl, precision, **kw)
    s.set_bonds(wl["bonds"], wl["kbond"], wl["r0"])
    return s


def _oracle(orc, wl, x, fp32):
    return orc.forces(x, wl["types"], wl["n_types"], oracle_pairs(orc, wl), wl["box"], fp32=fp32,
                      bonds=wl["bonds"], kbond=wl["kbond"], r0=wl["r0"])


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_bonded_forces_match_oracle(orc, precision):
    wl = _wl()
    s = _gpu(wl, precision)
    s.compute_forces()
    ref = _oracle(orc, wl, wl["x"], precision == "fp32")
    assert ref["U_bond"] > 0.0
    F = s.forces()
    assert_forces_match(F, ref, TOL[precision], precision)
    th = s.thermo()
    tol = TOL[precision]
    assert abs(th["U2"] - (ref["U2"] + ref["U_bond"])) <= tol * (ref["scale_U2"] + ref["scale_Ub"])
    assert abs(th["U3"] - ref["U3"]) <= tol * ref["scale_U3"]
    assert np.all(np.abs(th["W"] - ref["W"]) <= tol * ref["scale_W"])
    assert th["n_bonds"] == ref["n_bonds"]


def test_vitrimer_full_size_forces_fp32(orc):
    """The 2M-bead network of the benchmark (box of 133 sigma) after a short
    run: every particle's force, the energies, virial and bond count against
    the oracle at the positions the run reached."""
    wl = inputs.vitrimer_workload(2_000_000, seed=1)
    assert wl["box"][0] > 128.0
    s = _gpu(wl, "fp32")
    s.run(200, wl["dt"], wl["kT"], wl["gamma"])
    s.compute_forces()
    x, _, _ = s.state()
    F = s.forces()
    th = s.thermo()
    ref = _oracle(orc, wl, x, True)
    assert_forces_match(F, ref, TOL["fp32"], "vitrimer2m")
    tol = TOL["fp32"]
    assert abs(th["U2"] - (ref["U2"] + ref["U_bond"])) <= tol * (ref["scale_U2"] + ref["scale_Ub"])
    assert abs(th["U3"] - ref["U3"]) <= tol * ref["scale_U3"]
    assert np.all(np.abs(th["W"] - ref["W"]) <= tol * ref["scale_W"])
    assert th["n_bonds"] == ref["n_bonds"]
    s.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_bonded_trajectory_matches_oracle(orc, precision):
    wl = _wl(n=2200, seed=3)
    dt, nsteps, kT = 0.001, 20, 0.5
    s = _gpu(wl, precision)
    s.run(nsteps, dt, kT, 1.0)
    x, v, img = s.state()
    xo, vo, imo, tho = orc.run(wl["x"], wl["v"], wl["types"], wl["mass"], wl["tags"], wl["n_types"],
                               oracle_pairs(orc, wl), wl["box"], dt, nsteps, kT=kT, gamma=1.0, seed=wl["seed"],
                               fp32=precision == "fp32", bonds=wl["bonds"], kbond=wl["kbond"], r0=wl["r0"])
    d = x - xo
    d -= wl["box"] * np.round(d / wl["box"])
    lim = {"fp32": (2e-6, 2e-4), "fp64": (1e-11, 1e-9)}[precision]
    assert np.abs(d).max() <= lim[0], np.abs(d).max()
    assert np.abs(v - vo).max() <= lim[1], np.abs(v - vo).max()
    assert np.array_equal(img, imo)


def test_bonds_survive_rebuilds_fp64(orc):
    """Hot and with a thin skin, the list is rebuilt (particles reordered) many
    times: the bonds must follow their tags."""
    wl = _wl(n=1100, seed=4, kT=1.0)
    wl["skin"] = 0.08
    dt, nsteps = 0.001, 150
    s = _gpu(wl, "fp64")
    s.run(nsteps, dt, 1.0, 1.0)
    assert s.thermo()["n_rebuilds"] >= 5
    x, v, img = s.state()
    xo, vo, imo, _ = orc.run(wl["x"], wl["v"], wl["types"], wl["mass"], wl["tags"], wl["n_types"],
                             oracle_pairs(orc, wl), wl["box"], dt, nsteps, kT=1.0, gamma=1.0, seed=wl["seed"],
                             bonds=wl["bonds"], kbond=wl["kbond"], r0=wl["r0"])
    d = x - xo
    d -= wl["box"] * np.round(d / wl["box"])
    assert np.abs(d).max() <= 1e-8, np.abs(d).max()


def test_set_bonds_rejects_bad_input():
    from paper_1912_08569_gb300 import _abi as A

    wl = _wl(n=1100)
    s = make_gpu(wl, "fp32")
    for bad in ([[0, 0]], [[0, 99999]], [[0, 1], [0, 1]], [[0, 1], [0, 2], [0, 3], [0, 4], [0, 5]]):
        with pytest.raises(A.SwpError):
            s.set_bonds(bad, 100.0, 1.0)
    s.set_bonds(np.zeros((0, 2), dtype=np.int32), 100.0, 1.0)  # no bonds: accepted
