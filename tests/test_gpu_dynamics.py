"""GPU time stepping vs the oracle's integrators (through the C-ABI).

Short trajectories are compared element by element with the oracle run from
the same seeded inputs (the Langevin noise is the same Philox4x32-10 stream on
both sides); longer runs are checked through properties that hold at any
size: energy conservation (NVE), equipartition (NVT), determinism.
"""
import numpy as np
import pytest

from gpu_helpers import TOL, make_gpu, oracle_pairs
from paper_1912_08569_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_08569_gb300.build import build

    build()


def _wl(n=2000, density=0.3, lam=1.0, shift=1, seed=2, kT=0.1):
    wl = inputs.workload("mix2k", lambda3=lam, n=n, density=density, seed=seed, shift=shift)
    wl["v"] = inputs.maxwell_velocities(n, kT, 1.0, seed=seed + 7)
    return wl


def _oracle_run(orc, wl, nsteps, dt, kT, gamma, fp32, seed):
    return orc.run(wl["x"], wl["v"], wl["types"], wl["mass"], wl["tags"], wl["n_types"],
                   oracle_pairs(orc, wl), wl["box"], dt, nsteps, kT=kT, gamma=gamma, seed=seed,
                   fp32=fp32)


def _min_image(d, box):
    return d - box * np.round(d / box)


# per-quantity trajectory tolerances after <= 20 steps (FP32: a few ulp of the
# positions amplified by 20 steps of the dynamics; FP64 likewise):
TRAJ = {"fp32": dict(x=2e-6, v=2e-4), "fp64": dict(x=1e-11, v=1e-9)}


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("gamma", [0.0, 1.0])
def test_short_trajectory_matches_oracle(orc, precision, gamma):
    wl = _wl()
    dt, kT, nsteps, seed = 0.001, 0.1, 20, 12345
    wl["seed"] = seed
    s = make_gpu(wl, precision)
    s.run(nsteps, dt, kT, gamma)
    x, v, img = s.state()
    th = s.thermo()
    xo, vo, imo, tho = _oracle_run(orc, wl, nsteps, dt, kT, gamma, precision == "fp32", seed)
    dx = np.abs(_min_image(x - xo, wl["box"]))
    assert dx.max() <= TRAJ[precision]["x"], dx.max()
    assert np.abs(v - vo).max() <= TRAJ[precision]["v"], np.abs(v - vo).max()
    unwrapped_gpu = x + img * wl["box"]
    unwrapped_orc = xo + imo * wl["box"]
    assert np.abs(unwrapped_gpu - unwrapped_orc).max() <= TRAJ[precision]["x"]
    assert th["step"] == nsteps
    # energies of the last step against the oracle's record of the same step
    ref = orc.forces(xo, wl["types"], 2, oracle_pairs(orc, wl), wl["box"], fp32=precision == "fp32")
    tol = max(TOL[precision], 1e3 * TRAJ[precision]["x"])
    assert abs(th["U2"] - tho[-1, 0]) <= tol * ref["scale_U2"]
    assert abs(th["U3"] - tho[-1, 1]) <= tol * ref["scale_U3"]
    assert th["K"] == pytest.approx(tho[-1, 2], rel=1e-4 if precision == "fp32" else 1e-10)


def test_trajectory_with_many_rebuilds_fp64(orc):
    # hot and with a thin skin: the list is rebuilt on the device many times
    wl = _wl(n=1500, density=0.3, kT=1.0)
    wl["skin"] = 0.08
    dt, kT, nsteps, seed = 0.001, 1.0, 300, 99
    s = make_gpu(wl, "fp64")
    s.run(nsteps, dt, kT, 1.0)
    x, v, img = s.state()
    th = s.thermo()
    assert th["n_rebuilds"] >= 5
    xo, vo, imo, _ = _oracle_run(orc, wl, nsteps, dt, kT, 1.0, False, wl["seed"])
    assert np.abs((x + img * wl["box"]) - (xo + imo * wl["box"])).max() <= 1e-8
    assert np.abs(v - vo).max() <= 1e-6


def test_runs_split_are_bit_identical():
    wl = _wl(n=3000, density=0.5, kT=0.2)
    a = make_gpu(wl, "fp32")
    a.run(200, 0.001, 0.2, 1.0)
    b = make_gpu(wl, "fp32")
    b.run(70, 0.001, 0.2, 1.0)
    b.run(130, 0.001, 0.2, 1.0)
    xa, va, ia = a.state()
    xb, vb, ib = b.state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(ia, ib)
    assert a.thermo()["U3"] == b.thermo()["U3"]


def test_nve_energy_conservation_fp32(orc):
    wl = _wl(n=2000, density=0.3, kT=0.1)
    dt, chunk, nchunks = 0.001, 50, 20
    s = make_gpu(wl, "fp32")
    E = []
    s.compute_forces()
    th = s.thermo()
    E.append(th["U2"] + th["U3"] + th["K"])
    for _ in range(nchunks):
        s.run(chunk, dt)
        th = s.thermo()
        E.append(th["U2"] + th["U3"] + th["K"])
    E = np.array(E)
    _, _, _, tho = _oracle_run(orc, wl, chunk * nchunks, dt, 0.0, 0.0, True, 0)
    Eo = tho[:, 0] + tho[:, 1] + tho[:, 2]
    gpu_dev = np.abs(E - E[0]).max()
    orc_dev = np.abs(Eo - E[0]).max()
    # the FP32 path conserves energy as well as the FP64 integrator does
    assert gpu_dev <= 2.0 * orc_dev + 1e-5 * wl["n"], (gpu_dev, orc_dev)


def test_nvt_equipartition():
    n = 4000
    box = inputs.cubic_box(n, 0.3)
    x = inputs.rsa_positions(n, box, 0.9, seed=21)
    wl = dict(n=n, n_types=2, box=box, x=x, types=np.zeros(n, dtype=np.int32), v=np.zeros((n, 3)),
              mass=np.ones(n), pairs=inputs.swap_pairs(), skin=0.3, seed=5)
    s = make_gpu(wl, "fp32")
    kT = 0.1
    s.run(1000, 0.002, kT, 1.0)
    Ks = []
    for _ in range(20):
        s.run(100, 0.002, kT, 1.0)
        Ks.append(s.thermo()["K"])
    assert np.mean(Ks) == pytest.approx(1.5 * n * kT, rel=0.02)


def test_list_stays_valid_over_a_long_run():
    # after 3000 steps with device-side rebuilds, every pair inside its cut-off
    # must still be in the list of both partners (checked on the read-back state)
    wl = _wl(n=5000, density=0.5, kT=0.3)
    s = make_gpu(wl, "fp32")
    s.run(3000, 0.001, 0.3, 1.0)
    x, _, _ = s.state()
    rows, counts = s.nlist()
    box = wl["box"]
    d = _min_image(x[:, None, :] - x[None, :, :], box)
    r2 = (d ** 2).sum(-1)
    cut = np.where(wl["types"][:, None] != wl["types"][None, :], 1.5, 2 ** (1 / 6))
    inside = (r2 < cut ** 2) & ~np.eye(len(x), dtype=bool)
    for i in range(len(x)):
        listed = set(rows[i, : counts[i, 1]].tolist())
        assert set(np.nonzero(inside[i])[0].tolist()) <= listed, i
    assert s.thermo()["n_rebuilds"] >= 2
