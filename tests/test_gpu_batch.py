"""Batched launches (many independent systems in one cooperative launch)
against the oracle, system by system.

Each system of a small uneven batch (different sizes, densities, lambda and
temperature) is advanced by the batched kernel and compared with the oracle's
run of the same system from the same seeded inputs, with the tolerances of
the single-system trajectory tests.  The work splits covered: every system
on blocks of its own (groups of several blocks, group barriers), every system
packed onto single blocks (block-local barriers, several systems per block),
and the balanced plan, whose blocks may run a group share and then whole
systems, with every block shape of the batched kernel (1024, 512, 384 and 256
threads per block in FP32, 1024 in FP64); a shape the precision lacks is
refused.
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


# (n, density, lambda, kT, seed): uneven sizes, one below a block's 1024 threads
SYSTEMS = [(300, 0.2, 0.0, 0.03, 11), (1500, 0.4, 1.0, 0.2, 12), (2600, 0.6, 5.0, 0.1, 13),
           (700, 0.3, 0.5, 0.05, 14), (4100, 0.5, 2.0, 0.12, 15)]
TRAJ = {"fp32": dict(x=2e-6, v=2e-4), "fp64": dict(x=1e-11, v=1e-9)}


def _wl(n, density, lam, kT, seed):
    wl = inputs.workload("mix2k", lambda3=lam, n=n, density=density, seed=seed, shift=0)
    wl["v"] = inputs.maxwell_velocities(n, kT, 1.0, seed=seed + 7)
    wl["seed"] = 1000 + seed
    return wl


def _min_image(d, box):
    return d - box * np.round(d / box)


def _assert_matches_oracle(orc, wl, s, kT, dt, nsteps, precision):
    fp32 = precision == "fp32"
    x, v, img = s.state()
    th = s.thermo()
    xo, vo, imo, tho = orc.run(wl["x"], wl["v"], wl["types"], wl["mass"], wl["tags"], wl["n_types"],
                               oracle_pairs(orc, wl), wl["box"], dt, nsteps, kT=kT, gamma=1.0,
                               seed=wl["seed"], fp32=fp32)
    assert th["step"] == nsteps
    dx = np.abs(_min_image(x - xo, wl["box"]))
    assert dx.max() <= TRAJ[precision]["x"], (wl["n"], dx.max())
    assert np.abs(v - vo).max() <= TRAJ[precision]["v"], (wl["n"], np.abs(v - vo).max())
    assert np.array_equal(img, imo)
    ref = orc.forces(xo, wl["types"], 2, oracle_pairs(orc, wl), wl["box"], fp32=fp32)
    tol = max(TOL[precision], 1e3 * TRAJ[precision]["x"])
    assert abs(th["U2"] - tho[-1, 0]) <= tol * ref["scale_U2"], wl["n"]
    assert abs(th["U3"] - tho[-1, 1]) <= tol * ref["scale_U3"], wl["n"]
    assert th["n_bonds"] == ref["n_bonds"], wl["n"]


@pytest.mark.parametrize("precision,threads", [("fp32", 1024), ("fp32", 512), ("fp32", 384), ("fp32", 256),
                                               ("fp64", 1024)])
@pytest.mark.parametrize("split", [0.0, 0.5, 1e9])
def test_batch_matches_oracle_per_system(orc, precision, threads, split):
    """Every block shape of the batched kernel, the balanced plan and both
    ends of the threshold plan."""
    from paper_1912_08569_gb300 import SwapBatch

    wls = [_wl(*p) for p in SYSTEMS]
    systems = [make_gpu(wl, precision) for wl in wls]
    kT = [p[3] for p in SYSTEMS]
    batch = SwapBatch(systems, split=split, threads=threads)
    dt, nsteps = 0.001, 20
    batch.run(nsteps, dt, kT, 1.0)
    for wl, s, t in zip(wls, systems, kT):
        _assert_matches_oracle(orc, wl, s, t, dt, nsteps, precision)


def test_balanced_plan_blocks_run_a_group_share_then_other_systems(orc):
    """80 systems of 150-3,000 particles on 256-thread blocks: the balanced
    plan gives some blocks a share of a multi-block group first and then whole
    systems; every system matches the oracle's run of it."""
    import torch

    from paper_1912_08569_gb300 import SwapBatch
    from paper_1912_08569_gb300 import _abi as A

    wls = inputs.batch_workload(80, seed=7, n_min=150, n_max=3000)
    nb = torch.cuda.get_device_properties(0).multi_processor_count
    ofs, items = A.swp_batch_plan([wl["n"] for wl in wls], nb, 0.0, 256, 256)
    mixed = [b for b in range(nb) if ofs[b + 1] - ofs[b] > 1 and items[ofs[b]][2] > 1]
    assert mixed, "the size mix should give some group member other systems"
    systems = [make_gpu(wl, "fp32") for wl in wls]
    batch = SwapBatch(systems, split=0.0, threads=256)
    dt, nsteps = 0.001, 20
    kT = [wl["kT"] for wl in wls]
    batch.run(nsteps, dt, kT, 1.0)
    for wl, s, t in zip(wls, systems, kT):
        _assert_matches_oracle(orc, wl, s, t, dt, nsteps, "fp32")


def test_batch_group_timeout_leaves_the_other_systems_running(orc):
    """Failure detection without a fault, batched: the first group barrier of a
    system on several blocks is withheld, its blocks' waits run out after 1 ms,
    and those blocks go on with the whole systems the balanced plan gave them.
    That system alone reports SWP_ERR_TIMEOUT; every other system matches the
    oracle's run of it."""
    import torch

    from paper_1912_08569_gb300 import SwapBatch
    from paper_1912_08569_gb300 import _abi as A

    wls = inputs.batch_workload(80, seed=7, n_min=150, n_max=3000)
    nb = torch.cuda.get_device_properties(0).multi_processor_count
    ofs, items = A.swp_batch_plan([wl["n"] for wl in wls], nb, 0.0, 256, 256)
    mixed = [b for b in range(nb) if ofs[b + 1] - ofs[b] > 1 and items[ofs[b]][2] > 1]
    assert mixed
    bad = int(items[ofs[mixed[0]]][0])  # a group system whose member block has other systems
    after = [int(it[0]) for it in items[ofs[mixed[0]] + 1:ofs[mixed[0] + 1]]]
    systems = [make_gpu(wl, "fp32") for wl in wls]
    systems[bad].set_timeout(1_000_000)
    A.swp_set_withhold_arrival(systems[bad].ctx, 1)
    batch = SwapBatch(systems, split=0.0, threads=256)
    dt, nsteps = 0.001, 20
    kT = [wl["kT"] for wl in wls]
    batch.run(nsteps, dt, kT, 1.0, sync=False)
    with pytest.raises(A.SwpError) as e:
        A.swp_sync(systems[bad].ctx)
    assert e.value.code == A.SWP_ERR_TIMEOUT, str(e.value)
    torch.cuda.synchronize()  # nothing is left running
    assert after, "the member block runs other systems after its group share"
    for r, (wl, s, t) in enumerate(zip(wls, systems, kT)):
        if r != bad:
            _assert_matches_oracle(orc, wl, s, t, dt, nsteps, "fp32")


def test_batch_equals_single_runs_in_forces(orc):
    """After a batched run, each system's forces at its new positions agree with
    a fresh single-system evaluation of the same positions."""
    from paper_1912_08569_gb300 import SwapBatch

    wls = [_wl(*p) for p in SYSTEMS[:3]]
    systems = [make_gpu(wl, "fp32") for wl in wls]
    SwapBatch(systems, split=1e9).run(50, 0.001, [p[3] for p in SYSTEMS[:3]], 1.0)
    for wl, s in zip(wls, systems):
        s.compute_forces()
        x, _, _ = s.state()
        F = s.forces()
        ref = orc.forces(x, wl["types"], 2, oracle_pairs(orc, wl), wl["box"], fp32=True)
        err = np.linalg.norm(F - ref["F"], axis=1)
        assert np.all(err <= TOL["fp32"] * ref["fscale"])


def test_batch_overflow_recovers(orc):
    """A system whose list overflows inside the batch is finished alone; the
    others are unaffected."""
    from paper_1912_08569_gb300 import SwapBatch

    wls = [_wl(*p) for p in SYSTEMS[:3]]
    systems = [make_gpu(wl, "fp32") for wl in wls]
    systems[1] = make_gpu(wls[1], "fp32", max_nn=2)  # rows cannot fit
    SwapBatch(systems, split=1e9).run(20, 0.001, 0.1, 1.0)
    for wl, s in zip(wls, systems):
        th = s.thermo()
        assert th["step"] == 20
    assert systems[1].grows >= 1


def test_batch_rejects_mixed_precision():
    from paper_1912_08569_gb300 import SwapBatch

    wls = [_wl(*p) for p in SYSTEMS[:2]]
    with pytest.raises(ValueError):
        SwapBatch([make_gpu(wls[0], "fp32"), make_gpu(wls[1], "fp64")])


def test_batch_rejects_missing_block_shape():
    from paper_1912_08569_gb300 import SwapBatch
    from paper_1912_08569_gb300 import _abi as A

    systems = [make_gpu(_wl(*p), "fp64") for p in SYSTEMS[:2]]
    for threads in (512, 300):
        with pytest.raises(A.SwpError) as e:
            SwapBatch(systems, threads=threads).run(1, 0.001, 0.1, 1.0)
        assert e.value.code == A.SWP_ERR_INVALID
