#!/usr/bin/env python3
"""Benchmark: swap-potential particle-timesteps/s on one GB300 (FP32 path).

Workload (synthetic, seeded; the paper has no public dataset): 100,000
particles, A:B 1:1 alternating by tag, density 0.5, RSA positions with minimum
separation 0.9, A-B swap pair (eps = sigma = 1, n = 10, r_cut = 1.5, lambda 1
by default), A-A and B-B WCA (sigma = 1), BAOAB Langevin at kT = 0.05,
gamma = 1, dt = 0.001, skin 0.3, list rebuilt on the device on displacement.
One benchmark step = one launch of the persistent step kernel advancing
``--md-steps`` (default 1,000) time steps, with the energies, virial, kinetic
energy and bond count of every ``--thermo-every`` th step (default: every
step) written to the device thermo log and reduced into per-step records
after the launch; the inputs stay resident in HBM, and L2 is flushed (a
512 MB write) between timed launches.

Other workloads (``--workload``): batch256 (256 independent systems in one
launch), diff20k (force-matching gradient), vitrimer2m (2M-bead bonded
network), dumbbell (the paper's timing system at ``--particles`` and
``--rcut``).

Each rank (torchrun, one GPU each) runs its own independent replica: weak
scaling, no collective on the data path.  ``--impl reference`` times the FP64
CPU oracle on the same workload (bounded samples) instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "swap-potential particle-timesteps/s at 100k (FP32); % of HBM roofline"
UNIT = "particle-timesteps/s"
# swp_read_thermo copies the device control block (192 bytes) to the host.
CTL_BYTES = 192


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--lam", type=float, default=1.0)
    ap.add_argument("--md-steps", type=int, default=None,
                    help="time steps per launch (default 1000; 5000 for batch256)")
    ap.add_argument("--particles", "--n", dest="n", type=int, default=None,
                    help="particles (default 100,000; 16,384 for dumbbell)")
    ap.add_argument("--rcut", type=float, default=1.3, help="A-B cut-off of the dumbbell workload")
    ap.add_argument("--grid", type=int, default=0, help="step-kernel blocks (0: every SM)")
    ap.add_argument("--bps", type=int, default=0)
    ap.add_argument("--no-resident", action="store_true",
                    help="forbid the resident mode (one barrier per step): the two-barrier step")
    ap.add_argument("--thermo-every", type=int, default=1,
                    help="thermo-log interval of the mix100k workload in steps (0: only each launch's last step)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--workload", default="mix100k",
                    choices=["mix100k", "batch256", "diff20k", "vitrimer2m", "dumbbell"],
                    help="mix100k: the single 100k-particle system (default); batch256: 256 "
                         "independent systems of 1k-32k particles in one launch per step; diff20k: "
                         "force-matching gradient over 64 snapshots of 20k particles; vitrimer2m: "
                         "2M-bead bonded network with swapping crosslinkers; dumbbell: the paper's "
                         "timing system (dumbbell mixture, n=100) at --particles and --rcut")
    ap.add_argument("--snapshots", type=int, default=64)
    ap.add_argument("--systems", type=int, default=256)
    return ap.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value, device):
    """The largest value over the ranks of the default process group (the
    value itself without one): timed regions are reported as the slowest rank's."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_rank, steps_per_launch, launches, total_ms):
    """Whole-job rate: every rank's units times steps over the slowest rank's time."""
    return world * units_per_rank * steps_per_launch * launches / (total_ms / 1e3)


def _workload(n, lam, rank):
    from paper_1912_08569_gb300 import inputs

    return inputs.workload("mix100k", lambda3=lam, n=n, seed=1 + rank)


def _dumbbell(n, rcut, rank):
    """The paper's timing system: n particles, A:B = 3:2 as in the 600 + 400
    dumbbell mixture, every B bonded to an A at the start, density 0.125, A-B
    swap pair n=100 with cut-off rcut (1.3 or 1.15), BAOAB kT=0.03."""
    from paper_1912_08569_gb300 import inputs

    na = (3 * n) // 5
    return inputs.dumbbell_workload(seed=1 + rank, kT=0.03, n_a=na, n_b=n - na, rcut=rcut)


def _config(a, n, world):
    return {"workload": f"mix{n // 1000}k: N={n}, A:B 1:1, density 0.5, n=10, r_cut=1.5, "
                        f"lambda={a.lam:g}, BAOAB kT=0.05 gamma=1 dt=0.001, skin 0.3",
            "n_particles": n, "md_steps_per_step": a.md_steps, "lambda": a.lam,
            "replicas": world, "l2": "flushed (512 MB write) between timed launches",
            "thermo": (f"energies, virial, kinetic energy and bond count of every {a.thermo_every} step(s), "
                       "logged on the device and reduced per step after each launch (in the timed region)"
                       if a.thermo_every > 0 else "energies and virial of each launch's last step only"),
            "parallelism": f"replicas x{world}"}


# ---------------------------------------------------------------------------
# clocks sampled during the timed region

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [s.strip() for s in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if p[5 + k].lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        load = [s for s in sm if s > 0.5 * max(sm)]
        return {"sm_mhz": float(np.median(load)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# roofline bookkeeping

def _kernel_digest():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1912_08569_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def host_info():
    """The host the CPU baseline ran on: logical cores and CPU model."""
    model, arm = None, {}
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if ":" not in line:
                    continue
                key, val = (t.strip() for t in line.split(":", 1))
                if key.lower() in ("model name", "cpu model") and model is None:
                    model = val
                elif key in ("CPU implementer", "CPU part") and key not in arm:
                    arm[key] = val  # Arm cores name themselves by these codes
    except OSError:
        pass
    if model is None and arm:
        model = ", ".join(f"{k} {v}" for k, v in arm.items())
    import platform

    return {"nproc": os.cpu_count(), "machine": platform.machine(), "cpu": model}


def _profile_traffic(n, md_steps):
    """DRAM bytes of one step-kernel launch (dram__bytes_read.sum +
    dram__bytes_write.sum) from the committed ncu record, if it was taken on
    the current kernel sources and on this launch size (else None)."""
    p = os.path.join(ROOT, "profiles", "k_run_traffic.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
    except Exception:
        return None
    if d.get("kernel_digest") != _kernel_digest():
        return None
    if d.get("n") != n or d.get("md_steps") != md_steps:
        return None
    return d.get("dram_bytes_per_launch")


def algorithmic_bytes(n, md_steps, nn, nn_r, rebuilds):
    """Bytes one launch must move (each array read or written once per pass
    that needs it): per particle-step 16 (position, S pass) + 16 (position,
    force pass) + 16 (new position) + 48 (fixed-point position read+write) +
    32 (velocity read+write) + 16 (force) + 8 (S write+read) + 8 (row counts)
    + 4 (nn + nn_r) (list indices); per particle and rebuild 120 (sort) +
    4 nn (list write)."""
    per_step = 160.0 + 4.0 * (nn + nn_r)
    per_rebuild = 120.0 + 4.0 * nn
    return n * (md_steps * per_step + rebuilds * per_rebuild)


# ---------------------------------------------------------------------------

def cpu_oracle_sample(wl, seconds, steps_cap=200, threaded=False):
    """Times the FP64 oracle on the same workload for a bounded number of steps
    (threaded: its OpenMP build on every host core)."""
    import oracle

    tab = oracle.pair_table(wl["n_types"], wl["pairs"])
    t0 = time.perf_counter()
    oracle.forces(wl["x"], wl["types"], wl["n_types"], tab, wl["box"], fp32=True, threaded=threaded)
    t_force = time.perf_counter() - t0
    nsteps = int(max(2, min(steps_cap, seconds / max(t_force, 1e-6))))
    t0 = time.perf_counter()
    oracle.run(wl["x"], wl["v"], wl["types"], wl["mass"], wl["tags"], wl["n_types"], tab, wl["box"],
               wl["dt"], nsteps, kT=wl["kT"], gamma=wl["gamma"], seed=wl["seed"], fp32=True, threaded=threaded)
    el = time.perf_counter() - t0
    return wl["n"] * nsteps / el, nsteps, el


def cpu_baseline(wl, seconds, n_label):
    """The oracle on the host: on every core (its OpenMP build; the headline
    figure) and on one thread, each a bounded sample of the workload."""
    import oracle

    oracle.build()
    v1, s1, e1 = cpu_oracle_sample(wl, seconds)
    one = {"value": v1, "cores": 1,
           "sample": f"N={n_label}, {s1} BAOAB steps of the FP64 C oracle (explicit triplet loop, cell list "
                     f"every step), {e1:.1f} s, 1 thread"}
    try:
        oracle.build(openmp=True)
        nt = oracle.threads(True)
        vN, sN, eN = cpu_oracle_sample(wl, seconds, threaded=True)
    except Exception as e:  # no OpenMP runtime on this host: the one-thread figure is the baseline
        return dict(one, unit=UNIT, kind="oracle", host=host_info(), all_cores=f"unavailable: {e}")
    return {"value": vN, "unit": UNIT, "cores": nt, "kind": "oracle", "host": host_info(),
            "sample": f"N={n_label}, {sN} BAOAB steps of the FP64 C oracle built with OpenMP ({nt} threads: "
                      f"pair search, pair and triplet sums split over the threads), {eN:.1f} s",
            "one_thread": one}


def accuracy_vs_oracle(oracle, s, wl):
    """Error of the GPU's forces and thermo record on a snapshot of the run
    against the FP64 oracle at the same positions (FP32 decisions), per
    quantity, relative to the oracle's error scales."""
    s.compute_forces()
    x, _, _ = s.state()
    F = s.forces()
    th = s.thermo()
    ref = oracle.forces(x, wl["types"], wl["n_types"], oracle.pair_table(wl["n_types"], wl["pairs"]), wl["box"],
                        fp32=True)
    derr = np.linalg.norm(F - ref["F"], axis=1)
    ferr = derr / np.maximum(ref["fscale"], 1e-300)
    # the survey's per-particle scale (forces times their three-body factor),
    # over the particles where it is not zero
    c9 = oracle.fscale_c9(x, wl["types"], wl["n_types"], oracle.pair_table(wl["n_types"], wl["pairs"]), wl["box"],
                          fp32=True)
    on = c9 > 0
    c9err = derr[on] / c9[on]
    return {"F_max_err_over_scale": float(ferr.max()),
            "F_rel_l2": float(np.linalg.norm(F - ref["F"]) / np.linalg.norm(ref["F"])),
            "F_max_err_over_c9_scale": float(c9err.max()) if c9err.size else 0.0,
            "F_p999_err_over_c9_scale": float(np.percentile(c9err, 99.9)) if c9err.size else 0.0,
            "U2_err_over_scale": abs(th["U2"] - ref["U2"]) / ref["scale_U2"],
            "U3_err_over_scale": abs(th["U3"] - ref["U3"]) / max(ref["scale_U3"], 1e-300),
            "W_max_err_over_scale": float(np.max(np.abs(th["W"] - ref["W"]))) / ref["scale_W"],
            "n_bonds_diff": int(th["n_bonds"] - ref["n_bonds"]), "tolerance": 1e-5}


def run_reference(a):
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    if a.workload == "dumbbell":
        return run_reference_dumbbell(a, oracle)
    wl = _workload(a.n, a.lam, 0)
    tab = oracle.pair_table(wl["n_types"], wl["pairs"])
    # on every host core (the oracle's OpenMP build), else on one thread
    try:
        oracle.build(openmp=True)
        threaded, cores = True, oracle.threads(True)
    except Exception:
        threaded, cores = False, 1
    t0 = time.perf_counter()
    oracle.forces(wl["x"], wl["types"], wl["n_types"], tab, wl["box"], fp32=True, threaded=threaded)
    t_force = time.perf_counter() - t0
    # each step: a bounded sample of the workload (~8 s of CPU work)
    per = int(max(1, min(50, 8.0 / max(t_force, 1e-6))))
    x, v = wl["x"], wl["v"]
    times = []
    for k in range(a.warmup + a.steps):
        t0 = time.perf_counter()
        x, v, _, th = oracle.run(x, v, wl["types"], wl["mass"], wl["tags"], wl["n_types"], tab,
                                 wl["box"], wl["dt"], per, kT=wl["kT"], gamma=wl["gamma"],
                                 seed=wl["seed"], step0=k * per, fp32=True, threaded=threaded)
        if k >= a.warmup:
            times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(times))
    value = wl["n"] * per / (ms / 1e3)
    sample = f"N={wl['n']}, {per} NVT steps per step of the FP64 C oracle ({cores} threads)"
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": _config(a, wl["n"], 1),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                            "host": host_info()},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def run_ours(a):
    import torch
    import torch.distributed as dist

    rank, world, local = _dist()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    from paper_1912_08569_gb300 import SwapSystem
    from paper_1912_08569_gb300 import _abi as A
    from paper_1912_08569_gb300.build import build

    if rank == 0 or world == 1:
        build()
    if world > 1:
        dist.barrier()
    wl = _workload(a.n, a.lam, rank)
    n = wl["n"]
    s = SwapSystem(n, 2, wl["box"], wl["pairs"], precision="fp32", seed=wl["seed"], skin=wl["skin"],
                   blocks_per_sm=a.bps)
    s.set_state(wl["x"], wl["v"], wl["types"], wl["mass"])
    if a.grid:
        s.set_grid(a.grid)
    if a.no_resident:
        s.set_resident(False)
    s.compute_forces()
    _, counts = s.nlist()
    nn = float(counts[:, 1].mean())
    nn_r = float(counts[:, 0].mean())
    stream = s.stream
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    dt, kT, gamma = wl["dt"], wl["kT"], wl["gamma"]
    # the thermo log: one record per thermo_every steps of a launch
    log_cap = a.md_steps // a.thermo_every if a.thermo_every > 0 else 0
    if log_cap > 0:
        s.set_thermo_log(a.thermo_every, log_cap)
        log_rec = torch.empty((log_cap, 10), dtype=torch.float64, device=dev)
        log_stp = torch.empty(log_cap, dtype=torch.int64, device=dev)

    # warm-up (grows the list if a rebuild overflows)
    for _ in range(a.warmup):
        s.run(a.md_steps, dt, kT, gamma, sync=True)
    th0 = s.thermo()

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()
        time.sleep(0.3)
    evs = []
    t_wall = time.perf_counter()
    with torch.cuda.stream(stream):
        for _ in range(a.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e2 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.run(a.md_steps, dt, kT, gamma, sync=False)
            e1.record(stream)
            if log_cap > 0:  # the launch's per-step records (waits for the launch, then one reduction kernel)
                got = A.swp_thermo_log(s.ctx, log_rec, log_stp, log_cap)
                assert got == log_cap, (got, log_cap)
            e2.record(stream)
            evs.append((e0, e1, e2))
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    s.sync()  # raises if the device reported an error during the timed launches
    th1 = s.thermo()
    if world > 1:
        dist.barrier()
    clk = clocks.stop() if clocks else None
    launch_ms = [e0.elapsed_time(e1) for e0, e1, _ in evs]  # the step kernel alone (roofline)
    total_ms = float(np.sum([e0.elapsed_time(e2) for e0, _, e2 in evs]))  # with the log's reduction
    assert th1["step"] - th0["step"] == a.steps * a.md_steps, "timed launches did not complete"
    rebuilds = (th1["n_rebuilds"] - th0["n_rebuilds"]) / a.steps
    total_ms = max_over_ranks(total_ms, dev)
    ms_per_step = total_ms / a.steps
    value = job_throughput(world, n, a.md_steps, a.steps, total_ms)

    # roofline of the persistent step kernel (the only kernel in the timed region)
    peak, peak_kind = _peaks()
    b_alg = algorithmic_bytes(n, a.md_steps, nn, nn_r, rebuilds)
    achieved = b_alg / (float(np.mean(launch_ms)) / 1e3) / 1e9
    if log_cap > 0:  # the last launch's records: its steps, finite energies
        steps_logged = log_stp.cpu().numpy()
        assert np.array_equal(steps_logged, th1["step"] - a.md_steps + a.thermo_every * np.arange(1, log_cap + 1))
        assert np.all(np.isfinite(log_rec.cpu().numpy()))
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": _profile_traffic(n, a.md_steps),
            "peak_kind": peak_kind, "alg_bytes_per_launch": b_alg,
            "nn_mean": nn, "nn_reactive_mean": nn_r, "rebuilds_per_launch": rebuilds}

    # end to end through the C-ABI with host buffers: pinned state in, run,
    # thermo record out, every step.  The state uploaded is the equilibrated
    # one the timed launches ended in (read back once, before this timing), so
    # that each step does the same work as a timed launch; the upload itself
    # rebuilds the list and recomputes the forces every step.
    e2e = None
    if not a.no_e2e:
        x_eq, v_eq, img_eq = s.state()
        xh = torch.from_numpy(np.ascontiguousarray(x_eq)).pin_memory()
        vh = torch.from_numpy(np.ascontiguousarray(v_eq)).pin_memory()
        th_ = torch.from_numpy(np.ascontiguousarray(wl["types"], dtype=np.int32)).pin_memory()
        mh = torch.from_numpy(np.ascontiguousarray(wl["mass"])).pin_memory()
        ih = torch.from_numpy(np.ascontiguousarray(img_eq, dtype=np.int32)).pin_memory()
        h2d = xh.numel() * 8 + vh.numel() * 8 + th_.numel() * 4 + mh.numel() * 8 + ih.numel() * 4
        ctx = s.ctx
        times = []
        d2h = CTL_BYTES
        if log_cap > 0:
            log_host = torch.empty((log_cap, 10), dtype=torch.float64).pin_memory()
            d2h += log_host.numel() * 8
        for k in range(a.warmup + a.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            A.swp_set_state(ctx, xh, vh, th_, mh, ih, A.SWP_HOST)
            A.swp_step_nvt(ctx, dt, kT, gamma, a.md_steps)
            if log_cap > 0:  # every logged step's record to the host
                A.swp_thermo_log(ctx, log_rec, log_stp, log_cap)
                log_host.copy_(log_rec)
            rec = A.swp_read_thermo(ctx)
            el = time.perf_counter() - t0
            if k >= a.warmup:
                times.append(el)
        e2e_ms = 1e3 * max_over_ranks(float(np.sum(times)), dev)
        e2e = {"value": job_throughput(world, n, a.md_steps, a.steps, e2e_ms), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "last_U": float(rec.U2 + rec.U3)}

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        import oracle

        oracle.build()
        cpu = cpu_baseline(wl, a.cpu_seconds, n)
        cpu["accuracy"] = accuracy_vs_oracle(oracle, s, wl)

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
               "warmup": a.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": _config(a, n, world), "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
               "gpu_launches": a.steps * (2 if log_cap > 0 else 1), "clocks": clk, "wall_s_timed": t_wall,
               "kernel_digest": _kernel_digest(),
               "resident_steps_last_launch": th1["resident_steps"],
               "thermo_last": {"U2": th1["U2"], "U3": th1["U3"], "K": th1["K"],
                               "n_bonds": th1["n_bonds"]}}
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    s.close()
    return 0


BATCH_METRIC = "batched swap-potential particle-timesteps/s (independent systems, one launch)"


def run_batch(a):
    """Batched form: a.systems independent systems (sizes log-uniform 1k-32k,
    density 0.2-0.6, lambda in {0, 0.5, 1, 2, 5}, kT in [0.03, 0.2]) advanced
    a.md_steps steps per launch; one bench step = one launch."""
    import torch

    from paper_1912_08569_gb300 import SwapBatch, SwapSystem
    from paper_1912_08569_gb300 import _abi as A
    from paper_1912_08569_gb300 import inputs
    from paper_1912_08569_gb300.build import build

    rank, world, local = _dist()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    if rank == 0 or world == 1:
        build()
    if world > 1:
        dist.barrier()
    wls = inputs.batch_workload(a.systems, seed=7 + rank)
    systems = []
    for wl in wls:
        s = SwapSystem(wl["n"], 2, wl["box"], wl["pairs"], precision="fp32", seed=wl["seed"], skin=wl["skin"])
        s.set_state(wl["x"], wl["v"], wl["types"], wl["mass"])
        systems.append(s)
    kT = [wl["kT"] for wl in wls]
    dt, gamma = 0.001, 1.0
    batch = SwapBatch(systems)
    for s in systems:
        s.compute_forces()
    nn = np.array([float(s.nlist()[1][:, 1].mean()) for s in systems])
    nn_r = np.array([float(s.nlist()[1][:, 0].mean()) for s in systems])
    ns = np.array([wl["n"] for wl in wls], dtype=np.float64)
    tune = batch.autotune(200, dt, kT, gamma)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    for _ in range(a.warmup):
        batch.run(a.md_steps, dt, kT, gamma)
    reb0 = np.array([s.thermo()["n_rebuilds"] for s in systems])
    stream = systems[0].stream
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()
        time.sleep(0.3)
    evs = []
    with torch.cuda.stream(stream):
        for _ in range(a.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            batch.run(a.md_steps, dt, kT, gamma, sync=False)
            e1.record(stream)
            evs.append((e0, e1))
    torch.cuda.synchronize()
    batch.sync()
    clk = clocks.stop() if clocks else None
    launch_ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    total_ms = max_over_ranks(float(np.sum(launch_ms)), dev)
    n_total = float(ns.sum())
    value = job_throughput(world, n_total, a.md_steps, a.steps, total_ms)
    reb = (np.array([s.thermo()["n_rebuilds"] for s in systems]) - reb0) / a.steps
    peak, peak_kind = _peaks()
    b_alg = float(np.sum([algorithmic_bytes(n, a.md_steps, x, y, r) for n, x, y, r in zip(ns, nn, nn_r, reb)]))
    achieved = b_alg / (float(np.mean(launch_ms)) / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": None, "peak_kind": peak_kind, "alg_bytes_per_launch": b_alg}
    e2e = None
    if not a.no_e2e:
        # the equilibrated states the timed launches ended in (see run_ours)
        pins = []
        for s, wl in zip(systems, wls):
            x_eq, v_eq, img_eq = s.state()
            pins.append((torch.from_numpy(np.ascontiguousarray(x_eq)).pin_memory(),
                         torch.from_numpy(np.ascontiguousarray(v_eq)).pin_memory(),
                         torch.from_numpy(np.ascontiguousarray(wl["types"], dtype=np.int32)).pin_memory(),
                         torch.from_numpy(np.ascontiguousarray(wl["mass"])).pin_memory(),
                         torch.from_numpy(np.ascontiguousarray(img_eq, dtype=np.int32)).pin_memory()))
        h2d = int(sum(x.numel() * 8 + v.numel() * 8 + ty.numel() * 4 + m.numel() * 8 + im.numel() * 4
                      for x, v, ty, m, im in pins))
        times = []
        for k in range(a.warmup + a.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for s, (x, v, ty, m, im) in zip(systems, pins):
                A.swp_set_state(s.ctx, x, v, ty, m, im, A.SWP_HOST)
            batch.run(a.md_steps, dt, kT, gamma, sync=False)
            for s in systems:
                A.swp_read_thermo(s.ctx)
            if k >= a.warmup:
                times.append(time.perf_counter() - t0)
        e2e_ms = 1e3 * max_over_ranks(float(np.sum(times)), dev)
        e2e = {"value": job_throughput(world, n_total, a.md_steps, a.steps, e2e_ms), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": CTL_BYTES * len(systems)}
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        import oracle

        oracle.build()
        k = int(np.argsort(ns)[len(ns) // 2])  # the median-size system
        v, steps_done, el = cpu_oracle_sample(wls[k], a.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_info(),
               "sample": f"system {k} (N={int(ns[k])}), {steps_done} BAOAB steps of the FP64 C oracle, "
                         f"{el:.1f} s, 1 thread"}
    if rank == 0:
        out = {"metric": BATCH_METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
               "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": f"batch{len(wls)}: {len(wls)} systems, N log-uniform 1k-32k "
                                      f"(total {int(n_total)}), density 0.2-0.6, lambda in {{0,0.5,1,2,5}}, "
                                      f"kT 0.03-0.2, BAOAB gamma=1 dt=0.001, skin 0.3",
                          "systems": len(wls), "particles": int(n_total), "md_steps_per_step": a.md_steps,
                          "split": tune[1], "block_threads": tune[2],
                          "autotune_ms_per_200_steps": {f"{th}x{sp:g}": round(ms, 3) for th, sp, ms in tune[3]},
                          "l2": "flushed (512 MB write) between timed launches",
                          "parallelism": f"replicas x{world}"},
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": a.steps, "clocks": clk,
               "kernel_digest": _kernel_digest()}
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


DIFF_METRIC = "force-matching gradient particle-evaluations/s (energy, forces, dU and dF by theta; 20k)"


def run_diff(a):
    """Differentiable form: one bench step = the gradient of a force-matching
    loss (mean squared force error over a.snapshots snapshots of 20,000
    particles, density 0.4) with respect to the reactive pair's (lambda, eps,
    sigma), through autodiff.energy and a double backward.  The reference
    forces are this library's own at theta_ref = (1, 1, 1) (a synthetic
    target; accuracy against the oracle is covered by the tests)."""
    import torch

    from paper_1912_08569_gb300 import SwapSystem, autodiff, inputs
    from paper_1912_08569_gb300.build import build

    rank, world, local = _dist()
    if world > 1 and rank != 0:
        return 0  # one GPU: the differentiable form runs on rank 0 only
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    build()
    snaps = [inputs.workload("mix100k", n=20000, density=0.4, seed=100 + k) for k in range(a.snapshots)]
    wl = snaps[0]
    s = SwapSystem(wl["n"], 2, wl["box"], wl["pairs"], precision="fp32", seed=wl["seed"], skin=wl["skin"])
    for w in snaps:  # size the list buffer for the densest snapshot (the evaluations do not read back)
        s.set_state(w["x"], None, w["types"])
        s.compute_forces()
    model = autodiff.SwapModel(s, wl["pairs"], wl["types"])
    xs = [torch.tensor(w["x"], dtype=torch.float64, device=dev) for w in snaps]
    theta_ref = torch.tensor([1.0, 1.0, 1.0], dtype=torch.float64, device=dev)
    with torch.no_grad():
        refs = [autodiff.forces(model, x, theta_ref).detach() for x in xs]
    theta0 = [1.3, 0.9, 1.02]

    # force matching over the snapshots as one batch (autodiff.energy_batch):
    # the energies' sum is differentiated with respect to every snapshot's
    # positions at once (the snapshots are independent, so each gradient is
    # that snapshot's -F), then the loss is back-propagated to theta through
    # the forces
    X = torch.stack(xs).requires_grad_(True)
    R = torch.stack(refs)

    def grad_step():
        theta = torch.tensor(theta0, dtype=torch.float64, device=dev, requires_grad=True)
        U = autodiff.energy_batch(model, X, theta).sum()
        (gX,) = torch.autograd.grad(U, X, create_graph=True)
        loss = ((gX + R) ** 2).mean()  # (-grad U - F_ref)^2
        loss.backward()
        return theta.grad

    def plain_step():
        th = torch.tensor(theta0, dtype=torch.float64, device=dev)
        for x in xs:
            model.evaluate(x, th, want_grad=False)

    for _ in range(a.warmup):
        grad_step()
    clocks = Clocks(0)
    clocks.start()
    time.sleep(0.3)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize()
    e[0].record()
    for _ in range(a.steps):
        g = grad_step()
    e[1].record()
    torch.cuda.synchronize()
    t_grad = e[0].elapsed_time(e[1]) / 1e3
    e[2].record()
    for _ in range(a.steps):
        plain_step()
    e[3].record()
    torch.cuda.synchronize()
    t_plain = e[2].elapsed_time(e[3]) / 1e3
    model.check()  # raises if any evaluation latched an error on the device
    clk = clocks.stop()
    n_eval = a.steps * len(xs) * wl["n"]
    value = n_eval / t_grad
    _, counts = s.nlist()
    nn, nn_r = float(counts[:, 1].mean()), float(counts[:, 0].mean())
    # bytes one snapshot's kernels must move per particle: state in (28) + one force
    # evaluation with a list build (160 + 4 (nn + nn_r) + 120 + 4 nn) + forces out (24) +
    # the two derivative passes (2 x (32 + 4 nn_r) + 16 + 72)
    b_alg = n_eval * (28 + 160 + 4 * (nn + nn_r) + 120 + 4 * nn + 24 + 2 * (32 + 4 * nn_r) + 16 + 72)
    peak, peak_kind = _peaks()
    achieved = b_alg / t_grad / 1e9
    out = {"metric": DIFF_METRIC, "value": value, "unit": "particle-evaluations/s", "n_gpus": 1,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * t_grad / a.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"diff20k: {len(xs)} snapshots of 20,000 particles, A:B 1:1, density 0.4, "
                                  f"n=10, r_cut=1.5, theta0=(1.3, 0.9, 1.02), target forces at theta=(1,1,1)",
                      "snapshots": len(xs), "particles": wl["n"], "parallelism": "single GPU",
                      "l2": "not flushed (evaluations enqueued back to back, no host synchronisation)"},
           "plain": {"value": n_eval / t_plain, "unit": "particle-evaluations/s",
                     "what": "energy and forces only, same snapshots", "ratio": (n_eval / t_grad) / (n_eval / t_plain)},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "traffic": None, "peak_kind": peak_kind},
           "grad": [float(v) for v in g.cpu().tolist()], "cpu_baseline": None, "e2e": None,
           "gpu_launches": a.steps * len(xs) * 8, "clocks": clk, "kernel_digest": _kernel_digest()}
    print(json.dumps(out), flush=True)
    s.close()
    return 0


VIT_METRIC = "vitrimer particle-timesteps/s (2M beads, chains of 50, harmonic bonds, swap crosslinks; FP32)"


def run_vitrimer(a):
    """Vitrimer network: 2,000,000 beads (chains of 50 with harmonic bonds k=100,
    r0=1, 10 % reactive A beads, as many free B crosslinkers, WCA between all
    other pairs, A-B swap pair lambda 1), density 0.85, BAOAB kT 0.5; one bench
    step = one launch of a.md_steps steps (defaults: 5 x 2000 = 10,000 timed
    steps)."""
    import torch

    from paper_1912_08569_gb300 import SwapSystem, inputs
    from paper_1912_08569_gb300.build import build

    rank, world, local = _dist()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    if rank == 0 or world == 1:
        build()
    if world > 1:
        dist.barrier()
    wl = inputs.vitrimer_workload(2_000_000, seed=1 + rank)
    n = wl["n"]
    s = SwapSystem(n, wl["n_types"], wl["box"], wl["pairs"], precision="fp32", seed=wl["seed"], skin=wl["skin"])
    s.set_state(wl["x"], wl["v"], wl["types"], wl["mass"])
    s.set_bonds(wl["bonds"], wl["kbond"], wl["r0"])
    s.compute_forces()
    dt, kT, gamma = wl["dt"], wl["kT"], wl["gamma"]
    for _ in range(a.warmup):
        s.run(a.md_steps, dt, kT, gamma)
    _, counts = s.nlist()
    nn, nn_r = float(counts[:, 1].mean()), float(counts[:, 0].mean())
    th0 = s.thermo()
    stream = s.stream
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()
        time.sleep(0.3)
    evs = []
    with torch.cuda.stream(stream):
        for _ in range(a.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.run(a.md_steps, dt, kT, gamma, sync=False)
            e1.record(stream)
            evs.append((e0, e1))
    torch.cuda.synchronize()
    s.sync()
    th1 = s.thermo()
    clk = clocks.stop() if clocks else None
    launch_ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    total_ms = max_over_ranks(float(np.sum(launch_ms)), dev)
    value = job_throughput(world, n, a.md_steps, a.steps, total_ms)
    rebuilds = (th1["n_rebuilds"] - th0["n_rebuilds"]) / a.steps
    # the pair path's bytes plus, per particle-step, the bonds: partner tags (16),
    # their slots (8) and positions (32)
    b_alg = algorithmic_bytes(n, a.md_steps, nn, nn_r, rebuilds) + n * a.md_steps * 56.0
    peak, peak_kind = _peaks()
    achieved = b_alg / (float(np.mean(launch_ms)) / 1e3) / 1e9
    if rank == 0:
        out = {"metric": VIT_METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
               "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": f"vitrimer2m: {n} beads, chains of 50 (k=100, r0=1), 10% A + free B "
                                      f"crosslinkers 1:1, WCA otherwise, density 0.85, lambda=1, BAOAB kT=0.5 "
                                      f"gamma=1 dt=0.001, skin 0.3, lattice start",
                          "n_particles": n, "md_steps_per_step": a.md_steps, "parallelism": f"replicas x{world}",
                          "l2": "working set larger than L2 (not flushed)"},
               "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                            "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                            "alg_bytes_per_launch": b_alg, "nn_mean": nn, "nn_reactive_mean": nn_r,
                            "rebuilds_per_launch": rebuilds},
               "cpu_baseline": None, "e2e": None, "gpu_launches": a.steps, "clocks": clk,
               "kernel_digest": _kernel_digest(),
               "thermo_last": {"U2": th1["U2"], "U3": th1["U3"], "K": th1["K"], "n_bonds": th1["n_bonds"]}}
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    s.close()
    return 0


DUMB_METRIC = "dumbbell-mixture particle-timesteps/s (the paper's timing system, n=100; FP32)"


def _dumb_config(a, n, world):
    return {"workload": f"dumbbell: N={n}, A:B 3:2 (every B bonded at the start), density 0.125, n=100, "
                        f"r_cut={a.rcut:g}, lambda=1, WCA A-A and B-B, BAOAB kT=0.03 gamma=1 dt=0.001, skin 0.3",
            "n_particles": n, "r_cut": a.rcut, "md_steps_per_step": a.md_steps, "grid": a.grid or "all SMs",
            "l2": "flushed (512 MB write) between timed launches", "parallelism": f"replicas x{world}"}


def run_reference_dumbbell(a, oracle):
    """The oracle on the dumbbell workload: bounded samples, one thread."""
    wl = _dumbbell(a.n, a.rcut, 0)
    tab = oracle.pair_table(wl["n_types"], wl["pairs"])
    t0 = time.perf_counter()
    oracle.forces(wl["x"], wl["types"], wl["n_types"], tab, wl["box"], fp32=True)
    t_force = time.perf_counter() - t0
    per = int(max(1, min(500, 4.0 / max(t_force, 1e-6))))
    x, v = wl["x"], wl["v"]
    times = []
    for k in range(a.warmup + a.steps):
        t0 = time.perf_counter()
        x, v, _, _ = oracle.run(x, v, wl["types"], wl["mass"], wl["tags"], wl["n_types"], tab, wl["box"],
                                wl["dt"], per, kT=wl["kT"], gamma=wl["gamma"], seed=wl["seed"], step0=k * per,
                                fp32=True)
        if k >= a.warmup:
            times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(times))
    value = wl["n"] * per / (ms / 1e3)
    sample = f"N={wl['n']}, {per} BAOAB steps per step of the FP64 C oracle (1 thread)"
    out = {"impl": "reference", "metric": DUMB_METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": _dumb_config(a, wl["n"], 1), "timesteps_per_s": per / (ms / 1e3),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                            "host": host_info()},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def run_dumbbell(a):
    """The paper's timing system (a mixture of dumbbells, every particle
    reactive or repelled, n = 100, r_cut 1.3 or 1.15) at a.n particles: one
    bench step = one launch of the persistent step kernel over a.md_steps time
    steps; also reported as time steps per second, the paper's measure."""
    import torch

    from paper_1912_08569_gb300 import SwapSystem
    from paper_1912_08569_gb300.build import build

    rank, world, local = _dist()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    if rank == 0 or world == 1:
        build()
    if world > 1:
        dist.barrier()
    wl = _dumbbell(a.n, a.rcut, rank)
    n = wl["n"]
    s = SwapSystem(n, wl["n_types"], wl["box"], wl["pairs"], precision="fp32", seed=wl["seed"], skin=wl["skin"])
    s.set_state(wl["x"], wl["v"], wl["types"], wl["mass"])
    s.set_grid(a.grid)
    s.compute_forces()
    dt, kT, gamma = wl["dt"], wl["kT"], wl["gamma"]
    for _ in range(a.warmup):
        s.run(a.md_steps, dt, kT, gamma)
    _, counts = s.nlist()
    nn, nn_r = float(counts[:, 1].mean()), float(counts[:, 0].mean())
    th0 = s.thermo()
    stream = s.stream
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()
        time.sleep(0.3)
    evs = []
    with torch.cuda.stream(stream):
        for _ in range(a.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.run(a.md_steps, dt, kT, gamma, sync=False)
            e1.record(stream)
            evs.append((e0, e1))
    torch.cuda.synchronize()
    s.sync()
    th1 = s.thermo()
    clk = clocks.stop() if clocks else None
    launch_ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    assert th1["step"] - th0["step"] == a.steps * a.md_steps, "timed launches did not complete"
    total_ms = max_over_ranks(float(np.sum(launch_ms)), dev)
    value = job_throughput(world, n, a.md_steps, a.steps, total_ms)
    rebuilds = (th1["n_rebuilds"] - th0["n_rebuilds"]) / a.steps
    b_alg = algorithmic_bytes(n, a.md_steps, nn, nn_r, rebuilds)
    peak, peak_kind = _peaks()
    achieved = b_alg / (float(np.mean(launch_ms)) / 1e3) / 1e9
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        import oracle

        oracle.build()
        v, steps_done, el = cpu_oracle_sample(wl, a.cpu_seconds, steps_cap=2000)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_info(), "timesteps_per_s": v / n,
               "sample": f"N={n}, {steps_done} BAOAB steps of the FP64 C oracle, {el:.1f} s, 1 thread",
               "accuracy": accuracy_vs_oracle(oracle, s, wl)}
    if rank == 0:
        out = {"metric": DUMB_METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
               "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": _dumb_config(a, n, world),
               "timesteps_per_s": a.md_steps * a.steps / (total_ms / 1e3),
               "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                            "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                            "alg_bytes_per_launch": b_alg, "nn_mean": nn, "nn_reactive_mean": nn_r,
                            "rebuilds_per_launch": rebuilds},
               "cpu_baseline": cpu, "e2e": None, "gpu_launches": a.steps, "clocks": clk,
               "kernel_digest": _kernel_digest(),
               "thermo_last": {"U2": th1["U2"], "U3": th1["U3"], "K": th1["K"], "n_bonds": th1["n_bonds"]}}
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    s.close()
    return 0


def main():
    a = _args()
    if a.n is None:
        a.n = 16384 if a.workload == "dumbbell" else 100_000
    if a.md_steps is None:
        a.md_steps = {"batch256": 5000, "vitrimer2m": 2000, "dumbbell": 4000}.get(a.workload, 1000)
    if a.impl == "reference":
        return run_reference(a)
    if a.workload == "batch256":
        return run_batch(a)
    if a.workload == "diff20k":
        return run_diff(a)
    if a.workload == "vitrimer2m":
        return run_vitrimer(a)
    if a.workload == "dumbbell":
        return run_dumbbell(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
