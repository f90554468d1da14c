"""Bond-swap dynamics of the dumbbell mixture (section "Effect of swaps"),
run on the GPU path: the bond autocorrelation function and its relaxation time.

The system (``inputs.dumbbell_workload``): 600 A and 400 B particles at number
density 0.125, A-B swap pair with n = 100 (eps = sigma = 1, lambda = 1), A-A and
B-B WCA with sigma = eps = 1, BAOAB Langevin at kT (gamma = 1, dt = 0.001).  At
kT = 0.03 every B stays bonded to one A (the minority forms dumbbells); a bond
changes partner only through a swap with one of the 200 free A particles.

Bond: an A-B pair closer than r_bond, the outer root of v = -eps/2 (1.0194 sigma
for n = 100).  c(t): the fraction of the A-B bonds present at a time origin
that are present again a time t later, averaged over time origins and
replicas.  tau: least-squares slope of log c(t) against t through the origin,
over the points with c > 0.05.  The paper shows an exponential decay of c(t)
with a relaxation time of 116 at kT = 0.03 and a faster decay at higher
temperature; its friction and time unit are not stated, so 116 is context,
not a target.

Mass split (section "Physical advantages of the method"): half of the A
particles get mass 1/10; c(t) is then taken separately over the bonds whose A
is light and those whose A is heavy.  The paper shows the light bonds relaxing
faster (60 against 98 for the heavy ones, both below the 116 of equal masses).

Host-side analysis of positions read back from the device: it is not part of
the time step.
"""
from __future__ import annotations

import json
import sys

import numpy as np

from . import inputs


def bond_pairs(x, types, box, rbond):
    """Set of (b, a) index pairs (B first) closer than rbond (minimum image)."""
    from scipy.spatial import cKDTree

    L = np.asarray(box, dtype=np.float64)
    xw = np.mod(np.asarray(x, dtype=np.float64), L)
    xw[xw >= L] = 0.0
    ia = np.nonzero(types == 0)[0]
    ib = np.nonzero(types == 1)[0]
    ta = cKDTree(xw[ia], boxsize=L)
    out = set()
    for k, lst in enumerate(ta.query_ball_point(xw[ib], rbond)):
        for j in lst:
            out.add((int(ib[k]), int(ia[j])))
    return out


def autocorrelation(bond_sets, max_lag):
    """c(lag) for lag = 0 .. max_lag samples, averaged over every time origin."""
    c = np.zeros(max_lag + 1)
    cnt = np.zeros(max_lag + 1)
    for t0 in range(len(bond_sets)):
        b0 = bond_sets[t0]
        if not b0:
            continue
        for lag in range(0, min(max_lag, len(bond_sets) - 1 - t0) + 1):
            c[lag] += len(b0 & bond_sets[t0 + lag]) / len(b0)
            cnt[lag] += 1
    return c / np.maximum(cnt, 1)


def fit_tau(t, c, cmin=0.05):
    m = (c > cmin) & (t > 0)
    if m.sum() < 2:
        return float("nan"), 0.0
    y = np.log(c[m])
    tau = -float(np.sum(t[m] * t[m]) / np.sum(t[m] * y))
    pred = -t[m] / tau
    ss_res = float(np.sum((y - pred) ** 2))
    ss_tot = float(np.sum((y - y.mean()) ** 2)) or 1.0
    return tau, 1.0 - ss_res / ss_tot


def run(kT=0.03, replicas=8, t_equil=20.0, t_max=400.0, sample_dt=1.0, seed=1, precision="fp32", split=1e9,
        light_mass=None, keep_final=False):
    """Advances `replicas` independent dumbbell systems together (one batched
    launch per sample interval) and returns the bond statistics.  light_mass:
    give half of the A particles (seeded choice) this mass and also return the
    statistics of the light-A and heavy-A bonds separately.  keep_final: also
    return every replica's last positions with the kernel's bond count of that
    step ("final": list of dicts x, types, box, pairs, n_bonds)."""
    from .system import SwapBatch, SwapSystem

    wls = [inputs.dumbbell_workload(seed=seed + 17 * r, kT=kT) for r in range(replicas)]
    light = []
    for r, wl in enumerate(wls):
        lt = np.zeros(wl["n"], dtype=bool)
        if light_mass is not None:
            ia = np.nonzero(wl["types"] == 0)[0]
            pick = np.random.Generator(np.random.Philox(seed + 91 * r)).choice(len(ia), len(ia) // 2, replace=False)
            lt[ia[pick]] = True
            wl["mass"] = np.where(lt, float(light_mass), 1.0)
            wl["v"] = inputs.maxwell_velocities(wl["n"], kT, wl["mass"], seed=wl["seed"] + 1000)
        light.append(lt)
    systems = []
    for wl in wls:
        s = SwapSystem(wl["n"], 2, wl["box"], wl["pairs"], precision=precision, seed=wl["seed"], skin=wl["skin"])
        s.set_state(wl["x"], wl["v"], wl["types"], wl["mass"])
        systems.append(s)
    batch = SwapBatch(systems, split=split)
    dt, gamma = 0.001, 1.0
    per = int(round(sample_dt / dt))
    batch.run(int(round(t_equil / dt)), dt, kT, gamma)
    rbond = wls[0]["pairs"][(0, 1)]["rbond"]
    sets = [[] for _ in range(replicas)]
    bonded_min, multi_max = 1.0, 0
    nsamp = int(round(t_max / sample_dt)) + 1
    for k in range(nsamp):
        if k:
            batch.run(per, dt, kT, gamma)
        for r, (s, wl) in enumerate(zip(systems, wls)):
            x, _, _ = s.state()
            bp = bond_pairs(x, wl["types"], wl["box"], rbond)
            sets[r].append(bp)
            nb = int((wl["types"] == 1).sum())
            partners_b = np.bincount([b for b, _ in bp], minlength=wl["n"])
            partners_a = np.bincount([a for _, a in bp], minlength=wl["n"])
            bonded_min = min(bonded_min, float(np.count_nonzero(partners_b[wl["types"] == 1])) / nb)
            multi_max = max(multi_max, int(partners_a.max()), int(partners_b.max()))
    max_lag = nsamp // 2
    c = np.mean([autocorrelation(sr, max_lag) for sr in sets], axis=0)
    t = np.arange(max_lag + 1) * sample_dt
    tau, r2 = fit_tau(t, c)
    split_stats = {}
    if light_mass is not None:
        for name, want in (("light", True), ("heavy", False)):
            sub = [[{(b, a) for (b, a) in bp if light[r][a] == want} for bp in sr] for r, sr in enumerate(sets)]
            cs = np.mean([autocorrelation(sr, max_lag) for sr in sub], axis=0)
            ts, rs = fit_tau(t, cs)
            split_stats[name] = dict(c=cs.tolist(), tau=ts, fit_r2=rs)
    th = [s.thermo() for s in systems]
    # the kernel's own bond count of the last step against the host count
    bond_count_diff = max(abs(int(h["n_bonds"]) - len(sr[-1])) for h, sr in zip(th, sets))
    final = []
    if keep_final:
        for s, wl, h in zip(systems, wls, th):
            x, _, _ = s.state()
            final.append(dict(x=x, types=wl["types"], box=wl["box"], pairs=wl["pairs"], n_bonds=int(h["n_bonds"])))
    for s in systems:
        s.close()
    return dict(kT=kT, replicas=replicas, t_max=t_max, sample_dt=sample_dt, t=t.tolist(), c=c.tolist(), tau=tau,
                fit_r2=r2, bonded_fraction_min=bonded_min, max_bonds_per_particle=multi_max,
                n_bonds_mean=float(np.mean([h["n_bonds"] for h in th])), bond_count_diff=bond_count_diff,
                mass_split=split_stats, final=final)


def main(argv=None):
    import argparse

    ap = argparse.ArgumentParser(description="bond autocorrelation of the dumbbell mixture")
    ap.add_argument("--kT", type=float, nargs="+", default=[0.03, 0.05])
    ap.add_argument("--replicas", type=int, default=8)
    ap.add_argument("--t-max", type=float, default=400.0)
    ap.add_argument("--light-mass", type=float, default=None,
                    help="mass of half of the A particles (the paper's split uses 0.1)")
    a = ap.parse_args(argv)
    for kT in a.kT:
        r = run(kT=kT, replicas=a.replicas, t_max=a.t_max, light_mass=a.light_mass)
        r.pop("t")
        r.pop("final")
        r["c"] = [round(v, 4) for v in r["c"][::10]]
        for v in r["mass_split"].values():
            v["c"] = [round(x, 4) for x in v["c"][::10]]
        print(json.dumps(r), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
