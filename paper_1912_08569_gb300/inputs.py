"""Seeded synthetic inputs shared by the tests, the oracle legs and the benchmark.

This module holds no arithmetic of the method: it only draws configurations.
Every array it returns is exactly representable in float32 (positions,
velocities, box lengths), so that an FP32 device path and an FP64 CPU path see
bit-identical inputs.

Recipe (the paper has no public dataset; these stand in for its workloads):

* positions: random sequential addition, uniform in a periodic orthorhombic box,
  with a minimum pair separation (0.9 sigma by default), drawn from numpy's
  Philox bit generator in batches; a candidate is rejected if it is closer than
  the minimum separation to any accepted particle or to an earlier candidate of
  its batch;
* types: alternate by tag (tag % n_types), A:B = 1:1 for two types;
* velocities: Maxwell-Boltzmann at kT with the centre-of-mass velocity removed;
* box: cubic, L = (N / density)^(1/3) rounded to float32.
"""
from __future__ import annotations

import numpy as np

try:  # scipy is present on both the build host and the GPU host
    from scipy.spatial import cKDTree
except Exception:  # pragma: no cover - fallback for minimal environments
    cKDTree = None


def f32(a):
    """Round to the nearest float32 and return as float64."""
    return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)


def cubic_box(n: int, density: float) -> np.ndarray:
    L = float(np.float32((n / density) ** (1.0 / 3.0)))
    return np.array([L, L, L])


def _min_dist_brute(cand, pts, box):
    if len(pts) == 0:
        return np.full(len(cand), np.inf)
    d = cand[:, None, :] - pts[None, :, :]
    d -= box * np.round(d / box)
    return np.sqrt((d * d).sum(-1)).min(axis=1)


def rsa_positions(n: int, box, min_sep: float = 0.9, seed: int = 1, batch: int | None = None,
                  max_tries: int = 10000) -> np.ndarray:
    """n positions (n x 3, float32-representable) with pairwise separation >= min_sep.

    Candidates are drawn in batches of 16,384 (262,144 above 500,000
    particles, where rebuilding the tree of accepted points per batch would
    dominate: a 2M-particle box then takes about a minute instead of several)."""
    if batch is None:
        batch = 16384 if n <= 500_000 else 262_144
    box = np.asarray(box, dtype=np.float64)
    rng = np.random.Generator(np.random.Philox(seed))
    pts = np.zeros((0, 3))
    tries = 0
    while len(pts) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("rsa_positions: could not place particles (density too high)")
        m = min(batch, max(64, 2 * (n - len(pts))))
        cand = f32(rng.random((m, 3)) * box)
        cand[cand >= box] = 0.0
        cand[cand < 2.0 ** -20] = 0.0
        if cKDTree is not None:
            if len(pts):
                tree = cKDTree(pts, boxsize=box)
                dmin, _ = tree.query(cand, k=1, distance_upper_bound=min_sep)
                ok = ~(dmin < min_sep)
            else:
                ok = np.ones(m, dtype=bool)
            cand = cand[ok]
            if len(cand) > 1:
                ct = cKDTree(cand, boxsize=box)
                pairs = ct.query_pairs(min_sep, output_type="ndarray")
                bad = np.zeros(len(cand), dtype=bool)
                if len(pairs):
                    bad[np.maximum(pairs[:, 0], pairs[:, 1])] = True
                cand = cand[~bad]
        else:
            ok = _min_dist_brute(cand, pts, box) >= min_sep
            cand = cand[ok]
            keep = []
            for i in range(len(cand)):
                if all(np.linalg.norm((cand[i] - cand[j]) - box * np.round((cand[i] - cand[j]) / box))
                       >= min_sep for j in keep):
                    keep.append(i)
            cand = cand[keep]
        pts = np.concatenate([pts, cand[: n - len(pts)]], axis=0)
    return pts


def alternating_types(n: int, n_types: int = 2) -> np.ndarray:
    return (np.arange(n) % n_types).astype(np.int32)


def maxwell_velocities(n: int, kT: float, mass, seed: int = 2) -> np.ndarray:
    """Maxwell-Boltzmann velocities (n x 3, float32-representable), zero total momentum."""
    rng = np.random.Generator(np.random.Philox(seed))
    m = np.broadcast_to(np.asarray(mass, dtype=np.float64), (n,))
    v = rng.standard_normal((n, 3)) * np.sqrt(kT / m)[:, None]
    if n > 0:
        v -= (m[:, None] * v).sum(0) / m.sum()
    return f32(v)


def swap_pairs(eps=1.0, sigma=1.0, n=10, rcut=1.5, lambda3=1.0, shift=0, rbond=None,
               wca_sigma=1.0, wca_eps=1.0, wca_n=6):
    """Two-type table of the paper's binary mixture: A-B swap, A-A and B-B WCA.

    Returned as {(ti, tj): params}; ``rbond`` defaults to the outer root of
    v = -eps/2 (where the normalised term equals one half).
    """
    if rbond is None:
        rbond = sigma * ((1.0 - np.sqrt(0.5)) / 2.0) ** (-1.0 / n)
    sw = dict(kind=2, eps=eps, sigma=sigma, n=n, rcut=rcut, lambda3=lambda3, shift=shift,
              rbond=rbond)
    wca = dict(kind=1, eps=wca_eps, sigma=wca_sigma, n=wca_n)
    return {(0, 1): sw, (0, 0): wca, (1, 1): wca}


def workload(name: str = "mix100k", lambda3: float = 1.0, seed: int = 1, n: int | None = None,
             density: float | None = None, shift: int = 0):
    """Named synthetic workloads.

    * ``mix2k``: 2,000 particles, A:B 1:1, density 0.2, NVE dt 0.001 from Maxwell
      velocities at kT 0.1 (the small FP64 parity case);
    * ``mix100k``: 100,000 particles, A:B 1:1, density 0.5, Langevin kT 0.05,
      gamma 1, dt 0.001, skin 0.3 (the FP32 throughput case).
    Both: A-B swap pair with eps = sigma = 1, n = 10, r_cut = 1.5; A-A and B-B
    WCA with sigma = 1; minimum separation 0.9.
    """
    if name == "mix2k":
        n = n or 2000
        density = density or 0.2
        kT, gamma, dt, skin = 0.1, 0.0, 0.001, 0.3
    elif name == "mix100k":
        n = n or 100_000
        density = density or 0.5
        kT, gamma, dt, skin = 0.05, 1.0, 0.001, 0.3
    else:
        raise ValueError(f"unknown workload {name!r}")
    box = cubic_box(n, density)
    x = rsa_positions(n, box, 0.9, seed=seed)
    types = alternating_types(n, 2)
    mass = np.ones(n)
    v = maxwell_velocities(n, kT, mass, seed=seed + 1000)
    return dict(name=name, n=n, density=density, box=box, x=x, v=v, types=types, mass=mass,
                tags=np.arange(n, dtype=np.uint32), n_types=2,
                pairs=swap_pairs(lambda3=lambda3, shift=shift), kT=kT, gamma=gamma, dt=dt,
                skin=skin, seed=seed)


def batch_workload(n_systems: int = 256, seed: int = 7, n_min: int = 1000, n_max: int = 32000,
                   density=(0.2, 0.6), lambdas=(0.0, 0.5, 1.0, 2.0, 5.0), kT=(0.03, 0.2)):
    """Independent systems of uneven size for a batched run (seeded).

    Sizes log-uniform in [n_min, n_max], densities uniform in ``density``,
    lambda cycling through ``lambdas``, temperatures uniform in ``kT``; each
    system is the binary A:B 1:1 mixture of ``workload`` (RSA positions,
    Maxwell velocities at its temperature), BAOAB gamma 1, dt 0.001, skin 0.3.
    """
    out = []
    for k, (n, rho, t, lam) in enumerate(batch_params(n_systems, seed, n_min, n_max, density, lambdas, kT)):
        wl = workload("mix100k", lambda3=lam, seed=seed * 1000 + k, n=n, density=rho)
        wl["kT"] = t
        wl["v"] = maxwell_velocities(n, t, wl["mass"], seed=seed * 1000 + k + 500)
        out.append(wl)
    return out


def batch_params(n_systems: int = 256, seed: int = 7, n_min: int = 1000, n_max: int = 32000,
                 density=(0.2, 0.6), lambdas=(0.0, 0.5, 1.0, 2.0, 5.0), kT=(0.03, 0.2)):
    """(n, density, kT, lambda) of each system of ``batch_workload`` with the
    same arguments, without generating the systems."""
    rng = np.random.Generator(np.random.Philox(seed))
    out = []
    for k in range(n_systems):
        n = int(round(np.exp(rng.uniform(np.log(n_min), np.log(n_max)))))
        rho = float(rng.uniform(*density))
        t = float(rng.uniform(*kT))
        out.append((n, rho, t, float(lambdas[k % len(lambdas)])))
    return out


class _SeparationGrid:
    """Points laid down one by one with a minimum separation dmin (minimum
    image): far(c) tells whether c is at least dmin from every point added so
    far, looking only at the 27 cells around c (cells at least dmin wide), so
    that it gives the same answer as a check against every point."""

    def __init__(self, box, dmin):
        self.box = np.asarray(box, dtype=np.float64)
        self.dmin2 = dmin * dmin
        self.m = np.floor(self.box / (dmin * (1.0 + 1e-6))).astype(np.int64)
        self.use_cells = bool(np.all(self.m >= 3))
        self.cells = {}
        self.all = []

    def _cell(self, c):
        return tuple(int(k) for k in np.minimum((c / self.box * self.m).astype(np.int64), self.m - 1))

    def far(self, c):
        if not self.all:
            return True
        if self.use_cells:
            cx, cy, cz = self._cell(c)
            mx, my, mz = (int(v) for v in self.m)
            near = []
            for dz in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        near.extend(self.cells.get(((cx + dx) % mx, (cy + dy) % my, (cz + dz) % mz), ()))
            if not near:
                return True
            others = np.array(near, dtype=np.float64)
        else:
            others = np.array(self.all, dtype=np.float64)
        d = others - c
        d -= self.box * np.round(d / self.box)
        return np.min(np.sum(d * d, axis=1)) >= self.dmin2

    def add(self, c):
        self.all.append(c)
        if self.use_cells:
            self.cells.setdefault(self._cell(c), []).append(c)

    def points(self):
        return np.array(self.all, dtype=np.float64).reshape(-1, 3)


def dumbbell_workload(seed: int = 1, kT: float = 0.03, n_a: int = 600, n_b: int = 400, density: float = 0.125,
                      n: int = 100, rcut: float = 1.3, lambda3: float = 1.0):
    """The dumbbell mixture of section "Effect of swaps": n_a A and n_b B
    particles at the given density, A-B swap pair with exponent n, A-A and B-B
    WCA.  Every B starts bonded: it is placed at distance 2^(1/n) (the minimum
    of the pair potential) from its own A, in a random direction, and the
    pairs and the free A are laid down by random sequential addition with a
    minimum separation of 1.0 from everything else (closer A-B pairs would
    start with the enormous energies of the n = 100 wall)."""
    if n_b > n_a:
        raise ValueError("needs n_b <= n_a (every B bonded to its own A)")
    rng = np.random.Generator(np.random.Philox(seed))
    N = n_a + n_b
    box = cubic_box(N, density)
    L = box[0]
    rmin = 2.0 ** (1.0 / n)
    grid = _SeparationGrid(box, 1.0)
    types = []
    tries = 0
    while len(types) < N:
        tries += 1
        if tries > 200000 + 20 * N:
            raise RuntimeError("dumbbell_workload: could not place particles")
        a = f32(rng.random(3) * box)
        a[a >= box] = 0.0
        pair = len(types) < 2 * n_b
        if pair:
            u = rng.standard_normal(3)
            u /= np.linalg.norm(u)
            b = f32(np.mod(a + rmin * u, L))
            b[b >= box] = 0.0
            if not (grid.far(a) and grid.far(b)):
                continue
            grid.add(a)
            grid.add(b)
            types += [0, 1]
        else:
            if not grid.far(a):
                continue
            grid.add(a)
            types.append(0)
    x = grid.points()
    types = np.asarray(types, dtype=np.int32)
    mass = np.ones(N)
    v = maxwell_velocities(N, kT, mass, seed=seed + 1000)
    pairs = swap_pairs(n=n, rcut=rcut, lambda3=lambda3)
    return dict(name="dumbbell", n=N, density=density, box=box, x=x, v=v, types=types, mass=mass,
                tags=np.arange(N, dtype=np.uint32), n_types=2, pairs=pairs, kT=kT, gamma=1.0, dt=0.001,
                skin=0.3, seed=seed)


def vitrimer_workload(n_total: int = 2_000_000, chain_len: int = 50, per_chain_a: int = 5, density: float = 0.85,
                      kT: float = 0.5, seed: int = 1, kbond: float = 100.0, r0: float = 1.0, lambda3: float = 1.0):
    """A vitrimer-like network: linear chains of chain_len beads joined by
    harmonic bonds (kbond, r0), per_chain_a of each chain's beads reactive
    (type A = 0), as many free crosslinkers (type B = 1), the other chain beads
    plain (type C = 2).  A-B: the swap pair (n = 10, r_cut = 1.5, lambda3); every
    other pair: WCA (sigma = eps = 1); the bonded pairs keep their WCA.

    Start: a simple cubic lattice filling the box at the given density,
    visited along a boustrophedon path (consecutive sites are lattice
    neighbours); each chain takes chain_len consecutive sites followed by its
    per_chain_a crosslinkers, so the crosslinkers are spread through the
    melt.  The A beads are drawn per chain (seeded).  Returns the usual
    workload dict plus "bonds" [m, 2] (tags) and the bond constants.
    """
    rng = np.random.Generator(np.random.Philox(seed))
    unit = chain_len + per_chain_a
    n_chains = max(1, n_total // unit)
    N = n_chains * unit
    box = cubic_box(N, density)
    L = box[0]
    m = int(np.ceil(N ** (1.0 / 3.0) - 1e-9))
    a = L / m
    # boustrophedon order of the m^3 sites
    sites = []
    for z in range(m):
        ys = range(m) if z % 2 == 0 else range(m - 1, -1, -1)
        for k, y in enumerate(ys):
            xs = range(m) if (z * m + k) % 2 == 0 else range(m - 1, -1, -1)
            for x in xs:
                sites.append((x, y, z))
                if len(sites) == N:
                    break
            if len(sites) == N:
                break
        if len(sites) == N:
            break
    pos = f32((np.asarray(sites, dtype=np.float64) + 0.5) * a)
    types = np.full(N, 2, dtype=np.int32)
    bonds = []
    for c in range(n_chains):
        base = c * unit
        bonds.extend([(base + i, base + i + 1) for i in range(chain_len - 1)])
        reactive = rng.choice(chain_len, size=per_chain_a, replace=False)
        types[base + reactive] = 0
        types[base + chain_len: base + unit] = 1
    mass = np.ones(N)
    v = maxwell_velocities(N, kT, mass, seed=seed + 1000)
    sw = dict(kind=2, eps=1.0, sigma=1.0, n=10, rcut=1.5, lambda3=lambda3, shift=0,
              rbond=((1.0 - np.sqrt(0.5)) / 2.0) ** (-1.0 / 10))
    wca = dict(kind=1, eps=1.0, sigma=1.0, n=6)
    pairs = {(0, 1): sw}
    for ti in range(3):
        for tj in range(ti, 3):
            if (ti, tj) != (0, 1):
                pairs[(ti, tj)] = wca
    return dict(name="vitrimer", n=N, density=density, box=box, x=pos, v=v, types=types, mass=mass,
                tags=np.arange(N, dtype=np.uint32), n_types=3, pairs=pairs, kT=kT, gamma=1.0, dt=0.001, skin=0.3,
                seed=seed, bonds=np.asarray(bonds, dtype=np.int32), kbond=kbond, r0=r0)
