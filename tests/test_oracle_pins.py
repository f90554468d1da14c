"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties one part of ``oracle/`` to something other than itself:
closed forms printed or implied by the paper (Eq. 2b, Eq. pot, Eq. 3bp and the
three regimes of section "The swap potential"), the lambda = 0 special case,
brute-force all-pairs/all-triples sums, finite differences of the energy,
the virial by affine deformation, symmetry invariants, integrator properties
and published generator test vectors.
"""
import math
import os

import numpy as np
import pytest

from brute import brute, brute_nlist
from paper_1912_08569_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = {}
    with open(os.path.join(GOLD, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            rows[parts[0]] = (float(parts[1]), float(parts[2]))
    return rows


def lj_closed(r, eps=1.0, sig=1.0, n=10):
    return 4 * eps * ((sig / r) ** (2 * n) - (sig / r) ** n)


SW = dict(eps=1.0, sigma=1.0, n=10, rcut=1.5, lambda3=1.0, shift=0, rbond=1.2)


def three_body_table(orc, lam, shift=0, n=10, eps=1.0):
    """Types: 0 = A, 1 = B.  A-B swap; A-A and B-B WCA (off beyond 2^(1/6))."""
    sw = dict(SW, kind=2, lambda3=lam, shift=shift, n=n, eps=eps)
    wca = dict(kind=1, eps=1.0, sigma=1.0, n=6)
    pairs = {(0, 1): sw, (0, 0): wca, (1, 1): wca}
    return orc.pair_table(2, pairs), pairs


def triad(r1, r2, angle=math.pi * 0.75, L=30.0):
    """B at the centre, A1 at r1 along x, A2 at r2 at the given angle."""
    c = np.array([L / 2, L / 2, L / 2])
    x = np.array([c, c + [r1, 0, 0], c + [r2 * math.cos(angle), r2 * math.sin(angle), 0]])
    return x, np.array([1, 0, 0], dtype=np.int32), np.array([L, L, L])


# ---------------------------------------------------------------------------
# Eq. 2b / Eq. pot closed forms


def test_golden_paper_values(orc):
    g = _golden("paper_values.txt")
    assert abs(2 ** (1 / 10) - g["rmin_n10"][0]) <= g["rmin_n10"][1]
    assert abs(orc.v2(g["rmin_n10"][0], 1, 1, 10) - g["v_at_rmin_n10"][0]) <= g["v_at_rmin_n10"][1]
    assert abs(orc.v2(g["rmin_n100"][0], 1, 1, 100) - g["v_at_rmin_n100"][0]) <= g["v_at_rmin_n100"][1]
    assert abs(abs(orc.dv2(1.15, 1, 1, 100)) - g["force_at_1p15_n100"][0]) <= g["force_at_1p15_n100"][1]
    assert abs(orc.v2(2.5, 1, 1, 6) - g["lj_at_2p5_n6"][0]) <= g["lj_at_2p5_n6"][1]
    # and the reading: v(1.15) itself is four orders of magnitude below LJ(2.5)
    assert 1e-5 < abs(orc.v2(1.15, 1, 1, 100) / orc.v2(2.5, 1, 1, 6)) < 1e-3


@pytest.mark.parametrize("n", [1, 3, 6, 10, 100])
@pytest.mark.parametrize("eps,sig", [(1.0, 1.0), (2.5, 0.8), (100.0, 1.3)])
def test_rmin_is_minimum_of_depth_eps(orc, n, eps, sig):
    rmin = sig * 2 ** (1 / n)
    assert orc.v2(rmin, eps, sig, n) == pytest.approx(-eps, rel=1e-13)
    assert abs(orc.dv2(rmin, eps, sig, n)) <= 1e-12 * eps * n / sig
    # a minimum: higher on both sides
    assert orc.v2(rmin * 1.01, eps, sig, n) > -eps and orc.v2(rmin * 0.99, eps, sig, n) > -eps


def test_textbook_lennard_jones(orc):
    # n = 6 is the 12-6 Lennard-Jones potential: zero at sigma, -eps at 2^(1/6) sigma
    assert abs(orc.v2(1.0, 1, 1, 6)) < 1e-15
    assert orc.v2(2 ** (1 / 6), 1, 1, 6) == pytest.approx(-1.0, rel=1e-14)
    assert orc.v2(2.0, 1.0, 1.0, 6) == pytest.approx(4 * (2.0 ** -12 - 2.0 ** -6), rel=1e-14)


def test_vhat_eq_pot(orc):
    rmin = 2 ** (1 / 10)
    for r in (0.8, 0.95, rmin):
        assert orc.vhat(r, **SW) == 1.0
    for r in (1.1, 1.2, 1.4, 1.499):
        assert orc.vhat(r, **SW) == pytest.approx(-lj_closed(r), rel=1e-14)
    assert orc.vhat(1.5, **SW) == 0.0 and orc.vhat(2.0, **SW) == 0.0
    # C1 at r_min: one-sided slope vanishes
    h = 1e-7
    assert abs(orc.vhat(rmin + h, **SW) - 1.0) < 1e-9
    # shifted form: continuous at r_cut, still 1 at r_min, in [0, 1]
    sh = dict(SW, shift=1)
    assert abs(orc.vhat(1.5 - 1e-9, **sh)) < 1e-8
    assert orc.vhat(rmin, **sh) == 1.0
    assert abs(orc.vhat(rmin + h, **sh) - 1.0) < 1e-9
    rs = np.linspace(rmin, 1.5, 50, endpoint=False)
    vals = [orc.vhat(r, **sh) for r in rs]
    assert all(0.0 <= v <= 1.0 for v in vals) and all(np.diff(vals) < 0)


# ---------------------------------------------------------------------------
# The three regimes of Fig. 1 (section "The swap potential")


@pytest.mark.parametrize("lam", [0.5, 1.0, 2.0, 5.0])
def test_regime_a_both_inside_rmin(orc, lam):
    tab, _ = three_body_table(orc, lam)
    x, ty, box = triad(1.0, 0.98)
    r = orc.forces(x, ty, 2, tab, box)
    tab0, _ = three_body_table(orc, 0.0)
    r0 = orc.forces(x, ty, 2, tab0, box)
    assert r["U3"] == pytest.approx(lam * 1.0, rel=1e-15)  # constant lambda*eps
    np.testing.assert_allclose(r["F"], r0["F"], rtol=0, atol=1e-12)  # no three-body force


@pytest.mark.parametrize("lam", [0.5, 1.0, 2.0, 5.0])
@pytest.mark.parametrize("r2", [1.1, 1.25, 1.4])
def test_regime_b_one_inside(orc, lam, r2):
    tab, _ = three_body_table(orc, lam)
    r1 = 1.02
    x, ty, box = triad(r1, r2)
    r = orc.forces(x, ty, 2, tab, box)
    # eq. regb: U = v(r1) + (1 - lambda) v(r2)
    assert r["U2"] + r["U3"] == pytest.approx(lj_closed(r1) + (1 - lam) * lj_closed(r2), rel=1e-13)
    # only A2 feels the three-body force: (1 - lambda) times its pair force
    dvdr = 4 * (-20 * r2 ** -21 + 10 * r2 ** -11)
    f_pair = -dvdr  # along the unit vector from B to A2
    u = (x[2] - x[0]) / r2
    np.testing.assert_allclose(r["F"][2], (1 - lam) * f_pair * u, rtol=1e-12, atol=1e-13)


def test_regime_b_lambda_one_shields_exactly(orc):
    tab, _ = three_body_table(orc, 1.0)
    energies = []
    for r2 in np.linspace(1.08, 1.49, 23):
        x, ty, box = triad(1.03, r2)
        r = orc.forces(x, ty, 2, tab, box)
        assert np.all(np.abs(r["F"][2]) < 1e-13)  # force on A2 is exactly zero
        energies.append(r["U2"] + r["U3"])
    # flat energy landscape (Fig. 2): total independent of r2
    assert np.ptp(energies) < 1e-13


@pytest.mark.parametrize("lam", [1.0, 2.0, 5.0])
def test_swap_barrier(orc, lam):
    g = _golden("paper_values.txt")
    tab, _ = three_body_table(orc, lam)
    rmin = 2 ** (1 / 10)
    x, ty, box = triad(rmin, rmin)
    both = orc.forces(x, ty, 2, tab, box)
    x, ty, box = triad(rmin, 3.0)
    one = orc.forces(x, ty, 2, tab, box)
    dE = (both["U2"] + both["U3"]) - (one["U2"] + one["U3"])
    assert dE == pytest.approx(lam - 1.0, abs=1e-13)  # eps (lambda - 1)
    if lam == 1.0:
        assert abs(dE - g["barrier_lambda1"][0]) <= g["barrier_lambda1"][1]
    if lam == 5.0:
        assert abs(dE - g["barrier_lambda5"][0]) <= g["barrier_lambda5"][1]


@pytest.mark.parametrize("lam", [0.5, 1.0, 5.0])
def test_regime_c_both_outside(orc, lam):
    tab, _ = three_body_table(orc, lam)
    r1, r2 = 1.12, 1.3
    x, ty, box = triad(r1, r2)
    r = orc.forces(x, ty, 2, tab, box)
    v1, v2 = lj_closed(r1), lj_closed(r2)
    assert r["U2"] + r["U3"] == pytest.approx(v1 + v2 + lam * v1 * v2, rel=1e-13)
    # both A feel a three-body force
    tab0, _ = three_body_table(orc, 0.0)
    r0 = orc.forces(x, ty, 2, tab0, box)
    assert np.linalg.norm(r["F"][1] - r0["F"][1]) > 1e-3
    assert np.linalg.norm(r["F"][2] - r0["F"][2]) > 1e-3


def test_lambda_zero_is_pair_potential(orc):
    box = inputs.cubic_box(300, 0.4)
    x = inputs.rsa_positions(300, box, 0.9, seed=5)
    ty = inputs.alternating_types(300)
    pairs = inputs.swap_pairs(lambda3=0.0, n=6, rcut=2.0)
    tab = orc.pair_table(2, pairs)
    r = orc.forces(x, ty, 2, tab, box)
    assert r["U3"] == 0.0
    # plain vectorised 12-6 LJ (A-B, cut 2.0) + WCA (like types) over all pairs
    d = x[:, None, :] - x[None, :, :]
    d -= box * np.round(d / box)
    r2 = (d ** 2).sum(-1)
    iu = np.triu_indices(300, 1)
    rr = np.sqrt(r2[iu])
    unlike = (ty[iu[0]] != ty[iu[1]])
    lj = 4 * (rr ** -12 - rr ** -6)
    u = np.where(unlike & (rr < 2.0), lj, 0.0) + np.where(~unlike & (rr < 2 ** (1 / 6)), lj + 1, 0.0)
    assert r["U2"] == pytest.approx(u.sum(), rel=1e-12)


# ---------------------------------------------------------------------------
# Brute force (all pairs, all triples)


def _small_system(seed, n=24, L=6.0, types=2, min_sep=0.85):
    box = np.array([L, L * 1.1, L * 0.95])
    box = inputs.f32(box)
    x = inputs.rsa_positions(n, box, min_sep, seed=seed)
    ty = (np.arange(n) % types).astype(np.int32)
    return x, ty, box


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("lam,shift", [(1.0, 0), (5.0, 0), (2.0, 1)])
def test_oracle_matches_brute_force(orc, seed, fp32, lam, shift):
    x, ty, box = _small_system(seed, n=30, L=5.6)
    pairs = inputs.swap_pairs(lambda3=lam, shift=shift)
    tab = orc.pair_table(2, pairs)
    r = orc.forces(x, ty, 2, tab, box, fp32=fp32)
    b = brute(x, ty, pairs, box, fp32=fp32)
    assert r["U3"] != 0.0
    assert r["U2"] == pytest.approx(b["U2"], rel=1e-12, abs=1e-12)
    assert r["U3"] == pytest.approx(b["U3"], rel=1e-12, abs=1e-12)
    np.testing.assert_allclose(r["F"], b["F"], rtol=1e-11, atol=1e-10)
    np.testing.assert_allclose(r["W"], b["W"], rtol=1e-11, atol=1e-10)
    assert r["n_bonds"] == b["n_bonds"]


def test_fp32_decision_distance_is_accurate_in_large_boxes():
    """The FP32 decision displacement (32-bit box fractions) is within a few
    units of 2^-32 L of the exact minimum-image displacement, whatever the
    coordinates: for a box of 133 sigma and pairs straddling the periodic
    faces, d2 agrees with the FP64 value to 1e-6 relative."""
    from brute import _d2_decision

    rng = np.random.default_rng(3)
    L = float(np.float32(133.7))
    box = np.array([L, L * 0.9, L * 1.1])
    box = inputs.f32(box)
    for k in range(400):
        xi = rng.random(3) * box
        if k % 2:  # half of the pairs straddle a face
            c = k % 3
            xi[c] = box[c] - rng.uniform(0.0, 1.0)
        d = rng.normal(size=3)
        d *= rng.uniform(0.5, 2.0) / np.linalg.norm(d)
        xj = np.mod(xi + d, box)
        exact = _d2_decision(xi, xj, box, False)
        approx = _d2_decision(xi, xj, box, True)
        assert abs(approx - exact) <= 1e-6 * exact, (approx, exact)


def test_oracle_brute_three_types_mixed_coefficients(orc):
    # c2 reading: prefactor sqrt(l_ij e_ij l_ik e_ik); checked only for consistency
    x, ty, box = _small_system(7, n=30, L=5.6, types=3)
    sw1 = dict(kind=2, eps=1.0, sigma=1.0, n=10, rcut=1.5, lambda3=1.5, rbond=1.2)
    sw2 = dict(kind=2, eps=2.0, sigma=0.9, n=8, rcut=1.4, lambda3=0.7, rbond=1.1)
    wca = dict(kind=1, eps=1.0, sigma=1.0, n=6)
    pairs = {(0, 1): sw1, (0, 2): sw2, (1, 2): wca, (0, 0): wca, (1, 1): wca, (2, 2): wca}
    tab = orc.pair_table(3, pairs)
    r = orc.forces(x, ty, 3, tab, box)
    b = brute(x, ty, pairs, box)
    assert r["U3"] == pytest.approx(b["U3"], rel=1e-12)
    np.testing.assert_allclose(r["F"], b["F"], rtol=1e-11, atol=1e-10)


@pytest.mark.parametrize("fp32", [False, True])
def test_oracle_nlist_matches_brute(orc, fp32):
    x, ty, box = _small_system(11, n=30, L=6.0)
    pairs = inputs.swap_pairs()
    tab = orc.pair_table(2, pairs)
    got = orc.nlist(x, ty, 2, tab, box, 0.3, fp32=fp32)
    ref = brute_nlist(x, ty, pairs, box, 0.3, fp32=fp32)
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)
    assert sum(len(a) for a in got) > 0


def test_oracle_cell_list_matches_all_pairs_at_scale(orc):
    # large enough for the 27-cell path; compared with a vectorised all-pairs search
    n = 1500
    box = inputs.cubic_box(n, 0.4)
    x = inputs.rsa_positions(n, box, 0.9, seed=3)
    ty = inputs.alternating_types(n)
    pairs = inputs.swap_pairs()
    tab = orc.pair_table(2, pairs)
    got = orc.nlist(x, ty, 2, tab, box, 0.3)
    d = x[:, None, :] - x[None, :, :]
    d -= box * np.round(d / box)
    r2 = (d[..., 0] ** 2 + d[..., 1] ** 2) + d[..., 2] ** 2
    cut = np.where(ty[:, None] != ty[None, :], 1.8, 2 ** (1 / 6) + 0.3)
    m = (r2 < cut * cut) & ~np.eye(n, dtype=bool)
    for i in range(n):
        np.testing.assert_array_equal(got[i], np.nonzero(m[i])[0])


# ---------------------------------------------------------------------------
# Finite differences, virial, invariants


def _far_from_kinks(x, box, pairs, ty, h):
    d = x[:, None, :] - x[None, :, :]
    d -= box * np.round(d / box)
    r = np.sqrt((d ** 2).sum(-1))
    iu = np.triu_indices(len(x), 1)
    rr = r[iu]
    kinks = [1.5, 2 ** 0.1, 2 ** (1 / 6)]
    return all(np.min(np.abs(rr - k)) > 50 * h for k in kinks)


@pytest.mark.parametrize("seed", [1, 2, 4])
@pytest.mark.parametrize("lam,shift", [(1.0, 0), (5.0, 1), (0.5, 0)])
def test_forces_are_minus_gradient(orc, seed, lam, shift):
    h = 1e-6
    for s in range(seed, seed + 50):
        x, ty, box = _small_system(s, n=30, L=5.6)
        pairs = inputs.swap_pairs(lambda3=lam, shift=shift)
        if _far_from_kinks(x, box, pairs, ty, h):
            break
    else:
        pytest.skip("no configuration away from the cut-off kinks")
    tab = orc.pair_table(2, pairs)
    r = orc.forces(x, ty, 2, tab, box)
    Fnum = np.zeros_like(x)
    for i in range(len(x)):
        for c in range(3):
            xp = x.copy()
            xp[i, c] += h
            xm = x.copy()
            xm[i, c] -= h
            up = orc.forces(xp, ty, 2, tab, box)
            um = orc.forces(xm, ty, 2, tab, box)
            Fnum[i, c] = -((up["U2"] + up["U3"]) - (um["U2"] + um["U3"])) / (2 * h)
    err = np.linalg.norm(Fnum - r["F"], axis=1)
    assert np.all(err <= 1e-6 * (r["fscale"] + 1.0))


def _cluster(seed, n=20):
    L = 40.0
    box = np.array([L, L, L])
    x = inputs.rsa_positions(n, np.array([4.0, 4.0, 4.0]), 0.85, seed=seed) + 18.0
    return x, (np.arange(n) % 2).astype(np.int32), box


@pytest.mark.parametrize("lam", [1.0, 3.0])
def test_virial_tensor_by_affine_deformation(orc, lam):
    x, ty, box = _cluster(3)
    pairs = inputs.swap_pairs(lambda3=lam, shift=1)
    tab = orc.pair_table(2, pairs)
    r = orc.forces(x, ty, 2, tab, box)
    assert r["U3"] != 0.0 or lam == 0
    Wfull = np.zeros((3, 3))
    idx = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (0, 1): 3, (0, 2): 4, (1, 2): 5}
    for (a, b), q in idx.items():
        Wfull[a, b] = Wfull[b, a] = r["W"][q]
    # W_ab = sum_i x_ia F_ib for an isolated cluster
    np.testing.assert_allclose(Wfull, x.T @ r["F"], rtol=1e-10, atol=1e-9)
    # and W_ab = -dU/d(delta) under x_b -> x_b + delta x_a
    h = 1e-7
    c = x.mean(0)
    for a in range(3):
        for b in range(3):
            def U(dl):
                y = x.copy()
                y[:, b] += dl * (x[:, a] - c[a])
                o = orc.forces(y, ty, 2, tab, box)
                return o["U2"] + o["U3"]
            num = -(U(h) - U(-h)) / (2 * h)
            assert num == pytest.approx(Wfull[a, b], rel=1e-5, abs=1e-5 * r["scale_W"])


def test_virial_trace_by_box_scaling(orc):
    x, ty, box = _small_system(5, n=30, L=5.6)
    pairs = inputs.swap_pairs(lambda3=2.0, shift=1)
    tab = orc.pair_table(2, pairs)
    r = orc.forces(x, ty, 2, tab, box)
    h = 1e-7

    def U(s):
        o = orc.forces(x * s, ty, 2, tab, box * s)
        return o["U2"] + o["U3"]

    trW = -(U(1 + h) - U(1 - h)) / (2 * h)
    assert trW == pytest.approx(r["W"][:3].sum(), rel=1e-5, abs=1e-6 * r["scale_W"])


def test_invariants(orc):
    x, ty, box = _cluster(8, n=24)
    pairs = inputs.swap_pairs(lambda3=1.0)
    tab = orc.pair_table(2, pairs)
    r = orc.forces(x, ty, 2, tab, box)
    scale = r["fscale"].sum()
    assert np.linalg.norm(r["F"].sum(0)) < 1e-13 * scale  # zero net force
    torque = np.cross(x - x.mean(0), r["F"]).sum(0)
    assert np.linalg.norm(torque) < 1e-12 * scale  # zero net torque (isolated)
    # permutation of the particle order leaves everything unchanged
    rng = np.random.default_rng(0)
    p = rng.permutation(len(x))
    rp = orc.forces(x[p], ty[p], 2, tab, box)
    assert rp["U2"] + rp["U3"] == pytest.approx(r["U2"] + r["U3"], rel=1e-14)
    np.testing.assert_allclose(rp["F"], r["F"][p], rtol=1e-12, atol=1e-12)
    assert rp["n_bonds"] == r["n_bonds"]


def test_single_bond_per_site_for_lambda_ge_1(orc):
    # a B with two A at the bond distance: with lambda >= 1 the triplet costs
    # eps (lambda - 1) >= 0 more than the dimer, so the pair prefers one bond
    for lam, sign in [(0.5, -1), (2.0, +1)]:
        tab, _ = three_body_table(orc, lam)
        rmin = 2 ** (1 / 10)
        x, ty, box = triad(rmin, rmin)
        both = orc.forces(x, ty, 2, tab, box)
        x, ty, box = triad(rmin, 2.5)
        one = orc.forces(x, ty, 2, tab, box)
        assert sign * ((both["U2"] + both["U3"]) - (one["U2"] + one["U3"])) > 0


# ---------------------------------------------------------------------------
# Integrators and the generator


def test_philox_known_answers(orc):
    with open(os.path.join(GOLD, "philox4x32_10_kat.txt")) as fh:
        rows = [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]
    for row in rows:
        v = [int(t, 16) for t in row if t != "->"]
        out = orc.philox4x32_10(v[0:4], v[4:6])
        assert list(out) == v[6:10]


def test_normals_statistics(orc):
    z = np.array([orc.normals3(42, s, t) for s in range(40) for t in range(100)]).ravel()
    assert abs(z.mean()) < 4 / math.sqrt(z.size)
    assert abs(z.var() - 1) < 6 * math.sqrt(2 / z.size)


def _nve_system(seed=3, n=256):
    box = inputs.cubic_box(n, 0.3)
    x = inputs.rsa_positions(n, box, 0.95, seed=seed)
    ty = inputs.alternating_types(n)
    v = inputs.maxwell_velocities(n, 0.1, 1.0, seed=seed)
    return x, v, ty, box


def test_nve_energy_conservation_scales_dt2(orc):
    x, v, ty, box = _nve_system()
    pairs = inputs.swap_pairs(lambda3=1.0, shift=1)
    tab = orc.pair_table(2, pairs)
    n = len(x)
    m = np.ones(n)
    tags = np.arange(n, dtype=np.uint32)
    flucts = []
    for dt, steps in [(0.002, 500), (0.001, 1000)]:
        _, _, _, th = orc.run(x, v, ty, m, tags, 2, tab, box, dt, steps)
        E = th[:, 0] + th[:, 1] + th[:, 2]
        flucts.append(np.abs(E - E[0]).max())
    # velocity Verlet: energy error O(dt^2)
    ratio = flucts[0] / flucts[1]
    assert 2.5 < ratio < 6.0, ratio
    assert flucts[1] / n < 2e-4  # per particle, n = 10 bonds at dt = 0.001


def test_nvt_equipartition(orc):
    # WCA fluid (single type, no bonding heat): BAOAB samples <K> = 3/2 N kT
    n = 1000
    box = inputs.cubic_box(n, 0.3)
    x = inputs.rsa_positions(n, box, 0.9, seed=9)
    ty = np.zeros(n, dtype=np.int32)
    v = np.zeros((n, 3))
    pairs = inputs.swap_pairs(lambda3=1.0)
    tab = orc.pair_table(2, pairs)
    kT = 0.1
    _, _, _, th = orc.run(x, v, ty, np.ones(n), np.arange(n, dtype=np.uint32), 2, tab, box,
                          0.002, 3000, kT=kT, gamma=1.0, seed=77)
    K = th[1000:, 2].mean()
    assert K == pytest.approx(1.5 * n * kT, rel=0.03)


def test_c9_force_scale_closed_forms(orc):
    """The second force scale (forces' size times the three-body factor they
    can receive) on isolated pairs: a WCA pair gives |dv/dr| to both ends; a
    reactive pair at r gives |dv/dr| (1 + lambda (vh(r) + vh(r))), with vh of
    Eq. pot; a pair beyond its cut-off gives nothing."""
    L = 20.0
    box = np.array([L, L, L])
    for kind, r, lam in (("wca", 1.05, 1.0), ("swap", 1.3, 1.0), ("swap", 1.3, 5.0), ("swap", 1.6, 1.0)):
        pairs = inputs.swap_pairs(lambda3=lam)
        tab = orc.pair_table(2, pairs)
        types = np.array([0, 0] if kind == "wca" else [0, 1], dtype=np.int32)
        x = np.array([[5.0, 5.0, 5.0], [5.0 + r, 5.0, 5.0]])
        c9 = orc.fscale_c9(x, types, 2, tab, box)
        if kind == "wca":
            n = 6
            want = abs(orc.dv2(r, n=n))
        elif r >= 1.5:
            want = 0.0
        else:
            vh = orc.vhat(r, eps=1.0, sigma=1.0, n=10, rcut=1.5, lambda3=lam)
            want = abs(orc.dv2(r, n=10)) * (1.0 + lam * 2.0 * vh)
        np.testing.assert_allclose(c9, [want, want], rtol=1e-13, atol=0.0)


def test_threaded_oracle_matches_one_thread(orc):
    """The OpenMP build (the all-cores CPU baseline) computes the same terms:
    equal to the one-thread oracle up to the grouping of the additions."""
    try:
        orc.build(openmp=True)
    except Exception as e:  # pragma: no cover - no OpenMP runtime here
        pytest.skip(f"no OpenMP build: {e}")
    wl = inputs.workload("mix2k", lambda3=5.0, n=3000, density=0.5, seed=5)
    tab = orc.pair_table(2, wl["pairs"])
    for fp32 in (False, True):
        a = orc.forces(wl["x"], wl["types"], 2, tab, wl["box"], fp32=fp32)
        b = orc.forces(wl["x"], wl["types"], 2, tab, wl["box"], fp32=fp32, threaded=True)
        assert np.all(np.linalg.norm(a["F"] - b["F"], axis=1) <= 1e-13 * a["fscale"])
        for q in ("U2", "U3"):
            assert abs(a[q] - b[q]) <= 1e-13 * a["scale_" + q]
        assert np.all(np.abs(a["W"] - b["W"]) <= 1e-13 * a["scale_W"])
        assert a["n_bonds"] == b["n_bonds"]
    xa, va, _, tha = orc.run(wl["x"], wl["v"], wl["types"], wl["mass"], wl["tags"], 2, tab, wl["box"], 0.001, 10,
                             kT=0.1, gamma=1.0, seed=3)
    xb, vb, _, thb = orc.run(wl["x"], wl["v"], wl["types"], wl["mass"], wl["tags"], 2, tab, wl["box"], 0.001, 10,
                             kT=0.1, gamma=1.0, seed=3, threaded=True)
    assert np.abs(xa - xb).max() <= 1e-11 and np.abs(va - vb).max() <= 1e-9


@pytest.mark.parametrize("gamma", [1.0, 4.0])
def test_langevin_friction_rate(orc, gamma):
    """The friction of the Langevin dynamics ("canonical Langevin", section
    "Self-assembly pitfalls"; Ornstein-Uhlenbeck velocity process): for a
    force-free particle dv = -gamma v dt + sqrt(2 gamma kT/m) dW, so the mean
    velocity from v(0) decays as exp(-gamma t) and the stationary variance is
    kT/m.  BAOAB (Leimkuhler & Matthews 2013) reproduces the decay exactly per
    step (B and A leave v alone without forces; O multiplies the mean by
    exp(-gamma dt)), so the sample mean over 3n components must equal
    exp(-gamma k dt) within its sampling error at every k.  A friction factor
    read as exp(-gamma dt / 2), or applied twice per step, fails by tens of
    standard errors.  Equipartition alone cannot tell: any factor keeps the
    Maxwell distribution stationary."""
    n, kT, dt = 2000, 0.05, 0.001
    box = np.array([50.0, 50.0, 50.0])
    x = inputs.rsa_positions(n, box, 0.9, seed=4)
    ty = np.zeros(n, dtype=np.int32)
    tab = orc.pair_table(1, {})  # no interaction at all
    tags = np.arange(n, dtype=np.uint32)
    v0 = np.ones((n, 3))
    for k in (50, 200, 500):
        _, v, _, th = orc.run(x, v0, ty, np.ones(n), tags, 1, tab, box, dt, k, kT=kT, gamma=gamma, seed=11)
        decay = math.exp(-gamma * k * dt)
        sem = math.sqrt((1.0 - decay ** 2) * kT / (3 * n))
        assert abs(v.mean() - decay) < 5.0 * sem, (k, v.mean(), decay, sem)
        # the variance about the mean: (1 - exp(-2 gamma t)) kT / m
        var = (1.0 - decay ** 2) * kT
        assert v.var() == pytest.approx(var, rel=0.1)
        assert np.all(th[:, 0] == 0.0) and np.all(th[:, 1] == 0.0)
    # long after the start: the stationary velocity variance kT / m
    _, v, _, _ = orc.run(x, v0, ty, np.ones(n), tags, 1, tab, box, dt, int(round(6.0 / (gamma * dt))),
                         kT=kT, gamma=gamma, seed=12)
    assert v.var() == pytest.approx(kT, rel=0.06)


def test_nvt_uses_tag_keyed_noise(orc):
    # the Langevin noise depends on (seed, step, tag) only: permuting storage order
    # with the tags permuted alongside gives the same trajectory
    x, v, ty, box = _nve_system(n=64)
    pairs = inputs.swap_pairs()
    tab = orc.pair_table(2, pairs)
    n = len(x)
    tags = np.arange(n, dtype=np.uint32)
    p = np.random.default_rng(1).permutation(n)
    a = orc.run(x, v, ty, np.ones(n), tags, 2, tab, box, 0.001, 5, kT=0.1, gamma=1.0, seed=3)
    b = orc.run(x[p], v[p], ty[p], np.ones(n), tags[p], 2, tab, box, 0.001, 5, kT=0.1, gamma=1.0,
                seed=3)
    np.testing.assert_allclose(b[0], a[0][p], rtol=0, atol=1e-12)


def test_inputs_recipe():
    box = inputs.cubic_box(5000, 0.5)
    x = inputs.rsa_positions(5000, box, 0.9, seed=1)
    assert np.all(x >= 0) and np.all(x < box)
    assert np.array_equal(x, inputs.f32(x))
    d = x[:, None, :] - x[None, :, :]
    d -= box * np.round(d / box)
    r2 = (d ** 2).sum(-1) + np.eye(len(x)) * 100
    assert r2.min() >= 0.9 ** 2 * (1 - 1e-6)
    assert box[0] == float(np.float32(box[0]))
    ty = inputs.alternating_types(5000)
    assert (ty == 0).sum() == 2500


# ---------------------------------------------------------------------------
# Harmonic bonds (the vitrimer network's chains): u = k/2 (r - r0)^2.

def test_single_bond_closed_form(orc):
    box = np.array([20.0, 20.0, 20.0])
    x = np.array([[5.0, 5.0, 5.0], [6.3, 5.0, 5.0]])
    ty = np.array([0, 0], dtype=np.int32)
    pairs = {(0, 0): dict(kind=0)}  # no pair interaction: the bond alone
    tab = orc.pair_table(1, {(0, 0): dict(kind=0, eps=1.0, sigma=1.0, n=6)})
    r = orc.forces(x, ty, 1, tab, box, bonds=[[0, 1]], kbond=100.0, r0=1.0)
    assert r["U_bond"] == pytest.approx(0.5 * 100.0 * 0.3 ** 2, rel=1e-14)
    # stretched bond pulls the two together: F_0 along +x, F_1 along -x
    np.testing.assert_allclose(r["F"], [[30.0, 0, 0], [-30.0, 0, 0]], rtol=1e-13, atol=1e-12)
    assert r["W"][0] == pytest.approx(-30.0 * 1.3, rel=1e-13)  # r_ij F_ij with r_ij = -1.3, F = +30
    del pairs


def test_bonded_chain_forces_are_minus_gradient(orc):
    """Chains bonded along the tags, with the swap and WCA pair terms: forces by
    central differences of the total energy."""
    h = 1e-6
    for s in range(10, 60):
        x, ty, box = _small_system(s, n=30, L=5.6)
        pairs = inputs.swap_pairs(lambda3=1.0, shift=1)
        if _far_from_kinks(x, box, pairs, ty, h):
            break
    else:
        pytest.skip("no configuration away from the cut-off kinks")
    bonds = [[i, i + 1] for i in range(0, 29) if i % 10 != 9]  # three chains of 10
    tab = orc.pair_table(2, pairs)
    kw = dict(bonds=bonds, kbond=100.0, r0=1.0)
    r = orc.forces(x, ty, 2, tab, box, **kw)
    assert r["U_bond"] > 0.0
    Fnum = np.zeros_like(x)
    for i in range(len(x)):
        for c in range(3):
            xp = x.copy()
            xp[i, c] += h
            xm = x.copy()
            xm[i, c] -= h
            up = orc.forces(xp, ty, 2, tab, box, **kw)
            um = orc.forces(xm, ty, 2, tab, box, **kw)
            Fnum[i, c] = -((up["U2"] + up["U3"] + up["U_bond"]) - (um["U2"] + um["U3"] + um["U_bond"])) / (2 * h)
    err = np.linalg.norm(Fnum - r["F"], axis=1)
    assert np.all(err <= 1e-6 * (r["fscale"] + 1.0))
    assert np.linalg.norm(r["F"].sum(0)) < 1e-10 * r["fscale"].sum()


def test_bonded_virial_trace_by_box_scaling(orc):
    x, ty, box = _small_system(5, n=30, L=5.6)
    pairs = inputs.swap_pairs(lambda3=2.0, shift=1)
    tab = orc.pair_table(2, pairs)
    kw = dict(bonds=[[i, i + 1] for i in range(29)], kbond=100.0, r0=1.0)
    r = orc.forces(x, ty, 2, tab, box, **kw)
    h = 1e-7

    def U(s):
        o = orc.forces(x * s, ty, 2, tab, box * s, **kw)
        return o["U2"] + o["U3"] + o["U_bond"]

    trW = -(U(1 + h) - U(1 - h)) / (2 * h)
    assert trW == pytest.approx(r["W"][:3].sum(), rel=1e-5, abs=1e-6 * r["scale_W"])


def test_bonded_nve_conserves_energy(orc):
    """Velocity Verlet with bonds: the total energy including the bonds drifts
    like dt^2."""
    x, ty, box = _small_system(7, n=30, L=5.6)
    pairs = inputs.swap_pairs(lambda3=1.0, shift=1)
    tab = orc.pair_table(2, pairs)
    kw = dict(bonds=[[i, i + 1] for i in range(0, 29) if i % 10 != 9], kbond=100.0, r0=1.0)
    rng = np.random.default_rng(3)
    v0 = rng.standard_normal((30, 3)) * 0.3
    m = np.ones(30)
    tags = np.arange(30, dtype=np.uint32)
    drift = []
    for dt in (0.002, 0.001):
        n = int(round(0.4 / dt))
        xo, vo, _, th = orc.run(x, v0, ty, m, tags, 2, tab, box, dt, n, **kw)
        E = th[:, 0] + th[:, 1] + th[:, 2] + th[:, 10]
        r0 = orc.forces(x, ty, 2, tab, box, **kw)
        E0 = r0["U2"] + r0["U3"] + r0["U_bond"] + 0.5 * (v0 ** 2).sum()
        drift.append(np.max(np.abs(E - E0)))
    assert drift[1] < drift[0] / 3.0  # second order in dt
    # the random configuration starts with stretched bonds (violent motion): a loose bound
    assert drift[1] < 5e-3 * abs(E0)
