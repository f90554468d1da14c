"""Seeded input generators (no arithmetic of the method): the cell-accelerated
minimum-separation check gives the same answer as a check against every
point, so the dumbbell mixture does not depend on how the check is done."""
import numpy as np

from paper_1912_08569_gb300 import inputs


def _far_brute(c, pts, box, dmin):
    if len(pts) == 0:
        return True
    d = np.asarray(pts) - c
    d -= box * np.round(d / box)
    return np.min(np.sum(d * d, axis=1)) >= dmin * dmin


def test_separation_grid_matches_all_points():
    rng = np.random.default_rng(7)
    for box in (np.array([9.3, 9.3, 9.3]), np.array([12.0, 7.5, 10.25]), np.array([2.5, 2.5, 2.5])):
        g = inputs._SeparationGrid(box, 1.0)
        pts = []
        for _ in range(600):
            c = rng.random(3) * box
            if rng.random() < 0.3:  # near a face: the periodic images matter
                k = rng.integers(3)
                c[k] = box[k] * (1.0 - 1e-3 * rng.random())
            want = _far_brute(c, pts, box, 1.0)
            assert g.far(c) == want
            if want:
                g.add(c)
                pts.append(c)
        assert np.array_equal(g.points(), np.array(pts).reshape(-1, 3))


def test_dumbbell_workload_recipe():
    wl = inputs.dumbbell_workload(seed=3, n_a=300, n_b=200, rcut=1.15)
    x, ty, box = wl["x"], wl["types"], wl["box"]
    assert wl["n"] == 500 and (ty == 0).sum() == 300 and (ty == 1).sum() == 200
    assert np.all(x >= 0) and np.all(x < box)
    rmin = 2.0 ** (1.0 / 100)
    # every B sits at r_min from its own A (the pair laid down just before it)
    for b in np.nonzero(ty == 1)[0]:
        d = x[b] - x[b - 1]
        d -= box * np.round(d / box)
        assert ty[b - 1] == 0 and abs(np.linalg.norm(d) - rmin) < 1e-5
    # everything else at least 1.0 apart
    d = x[:, None, :] - x[None, :, :]
    d -= box * np.round(d / box)
    r = np.sqrt((d * d).sum(-1)) + 10 * np.eye(len(x))
    pair = np.zeros_like(r, dtype=bool)
    for b in np.nonzero(ty == 1)[0]:
        pair[b, b - 1] = pair[b - 1, b] = True
    assert r[~pair].min() >= 1.0 - 1e-9
    assert wl["pairs"][(0, 1)]["rcut"] == 1.15
