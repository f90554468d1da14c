"""The host-side analysis of the swap-dynamics validation, on synthetic data
with known answers (CPU): bonds found across the periodic faces, the bond
autocorrelation of a known replacement pattern, and the relaxation time of an
exact exponential."""
import numpy as np
import pytest

from paper_1912_08569_gb300 import validation as V


def test_bond_pairs_include_periodic_images():
    pytest.importorskip("scipy")
    box = np.array([10.0, 10.0, 10.0])
    x = np.array([[0.2, 5.0, 5.0],    # A 0
                  [9.7, 5.0, 5.0],    # B 1: 0.5 from A 0 through the x face
                  [5.0, 5.0, 5.0],    # A 2
                  [5.0, 6.1, 5.0],    # B 3: 1.1 from A 2, outside rbond 1.0
                  [5.0, 5.0, 9.9],    # A 4
                  [5.0, 5.0, 0.3]])   # B 5: 0.4 from A 4 through the z face
    types = np.array([0, 1, 0, 1, 0, 1])
    got = V.bond_pairs(x, types, box, 1.0)
    assert got == {(1, 0), (5, 4)}
    # brute force over all A-B pairs with the minimum image
    want = set()
    for b in np.nonzero(types == 1)[0]:
        for a in np.nonzero(types == 0)[0]:
            d = x[b] - x[a]
            d -= box * np.round(d / box)
            if np.linalg.norm(d) < 1.0:
                want.add((int(b), int(a)))
    assert got == want


def test_autocorrelation_of_a_known_replacement_pattern():
    # four bonds, one replaced per sample: sets {k, .., k+3}; after `lag` samples
    # 4 - lag of the origin's bonds remain, for every origin
    sets = [{(k + m, 0) for m in range(4)} for k in range(12)]
    c = V.autocorrelation(sets, 5)
    np.testing.assert_allclose(c, [1.0, 0.75, 0.5, 0.25, 0.0, 0.0], rtol=0, atol=1e-15)


def test_autocorrelation_counts_presence_not_persistence():
    # a bond that breaks and comes back counts as present again (the reading
    # taken for "still unswapped")
    sets = [{(1, 0)}, set(), {(1, 0)}]
    c = V.autocorrelation(sets, 2)
    assert c[0] == 1.0 and c[2] == 1.0


def test_fit_tau_recovers_an_exponential():
    t = np.arange(0, 400.0)
    tau, r2 = V.fit_tau(t, np.exp(-t / 57.0))
    assert tau == pytest.approx(57.0, rel=1e-12)
    assert r2 == pytest.approx(1.0, abs=1e-12)
    # points below c = 0.05 are left out of the fit
    c = np.exp(-t / 57.0)
    c[t > 200] = 1e-3 * (1 + np.sin(t[t > 200]))
    tau2, _ = V.fit_tau(t, c)
    assert tau2 == pytest.approx(57.0, rel=1e-12)
