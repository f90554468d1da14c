"""Shared helpers of the GPU parity tests: build systems on both sides from the
same seeded inputs and compare with the tolerances derived from the arithmetic.

Tolerances (FP32 path: 1e-5; FP64 path: 1e-12), relative to the error scale
the oracle returns for each quantity: for a force, the sum over every term
acting on the particle of |term| + r |d term / dr| -- the size of what is
summed plus its first-order sensitivity to a relative perturbation of the
distances, which is what FP32 rounding of distances and of the terms produces.
"""
import numpy as np

TOL = {"fp32": 1e-5, "fp64": 1e-12}


def oracle_pairs(orc, wl):
    return orc.pair_table(wl["n_types"], wl["pairs"])


def make_gpu(wl, precision="fp32", **kw):
    from paper_1912_08569_gb300 import SwapSystem

    s = SwapSystem(wl["n"], wl["n_types"], wl["box"], wl["pairs"], precision=precision,
                   seed=wl.get("seed", 0), skin=wl.get("skin", 0.3), **kw)
    s.set_state(wl["x"], wl.get("v"), wl["types"], wl.get("mass"))
    return s


def assert_forces_match(F, ref, tol, what=""):
    err = np.linalg.norm(F - ref["F"], axis=1)
    bound = tol * ref["fscale"]
    bad = np.nonzero(err > bound)[0]
    assert len(bad) == 0, (
        f"{what}: {len(bad)} particles out of tolerance; worst err/scale = "
        f"{np.max(err / np.maximum(ref['fscale'], 1e-300)):.3e} at {bad[:5]}")


def assert_thermo_match(th, ref, tol, what=""):
    assert abs(th["U2"] - ref["U2"]) <= tol * ref["scale_U2"], (what, th["U2"], ref["U2"])
    assert abs(th["U3"] - ref["U3"]) <= tol * ref["scale_U3"], (what, th["U3"], ref["U3"])
    np.testing.assert_array_less(np.abs(th["W"] - ref["W"]), tol * ref["scale_W"] + 1e-300)
    assert th["n_bonds"] == ref["n_bonds"], (what, th["n_bonds"], ref["n_bonds"])
