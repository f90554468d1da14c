"""FP64 CPU oracle for the associative bond-swap potential (test infrastructure).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product package never imports it, and it imports nothing from the product.

The arithmetic lives in ``swap_oracle.c`` (plain C, FP64, built with
``-ffp-contract=off``); this module compiles it on first use and wraps it with
ctypes.  What each function computes, with the passage of the paper it
follows:

* ``pair_energy`` / ``vhat``: Eq. 2b (generalised Lennard-Jones) and Eq. pot
  (the normalised two-body term, 1 inside r_min = sigma 2^(1/n)).
* ``forces``: U = sum of two-body terms + Eq. 3bp summed over every centre and
  every unordered pair of its reactive partners (an explicit triplet loop),
  forces as -dU/dx, virial as in Eq. p3, bond count.
* ``nlist``: neighbour-list membership for a given skin (the set every valid
  Verlet list built from a cell list must contain, and nothing more).
* ``forces(..., bonds=...)`` / ``run(..., bonds=...)``: harmonic bonds
  k/2 (r - r0)^2 of a fixed topology added to the pair terms (the chains of the
  vitrimer network; the paper does not give the form, the harmonic one with
  k = 100, r0 = 1 is this build's configuration).
* ``run``: velocity Verlet (NVE) or BAOAB Langevin (NVT; the paper's
  "canonical Langevin dynamics" of section "Self-assembly pitfalls").
* ``philox4x32_10`` / ``normals3``: the counter-based generator of Salmon et al.
  (SC'11) and its Box-Muller normals, used for the Langevin noise.
* ``forces(..., threaded=True)`` / ``run(..., threaded=True)``: the same code
  built with OpenMP over every host core (OMP_NUM_THREADS), for the
  benchmark's all-cores CPU baseline; the additions are grouped per thread, so
  results agree with the one-thread build to rounding, not bit for bit.

Parity pins for every function are in ``tests/test_oracle_*.py``.  The
mixed-coefficient triplet prefactor sqrt(l_ij e_ij l_ik e_ik) is a reading of
the paper (it states only lambda*eps for one reactive pair type): parity
unpinned beyond agreement with the brute-force triple sum.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "swap_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_swap.so")
# the same source built with -fopenmp: the all-cores CPU baseline of the
# benchmark (same terms; the additions are grouped per thread)
_LIB_OMP = os.path.join(_HERE, "liboracle_swap_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

KIND_NONE, KIND_WCA, KIND_SWAP = 0, 1, 2

PAIR_DTYPE = np.dtype(
    [
        ("kind", np.int32),
        ("n", np.int32),
        ("shift", np.int32),
        ("pad", np.int32),
        ("eps", np.float64),
        ("sigma", np.float64),
        ("lambda3", np.float64),
        ("rcut", np.float64),
        ("rbond", np.float64),
    ]
)


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile ``swap_oracle.c`` into ``liboracle_swap.so`` (gcc, FP64, no
    contraction); with openmp, into ``liboracle_swap_omp.so`` with -fopenmp."""
    lib = _LIB_OMP if openmp else _LIB
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", *(["-fopenmp"] if openmp else []), "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, lib)
    return lib


def _load(threaded: bool = False):
    global _lib, _lib_omp
    with _lock:
        if (_lib_omp if threaded else _lib) is None:
            path = build(openmp=threaded)
            lib = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            up = ctypes.POINTER(ctypes.c_uint32)
            vp = ctypes.c_void_p
            lib.orc_forces.argtypes = [ctypes.c_int, dp, ip, ctypes.c_int, vp, dp, ctypes.c_int,
                                       dp, dp, dp, dp]
            lib.orc_forces.restype = ctypes.c_int
            lib.orc_nlist.argtypes = [ctypes.c_int, dp, ip, ctypes.c_int, vp, dp, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_int, ip, ip]
            lib.orc_nlist.restype = ctypes.c_int
            lib.orc_bonds.argtypes = [ctypes.c_int, dp, dp, ctypes.c_long, ip, ctypes.c_double, ctypes.c_double,
                                      dp, dp, dp, dp]
            lib.orc_bonds.restype = None
            lib.orc_run.argtypes = [ctypes.c_int, dp, dp, ip, ip, dp, up, ctypes.c_int, vp, dp,
                                    ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64, dp, ctypes.c_long, ip,
                                    ctypes.c_double, ctypes.c_double]
            lib.orc_run.restype = ctypes.c_int
            lib.orc_v2.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int]
            lib.orc_v2.restype = ctypes.c_double
            lib.orc_dv2.argtypes = lib.orc_v2.argtypes
            lib.orc_dv2.restype = ctypes.c_double
            lib.orc_vhat.argtypes = [vp, ctypes.c_double]
            lib.orc_vhat.restype = ctypes.c_double
            lib.orc_u2.argtypes = [vp, ctypes.c_double]
            lib.orc_u2.restype = ctypes.c_double
            lib.orc_philox4x32_10.argtypes = [up, up, up]
            lib.orc_philox4x32_10.restype = None
            lib.orc_normals3.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                         ctypes.c_uint32, dp]
            lib.orc_normals3.restype = None
            lib.orc_fscale_c9.argtypes = [ctypes.c_int, dp, ip, ctypes.c_int, vp, dp, ctypes.c_int, dp]
            lib.orc_fscale_c9.restype = ctypes.c_int
            lib.orc_threads.argtypes = []
            lib.orc_threads.restype = ctypes.c_int
            if threaded:
                _lib_omp = lib
            else:
                _lib = lib
    return _lib_omp if threaded else _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def pair_table(ntypes: int, entries: dict) -> np.ndarray:
    """Symmetric (ntypes*ntypes) table from {(ti, tj): dict(kind=..., ...)}."""
    tab = np.zeros(ntypes * ntypes, dtype=PAIR_DTYPE)
    for (a, b), p in entries.items():
        for (i, j) in ((a, b), (b, a)):
            t = tab[i * ntypes + j]
            t["kind"] = p.get("kind", KIND_NONE)
            t["n"] = p.get("n", 6)
            t["shift"] = p.get("shift", 0)
            t["eps"] = p.get("eps", 1.0)
            t["sigma"] = p.get("sigma", 1.0)
            t["lambda3"] = p.get("lambda3", 0.0)
            t["rcut"] = p.get("rcut", 0.0)
            t["rbond"] = p.get("rbond", 0.0)
            tab[i * ntypes + j] = t
    return tab


def _single(p: dict) -> np.ndarray:
    return pair_table(1, {(0, 0): p})


def v2(r: float, eps: float = 1.0, sigma: float = 1.0, n: int = 10) -> float:
    """Eq. 2b without cut-off."""
    return _load().orc_v2(float(r), float(eps), float(sigma), int(n))


def dv2(r: float, eps: float = 1.0, sigma: float = 1.0, n: int = 10) -> float:
    """d/dr of Eq. 2b."""
    return _load().orc_dv2(float(r), float(eps), float(sigma), int(n))


def vhat(r: float, **pair) -> float:
    """Eq. pot for one swap pair type (0 at and beyond r_cut)."""
    t = _single(dict(pair, kind=KIND_SWAP))
    return _load().orc_vhat(t.ctypes.data, float(r))


def u2(r: float, **pair) -> float:
    """Two-body energy of one pair type with its cut-off."""
    t = _single(pair)
    return _load().orc_u2(t.ctypes.data, float(r))


def _bond_arrays(bonds):
    if bonds is None or len(bonds) == 0:
        return 0, np.zeros(2, dtype=np.int32)
    b = np.ascontiguousarray(bonds, dtype=np.int32).reshape(-1, 2)
    return b.shape[0], b


def forces(x, types, ntypes, table, box, fp32: bool = False, bonds=None, kbond: float = 0.0,
           r0: float = 1.0, threaded: bool = False):
    """Energies, forces, virial and bond count of a configuration.

    Returns a dict with U2, U3, W (6: xx yy zz xy xz yz), n_bonds, F (n x 3),
    scale_U2, scale_U3, scale_W and fscale (n) -- the error scales used by the
    parity tolerances (sum of |term| + r |d term / dr| over the terms summed).
    bonds ([m, 2] indices): harmonic bonds k/2 (r - r0)^2 added to F, W and
    their scales; their energy is returned as U_bond (0 without bonds).
    """
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    n = x.shape[0]
    ty = np.ascontiguousarray(types, dtype=np.int32)
    box = np.ascontiguousarray(box, dtype=np.float64)
    tab = np.ascontiguousarray(table, dtype=PAIR_DTYPE)
    F = np.zeros((max(n, 1), 3))
    out = np.zeros(9)
    sc = np.zeros(3)
    fs = np.zeros(max(n, 1))
    rc = _load(threaded).orc_forces(n, _dp(x), _ip(ty), int(ntypes), tab.ctypes.data, _dp(box),
                            int(bool(fp32)), _dp(F), _dp(out), _dp(sc), _dp(fs))
    if rc != 0:
        raise MemoryError("oracle: allocation failed")
    nb, b = _bond_arrays(bonds)
    ub, sub = 0.0, 0.0
    if nb:
        ob = np.zeros(7)
        sb = np.zeros(2)
        _load().orc_bonds(n, _dp(x), _dp(box), nb, _ip(b), float(kbond), float(r0), _dp(F), _dp(ob), _dp(fs),
                          _dp(sb))
        out[2:8] += ob[1:7]
        ub, sub = ob[0], sb[0]
        sc[2] += sb[1]
    return dict(U2=out[0], U3=out[1], W=out[2:8].copy(), n_bonds=int(round(out[8])),
                F=F[:n].copy(), scale_U2=sc[0], scale_U3=sc[1], scale_W=sc[2],
                fscale=fs[:n].copy(), U_bond=ub, scale_Ub=sub)


def fscale_c9(x, types, ntypes, table, box, fp32: bool = False):
    """Per-particle sum over interacting pairs of |du2/dr| (1 + lambda (S_i + S_j))
    (reactive) or |du2/dr| (others): the size of the forces, without the
    distance-sensitivity term of forces()["fscale"]."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    n = x.shape[0]
    ty = np.ascontiguousarray(types, dtype=np.int32)
    box = np.ascontiguousarray(box, dtype=np.float64)
    tab = np.ascontiguousarray(table, dtype=PAIR_DTYPE)
    out = np.zeros(max(n, 1))
    if _load().orc_fscale_c9(n, _dp(x), _ip(ty), int(ntypes), tab.ctypes.data, _dp(box), int(bool(fp32)),
                             _dp(out)) != 0:
        raise MemoryError("oracle: allocation failed")
    return out[:n]


def nlist(x, types, ntypes, table, box, skin: float, fp32: bool = False, maxn: int = 256):
    """Per-particle sorted neighbour sets within r_cut(ti,tj) + skin."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    n = x.shape[0]
    ty = np.ascontiguousarray(types, dtype=np.int32)
    box = np.ascontiguousarray(box, dtype=np.float64)
    tab = np.ascontiguousarray(table, dtype=PAIR_DTYPE)
    counts = np.zeros(max(n, 1), dtype=np.int32)
    nbr = np.zeros(max(n, 1) * maxn, dtype=np.int32)
    mx = _load().orc_nlist(n, _dp(x), _ip(ty), int(ntypes), tab.ctypes.data, _dp(box),
                           int(bool(fp32)), float(skin), int(maxn), _ip(counts), _ip(nbr))
    if mx < 0:
        raise MemoryError("oracle: allocation failed")
    if mx > maxn:
        return nlist(x, types, ntypes, table, box, skin, fp32, maxn=mx)
    nbr = nbr.reshape(-1, maxn)
    return [nbr[i, :counts[i]].copy() for i in range(n)]


def run(x, v, types, mass, tags, ntypes, table, box, dt, nsteps, kT=0.0, gamma=0.0,
        seed=0, step0=0, fp32=False, img=None, bonds=None, kbond=0.0, r0=1.0, threaded=False):
    """Advance (x, v) by nsteps (BAOAB if gamma > 0, else velocity Verlet).

    Returns (x, v, img, thermo) with thermo[s] = [U2, U3, K, W(6), n_bonds,
    U_bond] (W includes the bonds' virial).
    """
    x = np.array(x, dtype=np.float64).reshape(-1, 3)
    v = np.array(v, dtype=np.float64).reshape(-1, 3)
    n = x.shape[0]
    im = np.zeros((n, 3), dtype=np.int32) if img is None else np.array(img, dtype=np.int32)
    ty = np.ascontiguousarray(types, dtype=np.int32)
    m = np.ascontiguousarray(mass, dtype=np.float64)
    tg = np.ascontiguousarray(tags, dtype=np.uint32)
    box = np.ascontiguousarray(box, dtype=np.float64)
    tab = np.ascontiguousarray(table, dtype=PAIR_DTYPE)
    th = np.zeros((max(nsteps, 1), 11))
    nb, b = _bond_arrays(bonds)
    rc = _load(threaded).orc_run(n, _dp(x), _dp(v), _ip(im), _ip(ty), _dp(m),
                         tg.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), int(ntypes),
                         tab.ctypes.data, _dp(box), int(bool(fp32)), float(dt), int(nsteps),
                         float(kT), float(gamma), int(seed), int(step0), _dp(th), nb, _ip(b), float(kbond),
                         float(r0))
    if rc != 0:
        raise MemoryError("oracle: allocation failed")
    return x, v, im, th[:nsteps]


def threads(threaded: bool = True) -> int:
    """Threads the (threaded) build's force sums use."""
    return int(_load(threaded).orc_threads())


def philox4x32_10(ctr, key):
    """Philox4x32-10 block function (Salmon et al., SC'11)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    p = ctypes.POINTER(ctypes.c_uint32)
    _load().orc_philox4x32_10(c.ctypes.data_as(p), k.ctypes.data_as(p), o.ctypes.data_as(p))
    return o


def normals3(seed: int, step: int, tag: int, purpose: int = 1):
    """Three Box-Muller normals for (seed, step, tag, purpose)."""
    z = np.zeros(3)
    _load().orc_normals3(int(seed), int(step), int(tag), int(purpose), _dp(z))
    return z
