"""ctypes binding of the C-ABI in ``include/swapmd.h``: argument marshalling only.

Every function here has the name of the C entry point it calls and raises
``SwpError`` on a negative status.  No arithmetic of the method happens in
Python: every step of the path runs in the CUDA kernels of ``libswapmd.so``.
The library must be built (``paper_1912_08569_gb300.build.build()``); loading
fails loudly otherwise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libswapmd.so")

SWP_OK = 0
SWP_ERR_INVALID = -1
SWP_ERR_CUDA = -2
SWP_ERR_NLIST_OVERFLOW = -3
SWP_ERR_TIMEOUT = -4
SWP_ERR_STATE = -5
SWP_ERR_NONFINITE = -6

SWP_FP32 = 0
SWP_FP64 = 1
SWP_PAIR_NONE = 0
SWP_PAIR_WCA = 1
SWP_PAIR_SWAP = 2
SWP_HOST = 0
SWP_DEVICE = 1

ERROR_NAMES = {
    SWP_ERR_INVALID: "SWP_ERR_INVALID",
    SWP_ERR_CUDA: "SWP_ERR_CUDA",
    SWP_ERR_NLIST_OVERFLOW: "SWP_ERR_NLIST_OVERFLOW",
    SWP_ERR_TIMEOUT: "SWP_ERR_TIMEOUT",
    SWP_ERR_STATE: "SWP_ERR_STATE",
    SWP_ERR_NONFINITE: "SWP_ERR_NONFINITE",
}

# Every entry point declared in include/swapmd.h.
EXPORTS = (
    "swp_abi_version", "swp_create", "swp_set_pair", "swp_set_nlist", "swp_workspace_size",
    "swp_nlist_size", "swp_bind_workspace", "swp_bind_nlist", "swp_set_state", "swp_set_step",
    "swp_build_nlist", "swp_compute_forces", "swp_step_nve", "swp_step_nvt", "swp_sync",
    "swp_read_thermo", "swp_read_forces", "swp_read_state", "swp_read_nlist", "swp_set_launch", "swp_set_grid",
    "swp_set_timeout", "swp_last_error", "swp_destroy", "swp_compute_forces_static",
    "swp_batch_workspace_size", "swp_batch_step", "swp_param_grad", "swp_set_bonds", "swp_set_resident",
    "swp_set_withhold_arrival", "swp_thermo_log_bytes", "swp_set_thermo_log", "swp_thermo_log", "swp_eval_grad",
    "swp_batch_plan",
)


class SwpError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        self.code = code
        super().__init__(f"{where}: {ERROR_NAMES.get(code, code)}: {msg}")


class swp_thermo(ctypes.Structure):
    _fields_ = [
        ("U2", ctypes.c_double),
        ("U3", ctypes.c_double),
        ("K", ctypes.c_double),
        ("W", ctypes.c_double * 6),
        ("n_bonds", ctypes.c_int64),
        ("step", ctypes.c_int64),
        ("n_rebuilds", ctypes.c_int64),
        ("steps_done", ctypes.c_int64),
        ("max_row", ctypes.c_int32),
        ("state", ctypes.c_int32),
        ("resident_steps", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libswapmd.so (built in-tree); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"CUDA library not built: {path} is missing; run paper_1912_08569_gb300.build.build()")
    lib = ctypes.CDLL(path)
    c_int, c_double, c_void_p, c_size_t = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
    P = ctypes.POINTER
    sig = {
        "swp_abi_version": ([], c_int),
        "swp_create": ([P(c_void_p), c_int, c_int, P(c_double), c_int, ctypes.c_uint64], c_int),
        "swp_set_pair": ([c_void_p, c_int, c_int, c_int, c_double, c_double, c_int, c_double, c_double,
                          c_int, c_double], c_int),
        "swp_set_nlist": ([c_void_p, c_double, c_int], c_int),
        "swp_workspace_size": ([c_void_p, P(c_size_t)], c_int),
        "swp_nlist_size": ([c_void_p, P(c_size_t)], c_int),
        "swp_bind_workspace": ([c_void_p, c_void_p, c_size_t, c_void_p], c_int),
        "swp_bind_nlist": ([c_void_p, c_void_p, c_size_t], c_int),
        "swp_set_state": ([c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int], c_int),
        "swp_set_step": ([c_void_p, ctypes.c_int64], c_int),
        "swp_build_nlist": ([c_void_p], c_int),
        "swp_compute_forces": ([c_void_p], c_int),
        "swp_step_nve": ([c_void_p, c_double, c_int], c_int),
        "swp_step_nvt": ([c_void_p, c_double, c_double, c_double, c_int], c_int),
        "swp_sync": ([c_void_p], c_int),
        "swp_read_thermo": ([c_void_p, P(swp_thermo)], c_int),
        "swp_read_forces": ([c_void_p, c_void_p, c_int], c_int),
        "swp_read_state": ([c_void_p, c_void_p, c_void_p, c_void_p, c_int], c_int),
        "swp_read_nlist": ([c_void_p, c_void_p, c_void_p, c_int], c_int),
        "swp_set_launch": ([c_void_p, c_int], c_int),
        "swp_set_grid": ([c_void_p, c_int], c_int),
        "swp_set_timeout": ([c_void_p, ctypes.c_int64], c_int),
        "swp_set_resident": ([c_void_p, c_int], c_int),
        "swp_set_withhold_arrival": ([c_void_p, c_int], c_int),
        "swp_thermo_log_bytes": ([c_void_p, ctypes.c_int64], c_size_t),
        "swp_set_thermo_log": ([c_void_p, c_int, ctypes.c_int64, c_void_p, c_size_t], c_int),
        "swp_thermo_log": ([c_void_p, c_void_p, c_void_p, ctypes.c_int64, P(ctypes.c_int64)], c_int),
        "swp_eval_grad": ([c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                           c_void_p], c_int),
        "swp_last_error": ([c_void_p], ctypes.c_char_p),
        "swp_destroy": ([c_void_p], c_int),
        "swp_compute_forces_static": ([c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p], c_int),
        "swp_param_grad": ([c_void_p, c_int, c_int, P(c_double), c_void_p], c_int),
        "swp_set_bonds": ([c_void_p, c_int, c_void_p, c_double, c_double], c_int),
        "swp_batch_workspace_size": ([c_int], c_size_t),
        "swp_batch_step": ([P(c_void_p), c_int, P(c_double), P(c_double), P(c_double), c_int, c_double,
                            c_int, c_void_p, c_size_t], c_int),
        "swp_batch_plan": ([P(ctypes.c_longlong), c_int, c_int, c_double, c_int, c_int, P(c_int), P(c_int),
                            P(c_int)], c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(ctx, rc: int, where: str):
    if rc < 0:
        msg = load_library().swp_last_error(ctx)
        raise SwpError(rc, where, (msg or b"").decode(errors="replace"))
    return rc


def _ptr(a):
    """Address of a numpy array / torch tensor (or None)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def swp_abi_version() -> int:
    return load_library().swp_abi_version()


def swp_create(n: int, n_types: int, box, precision: int, seed: int):
    lib = load_library()
    ctx = ctypes.c_void_p()
    b = (ctypes.c_double * 3)(*[float(v) for v in box])
    rc = lib.swp_create(ctypes.byref(ctx), int(n), int(n_types), b, int(precision), int(seed))
    if rc < 0:
        raise SwpError(rc, "swp_create", "cannot create context (bad sizes or no CUDA device)")
    return ctx


def swp_set_pair(ctx, ti, tj, kind, eps=1.0, sigma=1.0, n_exp=6, rcut=0.0, lambda3=0.0, shift=0,
                 rbond=0.0):
    return _check(ctx, load_library().swp_set_pair(ctx, int(ti), int(tj), int(kind), float(eps),
                                                   float(sigma), int(n_exp), float(rcut),
                                                   float(lambda3), int(shift), float(rbond)),
                  "swp_set_pair")


def swp_set_nlist(ctx, skin: float, max_nn: int):
    return _check(ctx, load_library().swp_set_nlist(ctx, float(skin), int(max_nn)), "swp_set_nlist")


def swp_workspace_size(ctx) -> int:
    v = ctypes.c_size_t()
    _check(ctx, load_library().swp_workspace_size(ctx, ctypes.byref(v)), "swp_workspace_size")
    return v.value


def swp_nlist_size(ctx) -> int:
    v = ctypes.c_size_t()
    _check(ctx, load_library().swp_nlist_size(ctx, ctypes.byref(v)), "swp_nlist_size")
    return v.value


def swp_bind_workspace(ctx, dev_ptr: int, nbytes: int, stream: int):
    return _check(ctx, load_library().swp_bind_workspace(ctx, ctypes.c_void_p(dev_ptr), nbytes,
                                                         ctypes.c_void_p(stream)),
                  "swp_bind_workspace")


def swp_bind_nlist(ctx, dev_ptr: int, nbytes: int):
    return _check(ctx, load_library().swp_bind_nlist(ctx, ctypes.c_void_p(dev_ptr), nbytes),
                  "swp_bind_nlist")


def swp_set_state(ctx, x, v=None, types=None, mass=None, img=None, where=SWP_HOST):
    return _check(ctx, load_library().swp_set_state(ctx, _ptr(x), _ptr(v), _ptr(types), _ptr(mass),
                                                    _ptr(img), int(where)), "swp_set_state")


def swp_set_step(ctx, step: int):
    return _check(ctx, load_library().swp_set_step(ctx, int(step)), "swp_set_step")


def swp_build_nlist(ctx):
    return _check(ctx, load_library().swp_build_nlist(ctx), "swp_build_nlist")


def swp_compute_forces(ctx):
    return _check(ctx, load_library().swp_compute_forces(ctx), "swp_compute_forces")


def swp_step_nve(ctx, dt: float, nsteps: int):
    return _check(ctx, load_library().swp_step_nve(ctx, float(dt), int(nsteps)), "swp_step_nve")


def swp_step_nvt(ctx, dt: float, kT: float, gamma: float, nsteps: int):
    return _check(ctx, load_library().swp_step_nvt(ctx, float(dt), float(kT), float(gamma), int(nsteps)),
                  "swp_step_nvt")


def swp_sync(ctx):
    return _check(ctx, load_library().swp_sync(ctx), "swp_sync")


def swp_read_thermo(ctx, check: bool = True) -> swp_thermo:
    t = swp_thermo()
    rc = load_library().swp_read_thermo(ctx, ctypes.byref(t))
    if check:
        _check(ctx, rc, "swp_read_thermo")
    return t


def swp_read_forces(ctx, out, where=SWP_HOST):
    return _check(ctx, load_library().swp_read_forces(ctx, _ptr(out), int(where)), "swp_read_forces")


def swp_read_state(ctx, x=None, v=None, img=None, where=SWP_HOST):
    return _check(ctx, load_library().swp_read_state(ctx, _ptr(x), _ptr(v), _ptr(img), int(where)),
                  "swp_read_state")


def swp_read_nlist(ctx, rows_dev, counts_dev, width: int):
    return _check(ctx, load_library().swp_read_nlist(ctx, _ptr(rows_dev), _ptr(counts_dev), int(width)),
                  "swp_read_nlist")


def swp_set_launch(ctx, blocks_per_sm: int = 0):
    return _check(ctx, load_library().swp_set_launch(ctx, int(blocks_per_sm)), "swp_set_launch")


def swp_set_grid(ctx, blocks: int = 0):
    return _check(ctx, load_library().swp_set_grid(ctx, int(blocks)), "swp_set_grid")


def swp_set_timeout(ctx, ns: int):
    return _check(ctx, load_library().swp_set_timeout(ctx, int(ns)), "swp_set_timeout")


def swp_set_resident(ctx, enable: int):
    return _check(ctx, load_library().swp_set_resident(ctx, int(enable)), "swp_set_resident")


def swp_set_withhold_arrival(ctx, on: int):
    return _check(ctx, load_library().swp_set_withhold_arrival(ctx, int(on)), "swp_set_withhold_arrival")


def swp_thermo_log_bytes(ctx, capacity: int) -> int:
    return int(load_library().swp_thermo_log_bytes(ctx, int(capacity)))


def swp_set_thermo_log(ctx, every: int, capacity: int = 0, ring=None, ring_bytes: int = 0):
    ptr = ring.data_ptr() if hasattr(ring, "data_ptr") else ring
    return _check(ctx, load_library().swp_set_thermo_log(ctx, int(every), int(capacity), ptr, int(ring_bytes)),
                  "swp_set_thermo_log")


def swp_thermo_log(ctx, rec, steps, max_records: int) -> int:
    """rec: device float64 [max_records][10]; steps: device int64 [max_records]."""
    n = ctypes.c_int64(0)
    _check(ctx, load_library().swp_thermo_log(ctx, rec.data_ptr(), steps.data_ptr(), int(max_records),
                                             ctypes.byref(n)), "swp_thermo_log")
    return int(n.value)


def swp_eval_grad(ctx, ti: int, tj: int, theta, x, types, U, F=None, dU=None, dF=None):
    """All arguments device tensors (float64; types int32), outputs written in place, no sync."""
    ptr = lambda t: None if t is None else t.data_ptr()
    return _check(ctx, load_library().swp_eval_grad(ctx, int(ti), int(tj), ptr(theta), ptr(x), ptr(types), ptr(U),
                                                    ptr(F), ptr(dU), ptr(dF)), "swp_eval_grad")


def swp_last_error(ctx) -> str:
    return (load_library().swp_last_error(ctx) or b"").decode(errors="replace")


def swp_compute_forces_static(ctx, x_dev, type_dev, f_dev, thermo_dev=None, stream: int = 0):
    """Forces into caller buffers with no device allocation (scratch in a static array)."""
    return _check(ctx, load_library().swp_compute_forces_static(ctx, _ptr(x_dev), _ptr(type_dev),
                                                                _ptr(f_dev), _ptr(thermo_dev),
                                                                ctypes.c_void_p(stream)),
                  "swp_compute_forces_static")


def swp_set_bonds(ctx, bonds, k: float, r0: float):
    """Harmonic bonds k/2 (r - r0)^2 between the tag pairs bonds [m, 2] (empty: none)."""
    b = np.ascontiguousarray(np.asarray(bonds, dtype=np.int32).reshape(-1, 2))
    return _check(ctx, load_library().swp_set_bonds(ctx, int(b.shape[0]), _ptr(b) if b.size else None, float(k),
                                                   float(r0)), "swp_set_bonds")


def swp_param_grad(ctx, ti: int, tj: int, dF_dev=None):
    """dU/d(lambda, eps, sigma) of the reactive pair (ti, tj) as a numpy array;
    dF/d(lambda, eps, sigma) into dF_dev ([3, n, 3] float64 device tensor) if given."""
    out = (ctypes.c_double * 3)()
    _check(ctx, load_library().swp_param_grad(ctx, int(ti), int(tj), out, _ptr(dF_dev)), "swp_param_grad")
    return np.array(list(out))


def swp_batch_workspace_size(n_systems: int) -> int:
    return int(load_library().swp_batch_workspace_size(int(n_systems)))


def swp_batch_step(ctxs, dt, kT, gamma, nsteps: int, split: float, ws_ptr: int, ws_bytes: int, threads: int = 0):
    """One launch advancing every context in ctxs nsteps steps (per-system dt, kT, gamma);
    threads: the batched kernel's block shape (0: 1024)."""
    m = len(ctxs)
    arr = (ctypes.c_void_p * m)(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])
    f = lambda v: (ctypes.c_double * m)(*[float(x) for x in v])
    rc = load_library().swp_batch_step(arr, m, f(dt), f(kT), f(gamma), int(nsteps), float(split), int(threads),
                                       ctypes.c_void_p(ws_ptr), int(ws_bytes))
    return _check(ctxs[0] if m else None, rc, "swp_batch_step")


def swp_batch_plan(w, n_blocks: int, split: float, max_group: int, min_part: int):
    """The batched work split for systems of w[r] particles on n_blocks blocks
    (host only): returns (item_ofs [n_blocks + 1], items [n, 4] rows of
    (system, rank in its group, group size, 0))."""
    m = len(w)
    wa = (ctypes.c_longlong * m)(*[int(x) for x in w])
    ofs = (ctypes.c_int * (n_blocks + 1))()
    items = (ctypes.c_int * (4 * (m + max(n_blocks, 0))))()
    n = ctypes.c_int(0)
    rc = load_library().swp_batch_plan(wa, m, int(n_blocks), float(split), int(max_group), int(min_part), ofs,
                                       items, ctypes.byref(n))
    _check(None, rc, "swp_batch_plan")
    return np.array(list(ofs), dtype=np.int64), np.array(list(items)[: 4 * n.value], dtype=np.int64).reshape(-1, 4)


def swp_destroy(ctx):
    return load_library().swp_destroy(ctx)
