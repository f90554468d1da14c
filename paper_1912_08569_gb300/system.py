"""``SwapSystem``: one simulation on one GPU through the C-ABI.

PyTorch provides only device memory (the workspace and the neighbour-list
buffer the library borrows) and the CUDA stream.  The neighbour-list length is
grown and the interrupted call resumed when the device reports an overflow.
"""
from __future__ import annotations

import math

import numpy as np

from . import _abi as A


def _round_up(x: int, m: int) -> int:
    return ((x + m - 1) // m) * m


class SwapSystem:
    """n particles of n_types types in a periodic box, with a type-pair table.

    pairs: {(ti, tj): dict(kind=1|2, eps, sigma, n, rcut, lambda3, shift, rbond)}
    (kind 1 = WCA, 2 = swap).  precision: "fp32" or "fp64".
    """

    def __init__(self, n, n_types, box, pairs, precision="fp32", seed=0, skin=0.3, max_nn=None,
                 blocks_per_sm=0, device=None, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("SwapSystem needs a CUDA device (no CPU fallback)")
        A.load_library()
        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        torch.cuda.set_device(self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.n = int(n)
        self.n_types = int(n_types)
        self.box = np.asarray(box, dtype=np.float64)
        self.precision = A.SWP_FP64 if precision in ("fp64", A.SWP_FP64) else A.SWP_FP32
        self.ctx = A.swp_create(self.n, self.n_types, self.box, self.precision, seed)
        self.skin = float(skin)
        for (ti, tj), p in pairs.items():
            A.swp_set_pair(self.ctx, ti, tj, p.get("kind", 0), p.get("eps", 1.0), p.get("sigma", 1.0),
                           p.get("n", 6), p.get("rcut", 0.0), p.get("lambda3", 0.0),
                           p.get("shift", 0), p.get("rbond", 0.0) or 0.0)
        if max_nn is None:
            rl = max((p.get("rcut", 0.0) if p.get("kind") == 2 else p.get("sigma", 1.0) * 2 ** (1 / p.get("n", 6)))
                     for p in pairs.values()) + self.skin if pairs else 1.0
            rho = self.n / float(np.prod(self.box))
            expect = rho * 4.0 / 3.0 * math.pi * rl ** 3
            max_nn = max(16, _round_up(int(2.0 * expect + 16), 8))
        self.max_nn = int(max_nn)
        A.swp_set_nlist(self.ctx, self.skin, self.max_nn)
        A.swp_set_launch(self.ctx, blocks_per_sm)
        ws = A.swp_workspace_size(self.ctx)
        self.workspace = torch.empty(ws, dtype=torch.uint8, device=self.device)
        A.swp_bind_workspace(self.ctx, self.workspace.data_ptr(), ws, self.stream.cuda_stream)
        self._bind_nlist()
        self.grows = 0

    # -- buffers ------------------------------------------------------------
    def _bind_nlist(self):
        nb = A.swp_nlist_size(self.ctx)
        self.nlist_buf = self.torch.empty(nb, dtype=self.torch.uint8, device=self.device)
        A.swp_bind_nlist(self.ctx, self.nlist_buf.data_ptr(), nb)

    def _grow(self, needed: int):
        self.max_nn = _round_up(int(needed * 1.25) + 8, 8)
        A.swp_set_nlist(self.ctx, self.skin, self.max_nn)
        self._bind_nlist()
        self.grows += 1

    def set_launch(self, blocks_per_sm: int = 0):
        """Resident step-kernel blocks per SM (0: as many as fit)."""
        A.swp_set_launch(self.ctx, blocks_per_sm)

    def set_grid(self, blocks: int = 0):
        """Upper bound on the step kernel's blocks (0: every SM's resident blocks)."""
        A.swp_set_grid(self.ctx, blocks)

    def set_timeout(self, ns: int):
        A.swp_set_timeout(self.ctx, ns)

    def set_resident(self, enable: bool = True):
        """Allow (default) or forbid the resident mode of the FP32 step."""
        A.swp_set_resident(self.ctx, 1 if enable else 0)

    def set_thermo_log(self, every: int, capacity: int = 1024):
        """Log the thermo record of every step whose number is a multiple of
        ``every`` into a device ring of ``capacity`` records (every=0: off)."""
        import torch

        if every <= 0:
            A.swp_set_thermo_log(self.ctx, 0)
            self._tlog = None
            return
        nb = A.swp_thermo_log_bytes(self.ctx, capacity)
        ring = torch.empty(nb, dtype=torch.uint8, device=self.device)
        A.swp_set_thermo_log(self.ctx, every, capacity, ring, nb)
        self._tlog = (ring, int(capacity))

    def thermo_log(self) -> dict:
        """The logged records, oldest first: step, U2, U3, K, W [m][6], n_bonds."""
        import torch

        if getattr(self, "_tlog", None) is None:
            raise RuntimeError("no thermo log: call set_thermo_log first")
        cap = self._tlog[1]
        rec = torch.empty((cap, 10), dtype=torch.float64, device=self.device)
        stp = torch.empty(cap, dtype=torch.int64, device=self.device)
        m = A.swp_thermo_log(self.ctx, rec, stp, cap)
        r = rec[:m].cpu().numpy()
        return dict(step=stp[:m].cpu().numpy(), U2=r[:, 0], U3=r[:, 1], K=r[:, 2], W=r[:, 3:9],
                    n_bonds=np.rint(r[:, 9]).astype(np.int64))

    # -- state --------------------------------------------------------------
    def set_state(self, x, v=None, types=None, mass=None, img=None):
        """Host arrays (numpy) or device tensors (torch, cuda) in user order."""
        if hasattr(x, "is_cuda") and x.is_cuda:
            where = A.SWP_DEVICE
            t = self.torch
            cv = lambda a, dt: None if a is None else a.to(device=self.device, dtype=dt).contiguous()
            self._keep = [cv(x, t.float64), cv(v, t.float64), cv(types, t.int32), cv(mass, t.float64),
                          cv(img, t.int32)]
        else:
            where = A.SWP_HOST
            cv = lambda a, dt: None if a is None else np.ascontiguousarray(a, dtype=dt)
            self._keep = [cv(x, np.float64), cv(v, np.float64), cv(types, np.int32), cv(mass, np.float64),
                          cv(img, np.int32)]
        A.swp_set_state(self.ctx, *self._keep, where=where)

    def set_bonds(self, bonds, k: float, r0: float):
        """Harmonic bonds k/2 (r - r0)^2 between tag pairs (an [m, 2] array)."""
        A.swp_set_bonds(self.ctx, bonds, k, r0)

    def set_step(self, step: int):
        A.swp_set_step(self.ctx, step)

    # -- work ---------------------------------------------------------------
    def _retry_overflow(self, call):
        for _ in range(8):
            call()
            try:
                A.swp_sync(self.ctx)
                return
            except A.SwpError as e:
                if e.code != A.SWP_ERR_NLIST_OVERFLOW:
                    raise
                th = A.swp_read_thermo(self.ctx, check=False)
                self._grow(th.max_row)
        raise RuntimeError("neighbour list kept overflowing")

    def build_nlist(self):
        self._retry_overflow(lambda: A.swp_build_nlist(self.ctx))

    def compute_forces(self):
        self._retry_overflow(lambda: A.swp_compute_forces(self.ctx))

    def run(self, nsteps: int, dt: float, kT: float = 0.0, gamma: float = 0.0, sync: bool = True):
        """Advance nsteps (BAOAB if gamma > 0, else velocity Verlet)."""
        if not sync:
            A.swp_step_nvt(self.ctx, dt, kT, gamma, nsteps)
            return
        remaining = [int(nsteps)]

        def call():
            A.swp_step_nvt(self.ctx, dt, kT, gamma, remaining[0])

        for _ in range(16):
            call()
            try:
                A.swp_sync(self.ctx)
                return
            except A.SwpError as e:
                if e.code != A.SWP_ERR_NLIST_OVERFLOW:
                    raise
                th = A.swp_read_thermo(self.ctx, check=False)
                remaining[0] -= int(th.steps_done)
                self._grow(th.max_row)
        raise RuntimeError("neighbour list kept overflowing")

    def sync(self):
        A.swp_sync(self.ctx)

    # -- read-out -----------------------------------------------------------
    def thermo(self) -> dict:
        t = A.swp_read_thermo(self.ctx)
        return dict(U2=t.U2, U3=t.U3, K=t.K, W=np.array(list(t.W)), n_bonds=int(t.n_bonds),
                    step=int(t.step), n_rebuilds=int(t.n_rebuilds), steps_done=int(t.steps_done),
                    max_row=int(t.max_row), state=int(t.state), resident_steps=int(t.resident_steps))

    def forces(self) -> np.ndarray:
        f = np.zeros((max(self.n, 1), 3))
        A.swp_read_forces(self.ctx, f)
        return f[: self.n]

    def state(self):
        x = np.zeros((max(self.n, 1), 3))
        v = np.zeros((max(self.n, 1), 3))
        img = np.zeros((max(self.n, 1), 3), dtype=np.int32)
        A.swp_read_state(self.ctx, x, v, img)
        return x[: self.n], v[: self.n], img[: self.n]

    def nlist(self, width: int = 64):
        """(rows, counts): rows[i, :counts[i,1]] are the tags in i's list, reactive first
        (rows are cut at `width`; a second read is made when some row is longer)."""
        t = self.torch
        counts = t.zeros((max(self.n, 1), 2), dtype=t.int32, device=self.device)
        for _ in range(2):
            rows = t.full((max(self.n, 1), width), -1, dtype=t.int32, device=self.device)
            A.swp_read_nlist(self.ctx, rows, counts, width)
            longest = int(counts[:, 1].max().item()) if self.n else 0
            if longest <= width:
                break
            width = longest
        return rows.cpu().numpy()[: self.n], counts.cpu().numpy()[: self.n]

    def close(self):
        if getattr(self, "ctx", None) is not None:
            A.swp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SwapBatch:
    """Independent SwapSystem objects advanced together, one launch per call.

    The systems may differ in size, box, coefficients and temperature; they
    share precision, device and stream.  ``split`` selects the work split
    (0: the balanced plan; > 0: the threshold plan with that factor) and
    ``threads`` the batched kernel's block shape (see swp_batch_step);
    ``autotune`` picks both by timing.
    """

    SHAPES = {A.SWP_FP32: (1024, 512, 384, 256), A.SWP_FP64: (1024,)}  # threads per block

    def __init__(self, systems, split: float = 0.0, threads: int = 1024):
        import torch

        self.systems = list(systems)
        if not self.systems:
            raise ValueError("empty batch")
        s0 = self.systems[0]
        for s in self.systems:
            if s.device != s0.device or s.stream.cuda_stream != s0.stream.cuda_stream:
                raise ValueError("batched systems need one device and one stream")
            if s.precision != s0.precision:
                raise ValueError("batched systems need one precision")
        self.torch = torch
        self.split = float(split)
        self.threads = int(threads)
        nb = A.swp_batch_workspace_size(len(self.systems))
        self.ws = torch.empty(nb, dtype=torch.uint8, device=s0.device)

    def _per(self, v):
        if np.ndim(v) == 0:
            return [float(v)] * len(self.systems)
        v = [float(x) for x in v]
        if len(v) != len(self.systems):
            raise ValueError("one value per system")
        return v

    def run(self, nsteps: int, dt, kT=0.0, gamma=0.0, sync: bool = True):
        """Advance every system nsteps steps (per-system or common dt, kT, gamma)."""
        dt, kT, gamma = self._per(dt), self._per(kT), self._per(gamma)
        A.swp_batch_step([s.ctx for s in self.systems], dt, kT, gamma, int(nsteps), self.split,
                         self.ws.data_ptr(), self.ws.numel(), self.threads)
        if not sync:
            return
        for k, s in enumerate(self.systems):
            try:
                A.swp_sync(s.ctx)
            except A.SwpError as e:
                if e.code != A.SWP_ERR_NLIST_OVERFLOW:
                    raise
                # this system stopped at the overflow: grow its list, finish alone
                th = A.swp_read_thermo(s.ctx, check=False)
                s._grow(th.max_row)
                s.run(int(nsteps) - int(th.steps_done), dt[k], kT[k], gamma[k])

    def sync(self):
        for s in self.systems:
            A.swp_sync(s.ctx)

    def autotune(self, nsteps: int, dt, kT=0.0, gamma=0.0, splits=(0.0, 0.5, 1.0, 2.0, 1e9), shapes=None):
        """Times one nsteps run per (block shape, split) candidate -- every
        shape the precision has, by default -- with the systems advancing, and
        keeps the fastest; returns (ms, split, threads, table of every timing)."""
        t = self.torch
        shapes = self.SHAPES[self.systems[0].precision] if shapes is None else shapes
        best, table = None, []
        for th in shapes:
            for sp in splits:
                self.threads, self.split = int(th), float(sp)
                self.run(1, dt, kT, gamma)  # warm-up (and list builds for the new grouping)
                e0, e1 = t.cuda.Event(enable_timing=True), t.cuda.Event(enable_timing=True)
                stream = self.systems[0].stream
                e0.record(stream)
                self.run(nsteps, dt, kT, gamma, sync=False)
                e1.record(stream)
                self.sync()
                ms = e0.elapsed_time(e1)
                table.append((int(th), float(sp), ms))
                if best is None or ms < best[0]:
                    best = (ms, float(sp), int(th))
        self.split, self.threads = best[1], best[2]
        return best + (table,)
