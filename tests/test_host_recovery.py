"""Host-side recovery logic of the Python layer, on CPU with a faked binding.

When the device reports a neighbour-row overflow, ``SwapSystem`` grows the
list capacity and resumes the interrupted call with the steps that remain;
``SwapBatch`` lets the system that overflowed finish alone.  Every other
error propagates.  The C-ABI calls are replaced by recording fakes, so no GPU
(and no failure on one) is involved.
"""
import types

import pytest

from paper_1912_08569_gb300 import _abi as A
from paper_1912_08569_gb300 import system as S


class FakeLib:
    """Records the ABI calls of one or more contexts; sync outcomes are scripted
    per context as a list of error codes (0 = success)."""

    def __init__(self, script, thermo):
        self.script = {k: list(v) for k, v in script.items()}
        self.thermo = thermo
        self.calls = []

    def swp_step_nvt(self, ctx, dt, kT, gamma, nsteps):
        self.calls.append(("step", ctx, int(nsteps), float(kT)))

    def swp_compute_forces(self, ctx):
        self.calls.append(("forces", ctx))

    def swp_batch_step(self, ctxs, dt, kT, gamma, nsteps, split, ws, nbytes, threads=0):
        self.calls.append(("batch", tuple(ctxs), int(nsteps)))

    def swp_sync(self, ctx):
        code = self.script[ctx].pop(0) if self.script[ctx] else 0
        self.calls.append(("sync", ctx, code))
        if code:
            raise A.SwpError(code, "swp_sync", "scripted")

    def swp_read_thermo(self, ctx, check=True):
        return self.thermo[ctx]

    def swp_set_nlist(self, ctx, skin, max_nn):
        self.calls.append(("set_nlist", ctx, int(max_nn)))


def _system(ctx, n=1000, max_nn=64):
    s = object.__new__(S.SwapSystem)
    s.ctx, s.n, s.max_nn, s.skin, s.grows = ctx, n, max_nn, 0.3, 0
    s._bind_nlist = lambda: None  # the device buffer is not needed here
    s.close = lambda: None  # the fake context never reaches the library
    return s


@pytest.fixture
def fake(monkeypatch):
    def install(script, thermo):
        lib = FakeLib(script, thermo)
        for name in ("swp_step_nvt", "swp_compute_forces", "swp_batch_step", "swp_sync", "swp_read_thermo",
                     "swp_set_nlist"):
            monkeypatch.setattr(S.A, name, getattr(lib, name))
        return lib

    return install


def test_run_resumes_after_overflow_with_the_remaining_steps(fake):
    lib = fake({"c0": [A.SWP_ERR_NLIST_OVERFLOW, 0]},
               {"c0": types.SimpleNamespace(steps_done=30, max_row=90)})
    s = _system("c0")
    s.run(100, 0.001, 0.1, 1.0)
    steps = [c[2] for c in lib.calls if c[0] == "step"]
    assert steps == [100, 70]
    assert s.grows == 1 and s.max_nn == 120  # round_up(1.25 * 90 + 8, 8)
    assert ("set_nlist", "c0", 120) in lib.calls


def test_run_propagates_other_errors(fake):
    fake({"c0": [A.SWP_ERR_TIMEOUT]}, {"c0": types.SimpleNamespace(steps_done=0, max_row=0)})
    s = _system("c0")
    with pytest.raises(A.SwpError) as e:
        s.run(10, 0.001)
    assert e.value.code == A.SWP_ERR_TIMEOUT
    assert s.grows == 0


def test_run_gives_up_when_the_list_keeps_overflowing(fake):
    fake({"c0": [A.SWP_ERR_NLIST_OVERFLOW] * 100}, {"c0": types.SimpleNamespace(steps_done=0, max_row=200)})
    s = _system("c0")
    with pytest.raises(RuntimeError):
        s.run(10, 0.001)
    assert s.grows == 16


def test_compute_forces_retries_after_growing(fake):
    lib = fake({"c0": [A.SWP_ERR_NLIST_OVERFLOW, 0]}, {"c0": types.SimpleNamespace(steps_done=0, max_row=70)})
    s = _system("c0")
    s.compute_forces()
    assert [c[0] for c in lib.calls].count("forces") == 2
    assert s.grows == 1 and s.max_nn == 96


def test_batch_overflowing_system_finishes_alone(fake):
    lib = fake({"a": [0], "b": [A.SWP_ERR_NLIST_OVERFLOW, 0], "c": [0]},
               {"b": types.SimpleNamespace(steps_done=120, max_row=80)})
    systems = [_system(k) for k in ("a", "b", "c")]
    batch = object.__new__(S.SwapBatch)
    batch.systems, batch.split, batch.threads = systems, 1.0, 1024
    batch.ws = types.SimpleNamespace(data_ptr=lambda: 0, numel=lambda: 0)
    batch.run(500, 0.001, [0.1, 0.2, 0.3], 1.0)
    assert lib.calls[0] == ("batch", ("a", "b", "c"), 500)
    alone = [c for c in lib.calls if c[0] == "step"]
    assert alone == [("step", "b", 380, 0.2)]  # the steps b had left, with b's own kT
    assert systems[1].grows == 1 and systems[0].grows == 0 and systems[2].grows == 0
