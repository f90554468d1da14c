"""GB300-native associative bond-swap molecular dynamics (arXiv 1912.08569).

The hot path -- cell-sorted Verlet list, the per-centre S pass of the
three-body swap term, the force pass fused with the velocity-Verlet / BAOAB
integrator -- runs in hand-written sm_103a CUDA kernels behind the C-ABI of
``include/swapmd.h`` (``libswapmd.so``, built by ``build.build()``).  This
package is the thin Python side: ``_abi`` (ctypes binding, same names as the
C entry points), ``system.SwapSystem`` (torch-owned buffers and stream) and
``inputs`` (seeded synthetic configurations).  Importing it loads nothing;
using a ``SwapSystem`` without the built library raises.
"""
from . import _abi  # noqa: F401

__all__ = ["SwapSystem", "SwapBatch", "build"]


def __getattr__(name):
    if name == "SwapBatch":
        from .system import SwapBatch

        return SwapBatch
    if name == "SwapSystem":
        from .system import SwapSystem

        return SwapSystem
    if name == "build":
        from .build import build

        return build
    raise AttributeError(name)
