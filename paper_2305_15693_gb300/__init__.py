"""GB300-native FReSCo hot path: the structure-factor loss and its gradient through a
type-1 / type-2 NUFFT pair in hand-written CUDA (sm_103a) behind the C ABI of include/fresco.h.

`fresco` is the ctypes binding (same names as the C entry points); `inputs` holds the seeded
synthetic workloads. Build the shared library with `_build.build()`.
"""

from . import fresco, inputs  # noqa: F401

__all__ = ["inputs", "fresco"]
