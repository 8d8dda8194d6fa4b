"""GB300-native cascade for applying LTI transfer functions in the time domain
(Beylkin, "Fast convolution algorithm for state space models", arXiv 2411.17729).

The computation lives in libcascade.so (CUDA, sm_103a) behind the C ABI of
include/cascade.h; this package is its ctypes binding (``_abi``), a thin
tensor-level wrapper (``Cascade``) and the build step (``build``).
"""
from .build import build  # noqa: F401


def __getattr__(name):
    if name in ("Cascade", "CascadeFunction", "from_workload"):
        from . import cascade as _c
        return getattr(_c, name)
    raise AttributeError(name)
