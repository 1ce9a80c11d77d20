"""libafns: B300-native (sm_103a) per-RK-stage update of the compact fourth-order
positivity-preserving active flux method for compressible Navier-Stokes
(Duan, Barsukow, Klingenberg, arXiv 2609.29081).

The compute path is the CUDA library ``libafns.so`` behind the C-ABI of
``include/afns.h``; ``Solver`` is its thin Python binding.
"""
from . import workloads  # noqa: F401


def __getattr__(name):
    if name in ("Solver", "AfnsError", "load", "FP64", "MIXED", "LIM_NONE", "LIM_PP", "LIM_S_PP", "BatchSolver"):
        from . import _native
        return getattr(_native, name)
    raise AttributeError(name)
