"""GB300-native MLS-MPM substep (the soft-body engine of ManiSkill2, Sec. 3 and Algorithm 1).

The compute lives in a C-ABI CUDA library (``csrc/``, declared in ``include/mpm.h``);
``mpm`` is its thin ctypes binding with the same entry-point names, and ``Sim`` a
convenience wrapper that takes device memory and streams from PyTorch. Importing
this package loads nothing: the library is opened on first use and raises if it
has not been built.
"""

__all__ = ["scenes", "mpm", "Sim"]


def __getattr__(name):
    if name == "mpm":
        from . import _native as mpm
        return mpm
    if name == "Sim":
        from .sim import Sim
        return Sim
    raise AttributeError(name)
