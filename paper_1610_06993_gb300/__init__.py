"""GB300-native coarse-grid-projection (CGP) pressure-correction step.

The CUDA library ``libcgp.so`` (sources in ``csrc/``, C ABI in ``include/cgp.h``) implements the
IFE-CGP time step of Kashefi & Staples (Sect. 2.2, Eqs. 19-23). ``cgp`` is its ctypes binding,
``flow.Flow`` a small driver that keeps the state in torch device tensors.
"""
from . import cgp  # noqa: F401

__all__ = ["cgp"]
