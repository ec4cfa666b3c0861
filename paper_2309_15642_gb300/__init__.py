"""GB300 (sm_103a) simple-update Trotter evolution of the kicked Ising circuit on graph PEPS.

The compute path is the CUDA library ``libgpeps.so`` (C ABI in ``include/gpeps.h``);
``GPEPS`` is its thin Python binding.  Build the library with
``paper_2309_15642_gb300._build.build()``.
"""
from ._abi import GpepsError, load  # noqa: F401

__all__ = ["GPEPS", "GpepsError", "load"]


def __getattr__(name):
    if name == "GPEPS":
        from .gpeps import GPEPS
        return GPEPS
    raise AttributeError(name)
