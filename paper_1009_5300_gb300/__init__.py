"""GB300-native IOBM electron-transport solver (Egami, Hirose and Ono).

The hot path -- preconditioned COCG on the complex-symmetric real-space
finite-difference equations of the improved overbridging boundary-matching
method, with the jellium self-energy applied through lateral FFTs -- lives in
the CUDA library ``libiobm.so`` (C ABI: include/iobm.h).  This package only
builds it and marshals arguments.
"""
from ._lib import IOBMError, load  # noqa: F401

__all__ = ["IOBMError", "load", "IOBMSolver", "solve_batch", "conductance", "build_library"]


def build_library(force: bool = False, verbose: bool = False) -> str:
    """Compile libiobm.so in-tree for sm_103a (no-op when up to date)."""
    from .build import build as _build
    return _build(force=force, verbose=verbose)


def __getattr__(name):
    if name == "IOBMSolver":
        from .solver import IOBMSolver
        return IOBMSolver
    if name == "conductance":
        from .autograd import conductance
        return conductance
    if name == "solve_batch":
        from .solver import solve_batch
        return solve_batch
    if name == "channels_host":
        from .solver import channels_host
        return channels_host
    raise AttributeError(name)
