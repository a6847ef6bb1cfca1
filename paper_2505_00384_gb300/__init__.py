"""GB300 (sm_103a) library for the pressure solve and explicit fluxes of the
IMEX-DG compressible-Euler scheme of arXiv:2505.00384.

The compute path is ``libdgx.so`` (hand-written CUDA behind the C ABI in
``include/dgx.h``); ``dgx`` is its ctypes binding and ``inputs`` the seeded
synthetic-input generators.
"""
from . import dgx  # noqa: F401

__all__ = ["dgx"]
