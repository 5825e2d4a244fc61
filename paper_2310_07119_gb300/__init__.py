"""GB300 truncated-Wigner (TWA) ensemble library: CUDA kernels behind a C ABI (include/twa.h).

The Python layer only marshals arguments to libtwa.so; see ``twa`` for the
calls (same names as the C ABI) and the ``Ensemble`` convenience wrapper.
"""
from .twa import *  # noqa: F401,F403
from .twa import Ensemble, TwaError  # noqa: F401
