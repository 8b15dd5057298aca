"""GB300-native alternating cross interpolation (ACI) for elementwise operations on tensor trains.

The method (arXiv:2604.00037) computes a tensor train y ~ f(x^1, ..., x^N) with error control
in O(chi^3) per local update. This package is a thin Python layer over a C-ABI CUDA library
(``include/aci.h``): ``binding.Context`` marshals arguments to it, ``build.build()`` compiles it
for sm_103a. There is no CPU fallback: without the compiled library and a CUDA device the
calls raise.
"""

from .buildlib import build, LIB as LIBRARY_PATH  # noqa: F401


def Context(device: int = 0):
    """Create an ACI context on ``device`` (see binding.Context)."""
    from .binding import Context as _Ctx
    return _Ctx(device)
