"""GB300-native LOC line radiative transfer: the ALI ray march and the
statistical-equilibrium solve as sm_103a CUDA kernels behind a C ABI
(include/loc.h), with a thin ctypes binding (``loc``).  Importing the
package does not load the CUDA library; ``loc.load()`` does, and fails
loudly if it has not been built."""
from . import build  # noqa: F401
from . import loc  # noqa: F401

__all__ = ["build", "loc"]
