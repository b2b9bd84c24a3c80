"""GB300-native random batch sum-of-Gaussians (RBSOG) force evaluation.

The compute path is librbsog.so (CUDA for sm_103a behind the C ABI of
include/rbsog.h); ``binding`` marshals arguments to it and ``system.RBSOG``
wraps one system for torch users.  Importing the package loads the library
and fails if it has not been built."""
from . import binding  # noqa: F401  (loads librbsog.so or raises)
from .binding import RBSOGError  # noqa: F401
from .system import DEFAULT_B, DEFAULT_M, RBSOG, Batch, Server, make_params  # noqa: F401
