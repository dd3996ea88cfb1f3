"""RBSOG electrostatics for NPT molecular dynamics on GB300 (sm_103a).

The compute path is ``librbsog.so`` (hand-written CUDA kernels behind the C
ABI of ``include/rbsog.h``); ``rbsog`` is its ctypes binding."""
from . import rbsog  # noqa: F401
from .rbsog import Context, rbsog_default_params  # noqa: F401
