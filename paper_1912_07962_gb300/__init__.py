"""GB300-native slimLS: the sampled limited-memory row-action method on sm_103a.

The compute path is libslim.so (hand-written CUDA, C ABI in include/slim.h);
`slim` is its ctypes binding.
"""
from . import slim  # noqa: F401
from .slim import Slim, SlimError, damped_solve, load  # noqa: F401
