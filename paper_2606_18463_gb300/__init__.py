"""GB300-native (sm_103a) s-step / communication-avoiding SGD for GLMs.

The compute path is libglm.so (hand-written CUDA, C ABI in include/glm.h);
``paper_2606_18463_gb300.glm`` is its ctypes binding.
"""
from . import glm  # noqa: F401

__all__ = ["glm"]
