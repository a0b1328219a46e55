"""GB300-native hybrid symplectic N-body step (Mercury-Opal's integrator).

The compute path is the CUDA library built from ``csrc/`` for sm_103a and
reached through the C ABI in ``include/opal.h``; ``opal`` is its ctypes
binding.  Build with ``paper_2601_19654_gb300.build.build()``.
"""
import importlib

from .build import build  # noqa: F401

__all__ = ["build", "opal"]


def __getattr__(name):
    if name == "opal":
        return importlib.import_module(__name__ + ".opal")
    raise AttributeError(name)
