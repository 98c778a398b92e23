"""GB300-native Palindromic Discontinuous Galerkin (PDG) kinetic solver.

The compute path lives in the C-ABI shared library ``libpdg.so`` built from
``csrc/`` (CUDA for sm_103a); ``pdg`` is its thin ctypes binding (argument
marshalling only).  ``workloads`` holds the seeded synthetic input recipes.

Importing this package does not load the CUDA library; ``pdg`` does, and it
raises if the library is missing (there is no CPU fallback).
"""

__all__ = ["pdg", "workloads"]


def __getattr__(name):
    if name in ("pdg", "workloads"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
