"""GB300-native matrix-free two-level deflation + CSLP Helmholtz solver.

The compute path lives in the CUDA shared library ``libhz.so`` (built from
``csrc/`` for sm_103a) behind a C ABI (``include/hz.h``).  This package is a
thin ctypes binding over it plus the seeded input generators in
``workloads``.  Importing the package does not load the library; the first
call into ``Solver`` does, and raises if it is missing.
"""

__all__ = ["Solver", "Desc", "HzError", "load_library"]


def __getattr__(name):
    import importlib
    if name in ("Solver", "Desc", "HzError"):
        return getattr(importlib.import_module(__name__ + ".api"), name)
    if name == "load_library":
        return importlib.import_module(__name__ + "._lib").load_library
    raise AttributeError(name)
