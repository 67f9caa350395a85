"""TENO5-LAD compressible-Euler right-hand side on GB300 (sm_103a), FP64.

The arithmetic runs in the CUDA library ``libteno_gb300.so`` (C-ABI in
``include/teno.h``); this package holds its build script, a ctypes binding
(``_lib``), the PyTorch-facing API (``api``) and the seeded input generators
(``inputs``).  Importing the package does not load the library; the first
call does, and raises if it cannot.
"""
__all__ = ["api", "inputs", "build"]


def __getattr__(name):
    if name in ("api", "_lib", "build", "inputs"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
