"""GB300-native exact local-alignment search (ALAE, arXiv 1208.0274).

The library libae.so (CUDA kernels for sm_103a plus a C ABI, include/ae.h)
does all the work; ``paper_1208_0274_gb300.ae`` is its thin ctypes binding
with the same function names.  Importing the package does not load the
library (so ``paper_1208_0274_gb300.build`` can run first); the first use of
a binding name does, and fails loudly if the library was not built.
"""
import importlib


def __getattr__(name):
    if name.startswith("__"):
        raise AttributeError(name)
    if name in ("ae", "build"):
        return importlib.import_module(f"{__name__}.{name}")
    return getattr(importlib.import_module(f"{__name__}.ae"), name)
