"""GB300-native exact local-alignment search (ALAE, arXiv 1208.0274).

The library libae.so (CUDA kernels for sm_103a plus a C ABI, include/ae.h)
does all the work; ``paper_1208_0274_gb300.ae`` is its thin ctypes binding
with the same function names.
"""

from .ae import *  # noqa: F401,F403
