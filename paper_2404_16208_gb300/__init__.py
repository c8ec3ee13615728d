"""GB300 (sm_103a) RANC tick simulator: hand-written CUDA kernels behind the C
ABI of ``include/ranc.h``, with a ctypes binding in :mod:`.ranc`.

``from paper_2404_16208_gb300 import ranc`` loads the compiled library and
raises ImportError when it is missing; :func:`build_library` compiles it.
"""

from .build import build as build_library  # noqa: F401
