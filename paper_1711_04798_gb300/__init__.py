"""GB300-native CTM library for the iPEPS method of arXiv:1711.04798.

The compute path is the in-tree CUDA library ``_lib/libipeps_ctm.so`` (built
by ``build.build()``); ``binding`` is a thin ctypes layer over its C ABI
(``include/ipeps_ctm.h``).  There is no CPU fallback: loading fails loudly
when the library is missing.
"""
from .binding import CTM, Batch, CTMError, env_file_info, load_library  # noqa: F401
