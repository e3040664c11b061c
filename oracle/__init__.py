"""Plain FP64 CPU oracle for the CTM contraction of the paper's iPEPS method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

It shares no code with the CUDA library: numpy (LAPACK SVD / eig) and einsum
only, each function citing the passage of the paper it follows.
"""
from .ctm import *  # noqa: F401,F403
from .readout import *  # noqa: F401,F403
