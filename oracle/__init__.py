"""FP64 CPU oracle for SIFT-aided EIS inversion (arXiv 2207.14507). TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  It shares no code with the CUDA path and is never a
fallback for it.
"""
from .prnu_oracle import *  # noqa: F401,F403
from . import parallel  # noqa: F401,E402
