"""FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The library path never does: it fails
loudly when its CUDA extension is missing instead of falling back here.
"""
from .oracle import *  # noqa: F401,F403
