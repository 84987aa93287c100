"""FP64 CPU oracle of the anelastic pressure projection (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  It shares no code with the CUDA path.
"""
from .projection import *  # noqa: F401,F403
