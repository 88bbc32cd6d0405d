"""Plain FP64 CPU oracle for the XL-BOMD hot path (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library under
``paper_1705_10845_gb300`` never does, and shares no code with it.
"""
from .xlbomd import *  # noqa: F401,F403
