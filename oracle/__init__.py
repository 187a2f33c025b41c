"""CPU oracle (test infrastructure only): plain FP64 restatement of the paper's method.

Only tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg use
this package.  The library under ``paper_1810_02719_gb300`` never imports it.
"""
from . import bsp_oracle  # noqa: F401
