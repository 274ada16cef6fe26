"""GB300-native Quantile Rendering (Q-Render) hot path.

The compute path is the C-ABI library ``libqrender.so`` (hand-written sm_103a
CUDA, built from ``csrc/``); ``qrender`` is its thin ctypes binding.  Importing
this package loads nothing; ``paper_2512_20927_gb300.qrender`` loads the
library on first use and raises if it is missing.
"""
__all__ = ["scenes", "qrender"]
