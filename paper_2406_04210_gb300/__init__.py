"""GB300-native truncated Lennard-Jones molecular dynamics (arXiv 2406.04210 hot path).

The compute path is the C-ABI library ``libljmd.so`` (hand-written CUDA for
sm_103a, declared in ``include/ljmd.h``); :mod:`paper_2406_04210_gb300.ljmd`
is its thin ctypes binding.  Importing this package loads nothing; the first
call into :mod:`.ljmd` loads the library and raises if it is missing.
"""
__all__ = ["inputs", "ljmd"]
