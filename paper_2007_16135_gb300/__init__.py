"""GB300-native Time Warp Edit Distance (TWED).

The compute path is the CUDA library ``libtwed.so`` built from ``csrc/`` for
sm_103a; ``twed.py`` is a ctypes binding with the same entry-point names as
``include/twed.h``.  Importing this package does not load the library; the
first call into :mod:`paper_2007_16135_gb300.twed` does, and fails loudly if
it has not been built.
"""
__all__ = ["twed", "workloads"]
