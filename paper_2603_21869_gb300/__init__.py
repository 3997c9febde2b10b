"""GB300-native k-omega RANS finite-volume step (NeuralFVM method).

The compute path is the C-ABI library ``libfvm.so`` (CUDA kernels for
sm_103a) under ``csrc/``; ``binding`` loads it with ctypes.  ``cases`` holds
the seeded synthetic workloads.  Importing this package loads nothing; the
library is loaded on first use of :mod:`.binding`.
"""
__all__ = ["cases", "binding"]
