"""GB300-native fractional Adams-Bashforth-Moulton history convolution.

The compute path lives in the CUDA library ``csrc/`` (C ABI declared in
``include/abm.h``); ``abm`` is the thin ctypes binding over it and
``autograd`` wraps the adjoint for PyTorch.  Nothing is imported eagerly so
that the seeded input generators (``workloads``) load without a GPU.
"""
__all__ = ["abm", "workloads"]
