"""GB300-native batched shifted m-Hessenberg solver.

Solves (A - sigma_j I) X_j = B for many complex shifts through a one-time
controller-Hessenberg reduction and a persistent shift-batched CUDA solver
(Bosner, Bujanovic, Drmac, Sec. 2-3).  The compute path is the CUDA library
``_build/libssv.so`` (C ABI in ``include/ssv.h``); :mod:`.ssv` is its binding.
"""
from . import ssv  # noqa: F401
from .ssv import Handle, reduce, colmajor, footprint, handle_bytes  # noqa: F401
