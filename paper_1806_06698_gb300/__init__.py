"""GB300-native batched 3x3 real symmetric eigensolver (Borges, arXiv 1806.06698).

The compute path is the C-ABI library ``libsyev3.so`` built from ``csrc/``
(hand-written sm_103a CUDA); ``syev3`` is its thin ctypes binding.  The
library is loaded on first use and a missing build raises immediately: there
is no CPU fallback.
"""

__all__ = ["inputs", "syev3"]
