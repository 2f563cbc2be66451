"""FP64 CPU oracle for the SP2 density-matrix method -- TEST INFRASTRUCTURE.

This package is the independent, slow, obviously-correct reference that the
CUDA library is checked against.  It is NOT part of the product: only the
test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA path (the only
common dependency is the seeded input generator ``sp2_inputs``, which holds
none of the method's arithmetic).

Everything is float64 numpy; a library matrix product (``@``) serves as the
matrix-square step, nothing is blocked, fused or reordered.

Parity status of each function (what pins it, beyond itself) is listed in
``sp2_oracle.__doc__``.
"""
from .sp2_oracle import *  # noqa: F401,F403
from .sp2_oracle import __all__  # noqa: F401
