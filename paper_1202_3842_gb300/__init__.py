"""GB300-native stabilized Lattice Boltzmann-Enskog (DD-TR) hot path.

The compute path is the CUDA library ``liblbe.so`` built from ``csrc/`` for
sm_103a; ``lbe`` is its thin ctypes binding (same names as the C ABI in
``include/lbe.h``).  ``inputs`` builds seeded synthetic input arrays.
Importing this package loads nothing; the library is loaded on first use and
a missing library is an error, never a fallback.
"""

__all__ = ["lbe", "inputs"]
