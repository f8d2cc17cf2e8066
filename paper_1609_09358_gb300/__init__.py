"""GB300-native hybrid BP + CA-SCL polar decoder (arXiv 1609.09358).

The decoder runs in hand-written sm_103a CUDA kernels behind the C-ABI declared in
``include/polar_gb300.h``; ``api`` is the thin ctypes binding (argument marshalling only) and
``inputs`` draws seeded synthetic payload bits and noise.  Importing the package loads nothing:
the shared library is opened on the first decoder call and a missing library is an error.
"""
__all__ = ["api", "inputs"]
