"""fkski: faster kernel interpolation (GSGP / factorized SKI) on GB300.

The compute lives in the C-ABI library ``libfkski.so`` (CUDA for sm_103a, built from ``csrc/``);
``api`` is a thin ctypes binding with the same entry points.  Importing this package does not
load the library; ``api.load()`` does, and fails loudly if it is missing.
"""
__all__ = ["api", "synth"]
