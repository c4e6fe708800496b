"""GB300-native MLFMA-SMR matrix-vector product and solver (arXiv 2407.21724).

The compute path is the C-ABI library ``libsmr.so`` (hand-written CUDA for
sm_103a, declared in ``include/smr.h``); ``paper_2407_21724_gb300.smr`` is its
thin ctypes binding.  Importing this package loads nothing; the binding loads
the library on first use and raises if it has not been built.
"""
__version__ = "0.1.0"
