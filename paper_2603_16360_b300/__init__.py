"""B300-native approximate vector epsilon-join (merged index + soft work sharing
+ adaptive hybrid expansion), after "Fast Approximate Vector Joins via
Offline-Online Co-Design" (arXiv 2603.16360).

The compute path is the CUDA library ``libvj.so`` built from ``csrc/``; the
Python binding in :mod:`paper_2603_16360_b300.vj` only marshals arguments into
its C ABI (declared in ``include/vj.h``).  Importing this package does not load
the library; :func:`paper_2603_16360_b300.vj.load` does, and raises if it is
missing.
"""
__all__ = ["vj", "inputs"]
