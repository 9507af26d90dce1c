"""GB300-native Generalized Parallel Replica dynamics (Hedin & Lelievre, gen.parRep).

The compute path lives in the CUDA library ``libgrp.so`` (``csrc/``) behind the C ABI of
``include/grp.h``; ``binding`` is its thin ctypes layer.  Importing this package loads nothing:
``workloads`` (seeded synthetic inputs) stays importable on hosts without the library.
"""
__all__ = ["workloads", "binding"]
