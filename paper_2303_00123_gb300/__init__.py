"""GB300-native state-vector gate engine (QCLAB++, arXiv 2303.00123).

The compute path lives in the CUDA shared library built from ``csrc/`` and is
reached through the C ABI declared in ``include/qcgb300.h``; ``qcgb300`` is its
thin ctypes binding.  ``circuits`` builds seeded synthetic inputs.
"""
__all__ = ["circuits", "qcgb300"]
