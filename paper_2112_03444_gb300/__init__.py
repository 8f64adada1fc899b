"""GB300-native homotopy-continuation path tracker.

Submodules are imported lazily: ``inputs`` (seeded synthetic problem data)
needs neither CUDA nor the native library; ``hc`` is the thin ctypes binding
of the C-ABI in ``include/hc.h`` and fails loudly if ``libhc.so`` is missing.
"""
__all__ = ["inputs", "hc"]
