"""GB300-native round-synchronous contraction hierarchies (arXiv 2412.18008).

``ch`` is the binding of the CUDA library (``include/ch.h``), ``inputs`` the
seeded synthetic graph generators. Importing the package loads nothing; the
library is loaded (and built in-tree if needed) on first use.
"""
__all__ = ["ch", "inputs", "build"]
