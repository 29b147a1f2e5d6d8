"""GB300-native spherical harmonic transforms on the optimal-dimensionality sampling.

The transforms run in the CUDA library ``libsht.so`` (built from ``csrc/``) behind the C ABI
declared in ``include/sht.h``; ``sht`` is the thin Python binding.  Importing the package does not
load the library; the first call into ``sht`` does, and fails loudly if it is missing.
"""
