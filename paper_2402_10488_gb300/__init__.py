"""GB300-native ROM-enhanced SISA for the parametric radiative transfer equation.

The compute path lives in the CUDA library built from ``csrc/`` (C ABI declared in
``include/rte.h``); ``rte`` is its thin ctypes binding.  ``inputs`` holds the seeded problem
descriptions.  Importing this package does not load the library; ``rte.lib()`` does, and fails
loudly when the compiled library is missing.
"""
