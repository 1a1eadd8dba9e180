"""GB300-native over-relaxed diffusive integer lattice gas.

The compute path is the CUDA library ``libilg.so`` (sources in ``csrc/``, C
declarations in ``include/ilg.h``).  ``binding`` loads it with ctypes and fails
loudly when it is missing; ``inputs`` holds the seeded synthetic inputs.
Importing the package itself loads nothing.
"""
