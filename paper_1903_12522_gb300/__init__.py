"""GB300-native controllability CG (CMCG) solver for the Helmholtz equation.

The compute path is the CUDA shared library ``libcmcg.so`` (sources in ``csrc/``, C ABI in
``include/cmcg.h``); ``cmcg.py`` is a thin ctypes binding with the same entry points.
Importing this package does not load the library; ``cmcg.load()`` does, and raises if the
library has not been built.
"""
